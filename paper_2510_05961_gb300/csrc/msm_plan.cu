// msm_plan.cu -- host planner of the GB300 MSM library (FP64): grid counts
// and level ranges, softening coefficients, restriction coefficients,
// quasi-interpolation coefficients, the level stencils K^l and their strain
// derivatives, the work lists of every kernel and the workspace layout.
//
// Paper passages: level set-up of periodic cells (Sec. 4.1: spacing doubles
// until one point remains), splitting and softening (Sec. 3.4, Eq.
// coulomb_splitting_with_softener), restriction coefficients (Eq.
// restriction_prolongation_explicit_formulas), stencils (Eq.
// kernel_stencil_by_conv_with_universal_coeff; K^l = K^1 / 2^(l-1) for the
// intermediate levels, Sec. 3.4).
#include "msm_plan.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <cstring>

namespace msm {

// ------------------------------------------------------------------ math
// Softening gamma(rho) (Sec. 3.4): 1/rho for rho >= 1, else the Taylor
// polynomial of s^-1/2 about s = 1 to degree p-1, at s = rho^2. In the
// variable t = 1 - rho^2 it reads sum_k c_k t^k with c_0 = 1,
// c_k = c_(k-1) (2k - 1) / (2k).
static void softening_coeffs(int p, double* c) {
  c[0] = 1.0;
  for (int k = 1; k < p; k++) c[k] = c[k - 1] * (2.0 * k - 1.0) / (2.0 * k);
}

static double soft(int p, double rho) {
  if (rho >= 1.0) return 1.0 / rho;
  double c[8];
  softening_coeffs(p, c);
  double t = 1.0 - rho * rho, v = c[p - 1];
  for (int k = p - 2; k >= 0; k--) v = v * t + c[k];
  return v;
}

static double soft_d(int p, double rho) {  // d gamma / d rho
  if (rho >= 1.0) return -1.0 / (rho * rho);
  double c[8];
  softening_coeffs(p, c);
  double t = 1.0 - rho * rho, v = (p - 1) * c[p - 1];
  for (int k = p - 2; k >= 1; k--) v = v * t + k * c[k];
  return -2.0 * rho * v;
}

// grid-level partial kernel k_l (l >= 1) and its r-derivative
static double klev(const SysHost& S, int l, double r, bool deriv) {
  double s1 = S.a * std::ldexp(1.0, l - 1);
  if (l == S.nlev) return deriv ? soft_d(S.p, r / s1) / (s1 * s1) : soft(S.p, r / s1) / s1;
  double s2 = 2.0 * s1;
  if (r >= s2) return 0.0;
  if (deriv) return soft_d(S.p, r / s1) / (s1 * s1) - soft_d(S.p, r / s2) / (s2 * s2);
  return soft(S.p, r / s1) / s1 - soft(S.p, r / s2) / s2;
}

// ------------------------------------------------------------------ slab top level
// A slab (x, y periodic, z open) keeps its top level, whose grid has one point
// per period along x and y: the level-L kernel k_L summed over the 2-D lattice
// R = (i Lx, j Ly, 0) at the pure z offset. The sum of the 1/r tail diverges
// by a constant that multiplies the squared total charge (zero for neutral
// systems) and is left out; what remains is split the Ewald way:
//   sum_R k_L = sum_R [erfc(al s)/s - h_L(s)] + (pi/A) sum_(G != 0) (1/|G|) [u(G, z) + u(G, -z)]
//               - (2 pi/A) [z erf(al z) + exp(-al^2 z^2)/(al sqrt(pi))],
// s = |R + z e_z|, h_L(s) = 1/s - gamma(s/a_L)/a_L (zero beyond a_L),
// u(G, z) = e^(|G| z) erfc(|G|/(2 al) + al z), G = 2 pi (i/Lx, j/Ly), A = Lx Ly.
// At z = 0 the R = 0 term is its limit -2 al/sqrt(pi) + gamma(0)/a_L.

// e^(g z) erfc(g/(2 al) + al z) without overflow (scaled erfc for large arguments)
static double slab_u(double g, double z, double al) {
  const double x = g / (2.0 * al) + al * z;
  if (x <= 0.0) return std::exp(g * z) * std::erfc(x);
  double sc;  // e^(x^2) erfc(x)
  if (x < 10.0) {
    sc = std::exp(x * x) * std::erfc(x);
  } else {
    double term = 1.0, sum = 1.0;
    const double inv = 0.5 / (x * x);
    for (int k = 1; k <= 12; k++) {
      term *= -(2.0 * k - 1.0) * inv;
      sum += term;
    }
    sc = sum / (x * std::sqrt(M_PI));
  }
  return std::exp(-g * g / (4.0 * al * al) - al * al * z * z) * sc;
}

static double slab_top_kernel(const SysHost& S, double Lx, double Ly, double z) {
  const double aL = S.a * std::ldexp(1.0, S.nlev - 1);
  const double al = 6.0 / std::min(Lx, Ly), A = Lx * Ly;
  const double rc = 7.0 / al, gc = 14.0 * al;
  const bool at0 = std::fabs(z) < 1e-300;
  double v = 0.0;
  const int ni = (int)std::ceil(std::max(rc, aL) / Lx) + 1, nj = (int)std::ceil(std::max(rc, aL) / Ly) + 1;
  for (int i = -ni; i <= ni; i++)
    for (int j = -nj; j <= nj; j++) {
      if (at0 && i == 0 && j == 0) continue;
      const double sx = i * Lx, sy = j * Ly;
      const double sd = std::sqrt(sx * sx + sy * sy + z * z);
      if (sd < rc) v += std::erfc(al * sd) / sd;
      if (sd < aL) v -= 1.0 / sd - soft(S.p, sd / aL) / aL;
    }
  if (at0) v += -2.0 * al / std::sqrt(M_PI) + soft(S.p, 0.0) / aL;
  const int mi = (int)std::ceil(gc * Lx / (2.0 * M_PI)) + 1, mj = (int)std::ceil(gc * Ly / (2.0 * M_PI)) + 1;
  double rec = 0.0;
  for (int i = -mi; i <= mi; i++)
    for (int j = -mj; j <= mj; j++) {
      if (i == 0 && j == 0) continue;
      const double gx = 2.0 * M_PI * i / Lx, gy = 2.0 * M_PI * j / Ly;
      const double g = std::sqrt(gx * gx + gy * gy);
      if (g >= gc) continue;
      rec += (slab_u(g, z, al) + slab_u(g, -z, al)) / g;
    }
  v += M_PI / A * rec;
  v -= 2.0 * M_PI / A * (z * std::erf(al * z) + std::exp(-al * al * z * z) / (al * std::sqrt(M_PI)));
  return v;
}

// ------------------------------------------------------------------ wire top level
// A wire (one periodic axis, period Lw; the other two open) keeps its top
// level as well, one point per period along the wire: k_L summed over the
// 1-D lattice n Lw e at the transverse distance rho. The 1/r tail diverges
// logarithmically, by a constant that multiplies the squared total charge
// and is left out. Split:
//   sum_n k_L = sum_n [erfc(al s_n)/s_n - h_L(s_n)] + (2/Lw) sum_(k >= 1) F(G_k, rho)
//               + (1/Lw) [-gamma_E - ln rho^2 - E1(al^2 rho^2)],
// s_n = |(rho, n Lw)|, G_k = 2 pi k / Lw, F(G, rho) = int_0^(al^2) exp(-u rho^2
// - G^2/(4u)) du/u (the transform along the wire of erf(al r)/r). At rho = 0
// the bracket is ln al^2, F(G, 0) = E1(G^2/(4 al^2)) and the n = 0 term is the
// limit -2 al/sqrt(pi) + gamma(0)/a_L.
namespace {
constexpr double kEulerGamma = 0.5772156649015328606;

// 16-point Gauss-Legendre nodes and weights on [-1, 1] (Newton on the
// Legendre recurrence)
struct GaussLegendre16 {
  double x[16], w[16];
  GaussLegendre16() {
    const int n = 16;
    for (int i = 0; i < n; i++) {
      double t = std::cos(M_PI * (i + 0.75) / (n + 0.5)), d = 1.0;
      for (int it = 0; it < 60; it++) {
        double pm = 1.0, pc = t;
        for (int k = 2; k <= n; k++) {
          const double pn = ((2 * k - 1) * t * pc - (k - 1) * pm) / k;
          pm = pc;
          pc = pn;
        }
        d = n * (t * pc - pm) / (t * t - 1.0);
        const double step = pc / d;
        t -= step;
        if (std::fabs(step) < 1e-16) break;
      }
      x[i] = t;
      w[i] = 2.0 / ((1.0 - t * t) * d * d);
    }
  }
};
}  // namespace

static double wire_F(double G, double rho, double al) {
  const double b = G * G / (4.0 * al * al);
  if (b > 50.0) return 0.0;
  if (rho == 0.0) return -std::expint(-b);  // E1(b)
  // u = al^2 e^-t: int_0^inf exp(-al^2 rho^2 e^-t - b e^t) dt, cut at b e^t = 50,
  // panels of width <= 0.4
  static const GaussLegendre16 gl;
  const double c = al * al * rho * rho, tmax = std::log(50.0 / b);
  const int np = std::max(1, (int)std::ceil(tmax / 0.4));
  const double half = 0.5 * tmax / np;
  double acc = 0.0;
  for (int k = 0; k < np; k++)
    for (int i = 0; i < 16; i++) {
      const double t = (2 * k + 1) * half + half * gl.x[i];
      acc += gl.w[i] * std::exp(-c * std::exp(-t) - b * std::exp(t));
    }
  return acc * half;
}

static double wire_top_kernel(const SysHost& S, double Lw, double rho) {
  const double aL = S.a * std::ldexp(1.0, S.nlev - 1);
  const double al = 5.0 / Lw, rc = 7.0 / al;
  const bool at0 = rho < 1e-300;
  double v = 0.0;
  const int nn = (int)std::ceil(std::max(rc, aL) / Lw) + 1;
  for (int n = -nn; n <= nn; n++) {
    if (at0 && n == 0) continue;
    const double z = n * Lw, sd = std::sqrt(rho * rho + z * z);
    if (sd < rc) v += std::erfc(al * sd) / sd;
    if (sd < aL) v -= 1.0 / sd - soft(S.p, sd / aL) / aL;
  }
  if (at0) v += -2.0 * al / std::sqrt(M_PI) + soft(S.p, 0.0) / aL;
  double rec = 0.0;
  for (int k = 1;; k++) {
    const double G = 2.0 * M_PI * k / Lw;
    if (G * G / (4.0 * al * al) > 50.0) break;
    rec += wire_F(G, rho, al);
  }
  v += 2.0 / Lw * rec;
  const double x = al * al * rho * rho;
  v += (at0 ? std::log(al * al) : -kEulerGamma - std::log(rho * rho) + std::expint(-x)) / Lw;  // Ei(-x) = -E1(x)
  return v;
}

// Top level of a partially periodic system (one or two periodic axes): k_L
// summed over the lattice of the periodic axes, Lp the periods (entries of
// open axes unused), v the sample vector; offsets along periodic axes are
// lattice vectors there, so only the open components enter.
static double lattice_top_kernel(const SysHost& S, const double Lp[3], const double v[3]) {
  int per[3], opn[3], np = 0, no = 0;
  for (int d = 0; d < 3; d++) {
    if (S.pbc[d])
      per[np++] = d;
    else
      opn[no++] = d;
  }
  if (np == 2) return slab_top_kernel(S, Lp[per[0]], Lp[per[1]], v[opn[0]]);
  return wire_top_kernel(S, Lp[per[0]], std::hypot(v[opn[0]], v[opn[1]]));
}

// strain derivatives (comp 1..6 = xx, yy, zz, xy, xz, yz): lattice and offset
// strained by (1 + eps E_ab), central differences. A diagonal strain of a
// periodic axis scales its period, of an open axis the offset; a shear that
// involves a periodic axis leaves the sum unchanged to first order (it is
// even under the mirror of that axis); a shear of the two open axes of a
// wire moves the offset.
static double lattice_top_deps(const SysHost& S, const double v[3], int comp) {
  static const int AB[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  const int a = AB[comp - 1][0], b = AB[comp - 1][1];
  if (a != b && (S.pbc[a] || S.pbc[b])) return 0.0;
  const double e = 1e-5;
  double f[2];
  for (int k = 0; k < 2; k++) {
    const double sg = k == 0 ? e : -e;
    double Lp[3] = {S.L[0], S.L[1], S.L[2]}, w[3] = {v[0], v[1], v[2]};
    if (a == b && S.pbc[a])
      Lp[a] *= 1.0 + sg;
    else
      w[a] += sg * v[b];
    f[k] = lattice_top_kernel(S, Lp, w);
  }
  return (f[0] - f[1]) / (2.0 * e);
}

// Pieces of the centred B-spline Phi_p(t) = N_p(t + p/2), N_p the cardinal
// B-spline on [0, p): out[i][k] is the coefficient of s^k of Phi_p(i + s),
// s in [0, 1), i = 0 .. p/2 - 1. Built from N_1 = 1 on [0, 1) by the
// recursion N_m(x) = (x N_(m-1)(x) + (m - x) N_(m-1)(x - 1)) / (m - 1) applied
// to the polynomial of each unit interval in its local variable.
static void bspline_pieces(int p, double out[4][8]) {
  double cur[8][8] = {{1.0}}, nxt[8][8];
  for (int m = 2; m <= p; m++) {
    for (int j = 0; j < m; j++) {
      for (int k = 0; k < 8; k++) nxt[j][k] = 0.0;
      // (j + s) N_(m-1) on interval j, plus (m - j - s) N_(m-1) on interval j - 1
      for (int k = 0; k + 1 < m; k++) {
        const double a = (j < m - 1) ? cur[j][k] : 0.0;
        const double b = (j >= 1) ? cur[j - 1][k] : 0.0;
        nxt[j][k] += j * a + (m - j) * b;
        nxt[j][k + 1] += a - b;
      }
      for (int k = 0; k < m; k++) nxt[j][k] /= (m - 1);
    }
    for (int j = 0; j < m; j++)
      for (int k = 0; k < 8; k++) cur[j][k] = nxt[j][k];
  }
  for (int i = 0; i < 4; i++)
    for (int k = 0; k < 8; k++) out[i][k] = (i < p / 2 && k < p) ? cur[p / 2 + i][k] : 0.0;
}

// qi_mode 1: omega' = omega * omega, omega the inverse of the sampled
// B-spline b_n = Phi_p(n). omega solves the banded symmetric Toeplitz system
// T omega = e_0 on a window of 2W + 1 points by Gaussian elimination without
// pivoting (T is positive definite: its symbol is the B-spline sampling
// symbol, > 0); omega decays like |z_1|^|n| with |z_1| <= 0.54 (the root of
// the sampling polynomial nearest the unit circle, p <= 8), so the window
// edges do not reach the centre. Kept: |n| <= hw, hw the largest n with
// |omega'_n| >= 1e-12 |omega'_0|.
static int exact_omega(int p, std::vector<double>& omh) {
  double pc[4][8];
  bspline_pieces(p, pc);
  const int H = p / 2, bw = H - 1, nb = 2 * bw + 1;
  double b[4];
  for (int m = 0; m < H; m++) b[m] = pc[m][0];  // Phi_p(m): piece m at its left end
  const int W = 240, N = 2 * W + 1;
  std::vector<double> A((size_t)N * nb, 0.0), x(N, 0.0);
  auto at = [&](int i, int j) -> double& { return A[(size_t)i * nb + (j - i + bw)]; };
  for (int i = 0; i < N; i++)
    for (int j = std::max(0, i - bw); j <= std::min(N - 1, i + bw); j++) at(i, j) = b[std::abs(i - j)];
  x[W] = 1.0;
  for (int k = 0; k < N; k++)
    for (int i = k + 1; i <= std::min(N - 1, k + bw); i++) {
      const double f = at(i, k) / at(k, k);
      for (int j = k; j <= std::min(N - 1, k + bw); j++) at(i, j) -= f * at(k, j);
      x[i] -= f * x[k];
    }
  for (int k = N - 1; k >= 0; k--) {
    double s = x[k];
    for (int j = k + 1; j <= std::min(N - 1, k + bw); j++) s -= at(k, j) * x[j];
    x[k] = s / at(k, k);
  }
  const int nmax = 120;
  std::vector<double> wp(nmax + 1, 0.0);
  for (int n = 0; n <= nmax; n++) {
    double s = 0.0;
    for (int k = -W; k <= W; k++) {
      const int j = n - k;
      if (j >= -W && j <= W) s += x[k + W] * x[j + W];
    }
    wp[n] = s;
  }
  int hw = 0;
  for (int n = 0; n <= nmax; n++)
    if (std::abs(wp[n]) >= 1e-12 * std::abs(wp[0])) hw = n;
  omh.assign(wp.begin(), wp.begin() + hw + 1);
  return hw;
}

// omega'_0 .. omega'_(p/2-1) (symmetric), exact rationals: the shortest
// symmetric sequence whose symbol times the squared B-spline sampling symbol
// is 1 + O(theta^p) (equivalently, 1-D kernel interpolation reproduces
// polynomials of degree < p).
static void omega_half(int p, double* w) {
  switch (p) {
    case 4: w[0] = 5.0 / 3.0; w[1] = -1.0 / 3.0; break;
    case 6: w[0] = 121.0 / 40.0; w[1] = -71.0 / 60.0; w[2] = 41.0 / 240.0; break;
    default:
      w[0] = 5674.0 / 945.0; w[1] = -8261.0 / 2520.0; w[2] = 551.0 / 630.0; w[3] = -149.0 / 1512.0; break;
  }
}

// ------------------------------------------------------------------ stencils
// Dense 3-D array with an index origin: value at offset (x,y,z) stored at
// ((x-o0)*s1 + (y-o1))*s2 + (z-o2).
struct Box3 {
  int o[3], s[3];
  std::vector<double> v;
  void init(const int lo[3], const int sz[3]) {
    for (int d = 0; d < 3; d++) { o[d] = lo[d]; s[d] = sz[d]; }
    v.assign((size_t)s[0] * s[1] * s[2], 0.0);
  }
  double& at(int x, int y, int z) { return v[((size_t)(x - o[0]) * s[1] + (y - o[1])) * s[2] + (z - o[2])]; }
};

// K_m = sum_t omega'_tx omega'_ty omega'_tz sample(m - t) on the output box
// [-E, E] (per axis), sample(n) = f(h o n) for the level spacing hl. comp = 0:
// k_l(|v|); comp 1..6: k_l'(|v|) v_a v_b / |v| with ab = xx,yy,zz,xy,xz,yz.
static void build_stencil(const SysHost& S, int l, const int E[3], int comp, Box3& out) {
  const int npbc = S.pbc[0] + S.pbc[1] + S.pbc[2];
  const bool lat_top = l == S.nlev && npbc >= 1 && npbc <= 2;  // slab or wire top level
  const int r = S.hw;
  const std::vector<double>& wh = S.omh;
  double hl[3];
  for (int d = 0; d < 3; d++) hl[d] = S.h1[d] * std::ldexp(1.0, l - 1);
  static const int AB[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  int slo[3], ssz[3], olo[3], osz[3];
  for (int d = 0; d < 3; d++) {
    slo[d] = -E[d] - r;
    ssz[d] = 2 * (E[d] + r) + 1;
    olo[d] = -E[d];
    osz[d] = 2 * E[d] + 1;
  }
  Box3 smp;
  smp.init(slo, ssz);
  // the lattice-summed top level depends on the open components alone:
  // samples that differ only along periodic axes share one evaluation
  std::map<std::array<double, 3>, double> lat_memo;
  for (int x = slo[0]; x < slo[0] + ssz[0]; x++)
    for (int y = slo[1]; y < slo[1] + ssz[1]; y++)
      for (int z = slo[2]; z < slo[2] + ssz[2]; z++) {
        double v[3] = {hl[0] * x, hl[1] * y, hl[2] * z};
        if (S.tri) {
          // tilted cell: the index step n is the vector sum_d n_d 2^(l-1) / M_d a_d
          const double f[3] = {std::ldexp((double)x, l - 1) / S.M[0], std::ldexp((double)y, l - 1) / S.M[1],
                               std::ldexp((double)z, l - 1) / S.M[2]};
          for (int c = 0; c < 3; c++) v[c] = f[0] * S.A[c] + f[1] * S.A[3 + c] + f[2] * S.A[6 + c];
        }
        double rr = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double val;
        if (lat_top) {
          const std::array<double, 3> key = {S.pbc[0] ? 0.0 : v[0], S.pbc[1] ? 0.0 : v[1], S.pbc[2] ? 0.0 : v[2]};
          auto hit = lat_memo.find(key);
          if (hit != lat_memo.end()) {
            val = hit->second;
          } else {
            val = comp == 0 ? lattice_top_kernel(S, S.L, key.data()) : lattice_top_deps(S, key.data(), comp);
            lat_memo.emplace(key, val);
          }
          smp.at(x, y, z) = val;
          continue;
        }
        if (comp == 0) {
          val = klev(S, l, rr, false);
        } else {
          int a = AB[comp - 1][0], b = AB[comp - 1][1];
          val = rr > 0.0 ? klev(S, l, rr, true) * v[a] * v[b] / rr : 0.0;
        }
        smp.at(x, y, z) = val;
      }
  auto om = [&](int t) { return wh[t < 0 ? -t : t]; };
  // separable passes: z, then y, then x
  int alo[3] = {slo[0], slo[1], olo[2]}, asz[3] = {ssz[0], ssz[1], osz[2]};
  Box3 A;
  A.init(alo, asz);
  for (int x = slo[0]; x < slo[0] + ssz[0]; x++)
    for (int y = slo[1]; y < slo[1] + ssz[1]; y++)
      for (int z = olo[2]; z < olo[2] + osz[2]; z++) {
        double acc = 0.0;
        for (int t = -r; t <= r; t++) acc += om(t) * smp.at(x, y, z - t);
        A.at(x, y, z) = acc;
      }
  int blo[3] = {slo[0], olo[1], olo[2]}, bsz[3] = {ssz[0], osz[1], osz[2]};
  Box3 B;
  B.init(blo, bsz);
  for (int x = slo[0]; x < slo[0] + ssz[0]; x++)
    for (int y = olo[1]; y < olo[1] + osz[1]; y++)
      for (int z = olo[2]; z < olo[2] + osz[2]; z++) {
        double acc = 0.0;
        for (int t = -r; t <= r; t++) acc += om(t) * A.at(x, y - t, z);
        B.at(x, y, z) = acc;
      }
  out.init(olo, osz);
  for (int x = olo[0]; x < olo[0] + osz[0]; x++)
    for (int y = olo[1]; y < olo[1] + osz[1]; y++)
      for (int z = olo[2]; z < olo[2] + osz[2]; z++) {
        double acc = 0.0;
        for (int t = -r; t <= r; t++) acc += om(t) * B.at(x - t, y, z);
        out.at(x, y, z) = acc;
      }
}

// Raw kernel samples on [-E, E] (per axis), without the omega' convolution:
// comp 0: k_l(|v|); comp 1..6: k_l'(|v|) v_a v_b / |v|, v = h_l o n.
static void build_samples(const SysHost& S, int l, const int E[3], int comp, Box3& out) {
  double hl[3];
  for (int d = 0; d < 3; d++) hl[d] = S.h1[d] * std::ldexp(1.0, l - 1);
  static const int AB[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  int lo[3], sz[3];
  for (int d = 0; d < 3; d++) {
    lo[d] = -E[d];
    sz[d] = 2 * E[d] + 1;
  }
  out.init(lo, sz);
  for (int x = -E[0]; x <= E[0]; x++)
    for (int y = -E[1]; y <= E[1]; y++)
      for (int z = -E[2]; z <= E[2]; z++) {
        double v[3] = {hl[0] * x, hl[1] * y, hl[2] * z};
        if (S.tri) {
          const double f[3] = {std::ldexp((double)x, l - 1) / S.M[0], std::ldexp((double)y, l - 1) / S.M[1],
                               std::ldexp((double)z, l - 1) / S.M[2]};
          for (int c = 0; c < 3; c++) v[c] = f[0] * S.A[c] + f[1] * S.A[3 + c] + f[2] * S.A[6 + c];
        }
        double rr = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double val;
        if (comp == 0) {
          val = klev(S, l, rr, false);
        } else {
          int a = AB[comp - 1][0], b = AB[comp - 1][1];
          val = rr > 0.0 ? klev(S, l, rr, true) * v[a] * v[b] / rr : 0.0;
        }
        out.at(x, y, z) = val;
      }
}

// fold the periodic axes of an unfolded box onto [0, n) and scale
static void fold(const Box3& in, const int n[3], const int per[3], double scale, Box3& out) {
  int lo[3], sz[3];
  for (int d = 0; d < 3; d++) {
    lo[d] = per[d] ? 0 : in.o[d];
    sz[d] = per[d] ? n[d] : in.s[d];
  }
  out.init(lo, sz);
  for (int x = 0; x < in.s[0]; x++)
    for (int y = 0; y < in.s[1]; y++)
      for (int z = 0; z < in.s[2]; z++) {
        int m[3] = {x + in.o[0], y + in.o[1], z + in.o[2]}, f[3];
        for (int d = 0; d < 3; d++) {
          if (per[d]) {
            int rr = m[d] % n[d];
            f[d] = rr < 0 ? rr + n[d] : rr;
          } else {
            f[d] = m[d];
          }
        }
        out.at(f[0], f[1], f[2]) += scale * in.v[((size_t)x * in.s[1] + y) * in.s[2] + z];
      }
}

// Stencil values of a planned system for its current spacings h_1: K^1 and
// its strain derivatives, the folded boxes of the box levels, the ball
// samples, virial weights and column half-widths. With decide set it also
// chooses each level's kernel (ball or box) and radius; without, the kinds,
// radii and array sizes of the plan are kept (a new cell for an existing plan).
static void fill_stencils(SysHost& S, bool decide) {
  // level-1 shape stencil K^1 (intermediate levels are K^1 / 2^(l-1)) and its
  // strain derivatives; the ball kernels apply the raw samples s^1 instead,
  // to the omega'-prefiltered grid: K * q = (omega'^3 * s) * q = s * (omega'^3 * q)
  const bool any_mid = S.ncomp >= 1 && S.nlev > 1;
  if (decide) S.has_ball = false;
  Box3 K1, dK1[6];
  if (any_mid) {
    build_stencil(S, 1, S.R, 0, K1);
    for (int c = 0; c < 6; c++) build_stencil(S, 1, S.R, c + 1, dK1[c]);
  }
  for (int l = 1; l <= S.ncomp; l++) {
    LevelHost& Lv = S.lev[l - 1];
    Lv.scale = (float)std::ldexp(1.0, -(l - 1));
    bool top = (l == S.nlev);
    // ball kernels are compiled for radii up to kBallRmax; larger stencils use
    // the box kernel. A ball that overlaps itself on a small periodic grid is
    // still applied as a ball: its halo holds the periodic images (wrapped
    // more than once where the grid is shorter than the halo), which sums
    // every image of each offset exactly as the folded stencil does.
    if (decide) {
      // exact interpolation: dense boxes (wide stencils, accuracy reference)
      bool ball = !top && S.qi_mode == 0 && S.allow_ball;
      for (int d = 0; d < 3; d++)
        if (S.B[d] > kBallRmax) ball = false;
      // batch plans: a level of a few hundred points costs a ball kernel a whole
      // 32 x 32 tile per x-plane and a halo-padded copy much larger than itself;
      // folded onto the grid, its dense box has at most n^3 entries per point.
      // (Single-system plans keep every level a ball, which msm_plan_set_cell
      // can recompute on the device.)
      if (S.fold_small && (long long)Lv.n[0] * Lv.n[1] * Lv.n[2] <= kFoldPts) ball = false;
      for (int d = 0; d < 3; d++) Lv.R[d] = S.B[d];
      if (ball) {
        Lv.kind = 0;
        S.has_ball = true;
        continue;
      }
      Lv.kind = 1;
      for (int d = 0; d < 3; d++) Lv.R[d] = S.R[d];
    } else if (Lv.kind == 0) {
      continue;
    }
    Box3 Kf, dKf[6];
    if (top) {
      int E[3];
      for (int d = 0; d < 3; d++) E[d] = Lv.n[d] - 1;
      Box3 Kt, dKt[6];
      build_stencil(S, l, E, 0, Kt);
      for (int c = 0; c < 6; c++) build_stencil(S, l, E, c + 1, dKt[c]);
      fold(Kt, Lv.n, Lv.per, 1.0, Kf);
      for (int c = 0; c < 6; c++) fold(dKt[c], Lv.n, Lv.per, 1.0, dKf[c]);
    } else {
      double sc = std::ldexp(1.0, -(l - 1));
      fold(K1, Lv.n, Lv.per, sc, Kf);
      for (int c = 0; c < 6; c++) fold(dK1[c], Lv.n, Lv.per, sc, dKf[c]);
    }
    Lv.scale = 1.0f;
    for (int d = 0; d < 3; d++) {
      Lv.blo[d] = Kf.o[d];
      Lv.bsz[d] = Kf.s[d];
    }
    Lv.kbox.assign(Kf.v.begin(), Kf.v.end());
    Lv.dkbox.clear();
    for (int c = 0; c < 6; c++) Lv.dkbox.insert(Lv.dkbox.end(), dKf[c].v.begin(), dKf[c].v.end());
  }
  if (any_mid) {
    S.kball.assign(K1.v.begin(), K1.v.end());
    S.dk1.clear();
    for (int c = 0; c < 6; c++) S.dk1.insert(S.dk1.end(), dK1[c].v.begin(), dK1[c].v.end());
  }
  if (S.has_ball) {
    Box3 s1, ds1[6];
    if (S.prefilter) {
      build_samples(S, 1, S.B, 0, s1);
      for (int c = 0; c < 6; c++) build_samples(S, 1, S.B, c + 1, ds1[c]);
    } else {
      s1 = K1;
      for (int c = 0; c < 6; c++) ds1[c] = dK1[c];
    }
    const int nx = 2 * S.B[0] + 1, ny = 2 * S.B[1] + 1, nz = 2 * S.B[2] + 1;
    S.sball.assign(s1.v.begin(), s1.v.end());
    S.dsh.assign((size_t)6 * nx * ny * nz, 0.0f);
    S.fsh.assign(S.prefilter ? (size_t)nx * ny * nz : 0, 0.0f);
    // Column centres: zero for rectangular cells (every column is even in dz);
    // a tilted cell's column (dx, dy) holds its samples on an interval around
    // a shifted centre, taken here as the midpoint of the nonzero samples
    // (of K and of the virial weights) rounded down to a multiple of 4, so the
    // kernels' 16-byte row loads stay aligned after the shift.
    S.cball.assign((size_t)nx * ny, 0);
    if (S.tri)
      for (int x = -S.B[0]; x <= S.B[0]; x++)
        for (int y = -S.B[1]; y <= S.B[1]; y++) {
          int lo = 1 << 30, hi = -(1 << 30);
          for (int z = -S.B[2]; z <= S.B[2]; z++) {
            size_t at = ((size_t)(x + S.B[0]) * ny + (y + S.B[1])) * nz + (z + S.B[2]);
            bool nz0 = (float)s1.v[at] != 0.0f;
            for (int c = 0; c < 6 && !nz0; c++) nz0 = (float)ds1[c].v[at] != 0.0f;
            if (nz0) {
              lo = std::min(lo, z);
              hi = std::max(hi, z);
            }
          }
          int cen = lo <= hi ? (lo + hi) / 2 : 0;
          cen = (cen >= 0 ? cen : cen - 3) / 4 * 4;  // round down to a multiple of 4
          S.cball[(size_t)(x + S.B[0]) * ny + (y + S.B[1])] = cen;
        }
    // column half-widths about the centre, rounded up to even values (the
    // stored rows are zero beyond the support): half as many unrolled variants
    S.wball.assign((size_t)nx * ny, -1);
    S.whalf.assign((size_t)nx * ny, -1);
    for (int x = -S.B[0]; x <= S.B[0]; x++)
      for (int y = -S.B[1]; y <= S.B[1]; y++)
        for (int z = -S.B[2]; z <= S.B[2]; z++) {
          size_t at = ((size_t)(x + S.B[0]) * ny + (y + S.B[1])) * nz + (z + S.B[2]);
          size_t col = (size_t)(x + S.B[0]) * ny + (y + S.B[1]);
          const int zc = std::abs(z - S.cball[col]);
          if ((float)s1.v[at] != 0.0f) S.wball[col] = std::max(S.wball[col], zc + (zc & 1));
          // half-space weights: C'_d = C'_-d, so sum_d ds_d C'_d = ds_0 C'_0 + 2 sum_(d in half) ds_d C'_d
          bool half = x > 0 || (x == 0 && y > 0) || (x == 0 && y == 0 && z > 0);
          bool zero = x == 0 && y == 0 && z == 0;
          double f = half ? 2.0 : (zero ? 1.0 : 0.0);
          bool any = false;
          for (int c = 0; c < 6; c++) {
            float v = (float)(f * ds1[c].v[at]);
            S.dsh[(size_t)c * nx * ny * nz + at] = v;
            if (v != 0.0f) any = true;
          }
          if (S.prefilter && !S.tri) {
            // raw samples factor: ds_ab(n) = g(n) v_a v_b with g = k_1'(|v|)/|v|, v = h_1 o n
            const double vx = S.h1[0] * x, vy = S.h1[1] * y, vz = S.h1[2] * z;
            const double rr = std::sqrt(vx * vx + vy * vy + vz * vz);
            const float g = rr > 0.0 ? (float)(f * klev(S, 1, rr, true) / rr) : 0.0f;
            S.fsh[at] = g;
            any = g != 0.0f;
          }
          if (any) S.whalf[col] = std::max(S.whalf[col], zc + (zc & 1));
        }
    // z halo of the padded grid and of the stored rows: every shifted window
    // (centre +- the 4-rounded half-width) must stay inside it
    S.hzb = (S.B[2] + 3) & ~3;
    S.wmax = 0;
    for (size_t col = 0; col < S.cball.size(); col++) {
      const int w = std::max(S.wball[col], S.whalf[col]);
      if (w < 0) continue;
      S.wmax = std::max(S.wmax, w);
      if (S.tri) S.hzb = std::max(S.hzb, (std::abs(S.cball[col]) + ((w + 3) & ~3) + 3) & ~3);
    }
  }
}

// ------------------------------------------------------------------ planning
static int fail(std::string* err, int code, const char* msg) {
  if (err) *err = msg;
  return code;
}

// 3x3 inverse by cofactors; returns the determinant
static double inv3(const double* m, double* inv) {
  const double c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8], c02 = m[3] * m[7] - m[4] * m[6];
  const double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
  inv[0] = c00 / det;
  inv[1] = (m[2] * m[7] - m[1] * m[8]) / det;
  inv[2] = (m[1] * m[5] - m[2] * m[4]) / det;
  inv[3] = c01 / det;
  inv[4] = (m[0] * m[8] - m[2] * m[6]) / det;
  inv[5] = (m[2] * m[3] - m[0] * m[5]) / det;
  inv[6] = c02 / det;
  inv[7] = (m[1] * m[6] - m[0] * m[7]) / det;
  inv[8] = (m[0] * m[4] - m[1] * m[3]) / det;
  return det;
}

int plan_system(const msm_params& P, SysHost& S, std::string* err) {
  S.tri = false;
  for (int i = 0; i < 9; i++) {
    if (!std::isfinite(P.cell[i])) return fail(err, MSM_ERR_INVALID_ARG, "cell has a non-finite entry");
    if (i % 4 != 0 && P.cell[i] != 0.0) S.tri = true;
  }
  for (int i = 0; i < 9; i++) S.A[i] = P.cell[i];
  double det = 0.0;
  if (S.tri) {
    // a tilted cell (Sec. 3.2.2's transform to the unit cube): periodic only
    if (!(P.pbc[0] == 1 && P.pbc[1] == 1 && P.pbc[2] == 1))
      return fail(err, MSM_ERR_UNSUPPORTED, "a non-orthorhombic cell must be periodic along all three axes");
    det = inv3(S.A, S.Ainv);
    if (!(det > 0.0)) return fail(err, MSM_ERR_INVALID_ARG, "cell rows must form a right-handed basis");
  } else {
    for (int i = 0; i < 9; i++) S.Ainv[i] = 0.0;
    for (int d = 0; d < 3; d++) S.Ainv[4 * d] = 1.0 / P.cell[4 * d];
  }
  {
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) S.Tinv[3 * i + j] = S.Ainv[3 * j + i];
    for (int d = 0; d < 3; d++) {
      if (!S.tri) {
        S.wplane[d] = P.cell[4 * d];
        continue;
      }
      const double* u = S.A + 3 * ((d + 1) % 3);
      const double* v = S.A + 3 * ((d + 2) % 3);
      const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
      S.wplane[d] = det / std::sqrt(cx * cx + cy * cy + cz * cz);
    }
  }
  if (P.order != 4 && P.order != 6 && P.order != 8) return fail(err, MSM_ERR_INVALID_ARG, "order must be 4, 6 or 8");
  if (!(P.cutoff > 0.0) || !std::isfinite(P.cutoff)) return fail(err, MSM_ERR_INVALID_ARG, "cutoff must be > 0");
  if (P.qi_mode != 0 && P.qi_mode != 1) return fail(err, MSM_ERR_INVALID_ARG, "qi_mode must be 0 or 1");
  S.p = P.order;
  S.a = P.cutoff;
  S.qi_mode = P.qi_mode;
  if (S.qi_mode == 1) {
    S.hw = exact_omega(S.p, S.omh);
  } else {
    double wh[4];
    omega_half(S.p, wh);
    S.hw = S.p / 2 - 1;
    S.omh.assign(wh, wh + S.hw + 1);
  }
  int Mper = 0;
  for (int d = 0; d < 3; d++) {
    S.L[d] = S.tri ? std::sqrt(P.cell[3 * d] * P.cell[3 * d] + P.cell[3 * d + 1] * P.cell[3 * d + 1] +
                               P.cell[3 * d + 2] * P.cell[3 * d + 2])
                   : P.cell[4 * d];
    if (!(S.L[d] > 0.0)) return fail(err, MSM_ERR_INVALID_ARG, "cell lengths must be > 0");
    if (P.pbc[d] != 0 && P.pbc[d] != 1) return fail(err, MSM_ERR_INVALID_ARG, "pbc entries must be 0 or 1");
    S.pbc[d] = P.pbc[d];
    int M;
    if (P.grid_override[d] > 0) {
      M = P.grid_override[d];
    } else {
      if (!(P.h > 0.0) || !std::isfinite(P.h)) return fail(err, MSM_ERR_INVALID_ARG, "h must be > 0");
      double ratio = S.L[d] / P.h;
      if (S.pbc[d]) {
        int e = (int)std::floor(std::log2(ratio) + 0.5);
        e = std::max(e, 1);
        if (e > 16) return fail(err, MSM_ERR_UNSUPPORTED, "periodic grid above 65536 points per axis");
        M = 1 << e;
      } else {
        M = std::max(1, (int)std::ceil(ratio));
      }
    }
    if (M > 65536) return fail(err, MSM_ERR_UNSUPPORTED, "grid above 65536 intervals per axis");
    if (S.pbc[d]) {
      if (M < 2 || (M & (M - 1))) return fail(err, MSM_ERR_UNSUPPORTED, "periodic grid counts must be powers of two >= 2");
      if (Mper && Mper != M) return fail(err, MSM_ERR_UNSUPPORTED, "periodic axes must have equal grid counts");
      Mper = M;
    }
    S.M[d] = M;
    S.h1[d] = S.L[d] / M;
  }
  const int H = S.p / 2;
  // level ranges: open axes keep the indices restriction can reach
  int olo[kMaxLev][3], on[kMaxLev][3];
  for (int d = 0; d < 3; d++) {
    olo[0][d] = -H;
    on[0][d] = S.M[d] + 2 * H + 1;
    for (int l = 1; l < kMaxLev; l++) {
      int lo = olo[l - 1][d], hi = lo + on[l - 1][d] - 1;
      int a = lo - H, b = hi + H;
      int nlo = (a >= 0) ? (a + 1) / 2 : -((-a) / 2);  // ceil(a/2)
      int nhi = (b >= 0) ? b / 2 : -((-b + 1) / 2);    // floor(b/2)
      olo[l][d] = nlo;
      on[l][d] = nhi - nlo + 1;
    }
  }
  if (Mper) {
    int L = 1;
    while ((1 << (L - 1)) < Mper) L++;
    if (P.levels > 0 && P.levels != L)
      return fail(err, MSM_ERR_UNSUPPORTED, "levels is fixed by the periodic grid (log2(M) + 1)");
    S.nlev = L;
    // periodic cells drop the one-point top level (zero for neutral systems);
    // slabs and wires keep it, with k_L summed over the 2-D or 1-D lattice
    // of their periodic axes (slab_top_kernel, wire_top_kernel)
    S.ncomp = (S.pbc[0] && S.pbc[1] && S.pbc[2]) ? L - 1 : L;
  } else {
    if (P.levels > 0) {
      S.nlev = P.levels;
    } else {
      int cap = std::max(8, S.p + 1), L = 1;
      while (L < kMaxLev && (on[L - 1][0] > cap || on[L - 1][1] > cap || on[L - 1][2] > cap)) L++;
      S.nlev = L;
    }
    if (S.nlev > kMaxLev) return fail(err, MSM_ERR_UNSUPPORTED, "too many levels");
    S.ncomp = S.nlev;
  }
  S.lev.assign(S.ncomp, LevelHost());
  for (int l = 1; l <= S.ncomp; l++) {
    LevelHost& Lv = S.lev[l - 1];
    for (int d = 0; d < 3; d++) {
      Lv.per[d] = S.pbc[d];
      if (S.pbc[d]) {
        Lv.lo[d] = 0;
        Lv.n[d] = S.M[d] >> (l - 1);
      } else {
        Lv.lo[d] = olo[l - 1][d];
        Lv.n[d] = on[l - 1][d];
      }
    }
  }
  // stencil radius, binning cells
  for (int d = 0; d < 3; d++) {
    if (!S.tri) {
      S.S[d] = std::max(0, (int)std::ceil(2.0 * S.a / S.h1[d]) - 1);
    } else {
      // samples |A^T (n / M)| < 2a fill an ellipsoid whose extent along index
      // axis d is 2a M_d |column d of A^-1|
      double c2 = 0.0;
      for (int e = 0; e < 3; e++) c2 += S.Ainv[3 * e + d] * S.Ainv[3 * e + d];
      S.S[d] = std::max(0, (int)std::ceil(2.0 * S.a * S.M[d] * std::sqrt(c2)) - 1);
    }
    S.R[d] = S.S[d] + S.hw;
    S.prefilter = (S.p == 4 && S.qi_mode == 0);
    S.B[d] = S.prefilter ? S.S[d] : S.R[d];
    if (S.pbc[d]) {
      // periodic axis: cells aligned with the grid, k = 2^j level-1 intervals
      // per cell, the largest with k h_1 <= a/2 along x, y and <= a/4 along z
      // (k >= 1), at most 512 cells; h_1 is the spacing of the grid planes
      // (wplane / M for a tilted cell). Half-height cells along z (the axis of
      // the cell columns) cut the short-range candidates by a tenth.
      const double hp = S.tri ? S.wplane[d] / S.M[d] : S.h1[d];
      int k = 1;
      while (2 * k <= S.M[d] && 2 * k * hp <= (d == 2 ? 0.25 : 0.5) * S.a) k *= 2;
      while (S.M[d] / k > 512) k *= 2;
      S.C[d] = S.M[d] / k;
    } else {
      // open axis: edge >= a/2 along x, y and >= a/4 along z
      int C = (int)std::floor((d == 2 ? 4.0 : 2.0) * S.L[d] / S.a);
      S.C[d] = std::min(std::max(C, 1), 256);
    }
    S.edge[d] = S.wplane[d] / S.C[d];  // distance between cell faces
    S.nnbr[d] = (int)std::ceil(S.a / S.edge[d]);
  }
  fill_stencils(S, true);
  if (S.has_ball && S.wmax > kBallRmax) {
    // a tilted cell whose shifted columns are wider than the compiled ball kernels
    S.allow_ball = false;
    fill_stencils(S, true);
  }
  // scalar coefficients
  softening_coeffs(S.p, S.gc);
  {
    double binom = 1.0;
    for (int k = 0; k <= S.p; k++) {
      S.jc[k] = std::ldexp(binom, 1 - S.p);
      binom = binom * (S.p - k) / (k + 1);
    }
  }
  return MSM_OK;
}

// ------------------------------------------------------------------ engine
static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Spectra of the level-l stencil for the spectral level method (k_fft.cu) on a
// periodic grid of n points per axis: the octant k_d in [0, n_d / 2] of the
// discrete Fourier transform of K^l = K^1 / 2^(l-1) (the unfolded stencil's
// transform sampled at k / n equals the transform of the stencil folded onto
// the grid) and of the six strain-derivative stencils dK^1 / 2^(l-1) (xx yy zz
// xy xz yz). K and dK_aa are even in every axis (cosine sums); dK_ab is odd in
// a and b and even in the third axis, so its transform is minus the sum with
// sines along a and b. Separable sums in FP64 (z, then y, then x), stored as
// float times 1/N (K^) and -1/2 (1/N) (dK^), N = n_x n_y n_z, in seven
// consecutive octant arrays [k_x][k_y][k_z].
void level_spectra(const SysHost& S, int l, const int n[3], float* out) {
  const int R[3] = {S.R[0], S.R[1], S.R[2]};
  const int sz[3] = {2 * R[0] + 1, 2 * R[1] + 1, 2 * R[2] + 1};
  const int h[3] = {n[0] / 2 + 1, n[1] / 2 + 1, n[2] / 2 + 1};
  const size_t box = (size_t)sz[0] * sz[1] * sz[2];
  const size_t oct = (size_t)h[0] * h[1] * h[2];
  // trig[d][par][k * sz + (m + R)]: cos (par 0) or sin (par 1) of 2 pi k m / n_d, the
  // angle reduced exactly (k m mod n_d) before the FP64 evaluation
  std::vector<double> trig[3][2];
  for (int d = 0; d < 3; d++) {
    trig[d][0].assign((size_t)h[d] * sz[d], 0.0);
    trig[d][1].assign((size_t)h[d] * sz[d], 0.0);
    for (int k = 0; k < h[d]; k++)
      for (int m = -R[d]; m <= R[d]; m++) {
        long long km = ((long long)k * m) % n[d];
        if (km < 0) km += n[d];
        const double ang = 2.0 * M_PI * (double)km / (double)n[d];
        trig[d][0][(size_t)k * sz[d] + m + R[d]] = std::cos(ang);
        trig[d][1][(size_t)k * sz[d] + m + R[d]] = std::sin(ang);
      }
  }
  const double N = (double)n[0] * n[1] * n[2];
  const double scale = std::ldexp(1.0, -(l - 1)) / N;
  static const int par[7][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
  std::vector<double> Az((size_t)sz[0] * sz[1] * h[2]), Ay((size_t)sz[0] * h[1] * h[2]), Ax(oct);
  for (int arr = 0; arr < 7; arr++) {
    const double* A = arr == 0 ? S.kball.data() : S.dk1.data() + (size_t)(arr - 1) * box;
    const std::vector<double>& tx = trig[0][par[arr][0]];
    const std::vector<double>& ty = trig[1][par[arr][1]];
    const std::vector<double>& tz = trig[2][par[arr][2]];
    for (int x = 0; x < sz[0]; x++)
      for (int y = 0; y < sz[1]; y++) {
        const double* row = A + ((size_t)x * sz[1] + y) * sz[2];
        double* o = Az.data() + ((size_t)x * sz[1] + y) * h[2];
        for (int kz = 0; kz < h[2]; kz++) {
          const double* t = tz.data() + (size_t)kz * sz[2];
          double acc = 0.0;
          for (int z = 0; z < sz[2]; z++) acc += row[z] * t[z];
          o[kz] = acc;
        }
      }
    std::fill(Ay.begin(), Ay.end(), 0.0);
    for (int x = 0; x < sz[0]; x++)
      for (int ky = 0; ky < h[1]; ky++) {
        double* o = Ay.data() + ((size_t)x * h[1] + ky) * h[2];
        for (int y = 0; y < sz[1]; y++) {
          const double c = ty[(size_t)ky * sz[1] + y];
          const double* src = Az.data() + ((size_t)x * sz[1] + y) * h[2];
          for (int kz = 0; kz < h[2]; kz++) o[kz] += c * src[kz];
        }
      }
    std::fill(Ax.begin(), Ax.end(), 0.0);
    const size_t plane = (size_t)h[1] * h[2];
    for (int kx = 0; kx < h[0]; kx++) {
      double* o = Ax.data() + (size_t)kx * plane;
      for (int x = 0; x < sz[0]; x++) {
        const double c = tx[(size_t)kx * sz[0] + x];
        const double* src = Ay.data() + (size_t)x * plane;
        for (size_t e = 0; e < plane; e++) o[e] += c * src[e];
      }
    }
    const double f = (arr == 0 ? 1.0 : -0.5) * (arr >= 4 ? -1.0 : 1.0) * scale;
    for (size_t e = 0; e < oct; e++) out[(size_t)arr * oct + e] = (float)(f * Ax[e]);
  }
}



// Device pools of the stencil values: per system the ball stencil (a row of
// kSK(hz) floats per (dx, dy) column), its virial weights and column tables,
// then each box level's folded K and dK; records the offsets in the level
// descriptors and the systems. The layout depends only on the plan's sizes.
void Engine::assemble_pools(const std::vector<int>& lev0_of, std::vector<float>& kp, std::vector<int>& wp) {
  kp.clear();
  wp.clear();
  for (int s = 0; s < nsys; s++) {
    SysHost& S = sys[s];
    long long kball_off = -1, dkh_off = -1, wb_off = -1, wh_off = -1;
    if (S.has_ball) {
      // column layout read by the ball kernels: for each (dx, dy) a row of
      // kSK(hz) floats with dz = -hz .. hz at [0, 2hz]; virial weights [dx][6][dy][row]
      const int nx = 2 * S.B[0] + 1, ny = 2 * S.B[1] + 1, nz = 2 * S.B[2] + 1;
      const int hz = S.hzb, SK = kSK(hz);
      // row index of sample z of column (x, y): z about the column's centre (entries
      // outside the row are zero by construction of hzb)
      auto rowpos = [&](int x, int y, int z) { return z - S.B[2] - S.cball[(size_t)x * ny + y] + hz; };
      auto inrow = [&](int r) { return r >= 0 && r <= 2 * hz; };
      const bool fact = S.prefilter && !any_tri;
      while (kp.size() % 4) kp.push_back(0.f);
      kball_off = (long long)kp.size();
      kp.resize(kp.size() + (size_t)nx * ny * SK, 0.f);
      for (int x = 0; x < nx; x++)
        for (int y = 0; y < ny; y++)
          for (int z = 0; z < nz; z++) {
            const int r = rowpos(x, y, z);
            if (inrow(r)) kp[kball_off + ((size_t)x * ny + y) * SK + r] = S.sball[((size_t)x * ny + y) * nz + z];
          }
      dkh_off = (long long)kp.size();
      if (fact) {
        // factorized virial weights g(n), one array [dx][dy][row]
        kp.resize(kp.size() + (size_t)nx * ny * SK, 0.f);
        for (int x = 0; x < nx; x++)
          for (int y = 0; y < ny; y++)
            for (int z = 0; z < nz; z++)
              kp[dkh_off + ((size_t)x * ny + y) * SK + rowpos(x, y, z)] = S.fsh[((size_t)x * ny + y) * nz + z];
      } else {
        kp.resize(kp.size() + (size_t)nx * 6 * ny * SK, 0.f);
        for (int x = 0; x < nx; x++)
          for (int c = 0; c < 6; c++)
            for (int y = 0; y < ny; y++)
              for (int z = 0; z < nz; z++) {
                const int r = rowpos(x, y, z);
                if (inrow(r))
                  kp[dkh_off + (((size_t)x * 6 + c) * ny + y) * SK + r] =
                      S.dsh[(size_t)c * nx * ny * nz + ((size_t)x * ny + y) * nz + z];
              }
      }
      wb_off = (long long)wp.size();
      wp.insert(wp.end(), S.wball.begin(), S.wball.end());
      wh_off = (long long)wp.size();
      wp.insert(wp.end(), S.whalf.begin(), S.whalf.end());
      S.cb_off = (long long)wp.size();
      wp.insert(wp.end(), S.cball.begin(), S.cball.end());
    }
    S.kball_off = kball_off;
    S.dkh_off = dkh_off;
    S.wb_off = wb_off;
    S.wh_off = wh_off;
    for (int l = 1; l <= S.ncomp; l++) {
      LevDev& L = hlev[lev0_of[s] + l - 1];
      const LevelHost& Lv = S.lev[l - 1];
      if (L.kind == 0) {
        L.k_off = kball_off;
        L.dk_off = dkh_off;
        L.w_off = wb_off;
        L.wh_off = wh_off;
        L.c_off = S.cb_off;
      } else {
        while (kp.size() % 4) kp.push_back(0.f);
        L.k_off = (long long)kp.size();
        kp.insert(kp.end(), Lv.kbox.begin(), Lv.kbox.end());
        // virial weights interleaved per entry, 6 values padded to 8 (two 16-byte loads;
        // the array starts on a 16-byte boundary)
        while (kp.size() % 4) kp.push_back(0.f);
        L.dk_off = (long long)kp.size();
        const size_t nt = Lv.kbox.size();
        kp.resize(kp.size() + 8 * nt, 0.f);
        for (size_t t = 0; t < nt; t++)
          for (int c = 0; c < 6; c++) kp[L.dk_off + 8 * t + c] = Lv.dkbox[c * nt + t];
      }
    }
    while (kp.size() % 4) kp.push_back(0.f);
  }
  if (spec_ok) {
    // spectral level method: twiddles exp(-2 pi i j / 256), then each level's spectrum octants
    const SysHost& S = sys[0];
    const long long tw = (long long)kp.size();
    for (int j = 0; j < kSpecNmax; j++) {
      const double a = -2.0 * M_PI * j / kSpecNmax;
      kp.push_back((float)std::cos(a));
      kp.push_back((float)std::sin(a));
    }
    for (int l = 1; l <= S.ncomp; l++) {
      LevDev& L = hlev[lev0_of[0] + l - 1];
      while (kp.size() % 4) kp.push_back(0.f);
      L.tw_off = tw;
      L.sp_off = (long long)kp.size();
      const int hx = L.n[0] / 2 + 1, hy = L.n[1] / 2 + 1, hz = L.n[2] / 2 + 1, nz = L.n[2];
      const size_t oct = (size_t)hx * hy * hz;
      std::vector<float> seven(7 * oct);
      level_spectra(S, l, L.n, seven.data());
      // stored as k_spec_x reads them: [|k_x|][|k_y|][z position], the z position holding the
      // frequency whose bit reversal it is (the work buffer's order), eight floats per point
      // (two 16-byte loads); a tile's consecutive z positions are then consecutive in memory
      kp.resize(kp.size() + (size_t)8 * hx * hy * nz, 0.f);
      int lgz = 0;
      while ((1 << lgz) < nz) lgz++;
      for (int fx = 0; fx < hx; fx++)
        for (int fy = 0; fy < hy; fy++)
          for (int zp = 0; zp < nz; zp++) {
            int kz = 0;
            for (int b = 0; b < lgz; b++) kz |= ((zp >> b) & 1) << (lgz - 1 - b);
            const int fz = std::min(kz, nz - kz);
            const size_t o = ((size_t)fx * hy + fy) * hz + fz;
            const size_t at = (((size_t)fx * hy + fy) * nz + zp) * 8;
            for (int c = 0; c < 7; c++) kp[L.sp_off + at + c] = seven[c * oct + o];
          }
    }
  }
  if (kp.empty()) kp.push_back(0.f);
  if (wp.empty()) wp.push_back(0);
}

int Engine::build(const msm_params* prm, const int* counts, int nsys_, bool single_, std::string* err) {
  nsys = nsys_;
  single = single_;
  sys.assign(nsys, SysHost());
  for (int s = 0; s < nsys; s++) {
    sys[s].fold_small = !single_;
    int rc = plan_system(prm[s], sys[s], err);
    if (rc) return rc;
    if (counts[s] < 0) return fail(err, MSM_ERR_INVALID_ARG, "atom counts must be >= 0");
    if (sys[s].p != sys[0].p) return fail(err, MSM_ERR_UNSUPPORTED, "all systems of a batch need the same order");
  }
  p = sys[0].p;
  any_tri = false;
  for (const SysHost& S : sys) any_tri = any_tri || S.tri;
  // systems, atoms, cells, levels, grid pool
  std::vector<SysDev> hs(nsys);
  hlev.clear();
  atom_items.clear();
  long long grid_off = 0;
  int atom_off = 0, cell_off = 0;
  maxcomp = 0;
  for (int s = 0; s < nsys; s++) {
    SysHost& S = sys[s];
    SysDev& D = hs[s];
    std::memset(&D, 0, sizeof(D));
    D.n = counts[s];
    D.atom_off = atom_off;
    D.cell_off = cell_off;
    D.p = S.p;
    D.ncomp = S.ncomp;
    D.lev0 = (int)hlev.size();
    D.item0 = (int)atom_items.size();
    for (int d = 0; d < 3; d++) {
      D.C[d] = S.C[d];
      D.nnbr[d] = S.nnbr[d];
      D.cshift[d] = 0;
      while ((1 << D.cshift[d]) < S.C[d]) D.cshift[d]++;
      D.pbc[d] = S.pbc[d];
      D.M[d] = S.M[d];
      D.edge[d] = (float)S.edge[d];
      D.edged[d] = S.edge[d];
      D.Ld[d] = S.L[d];
      D.invL[d] = (float)(1.0 / S.L[d]);
      D.Mf[d] = (float)S.M[d];
      D.inv_h1[d] = (float)(1.0 / S.h1[d]);
      D.Lf[d] = (float)S.L[d];
      D.h1f[d] = (float)S.h1[d];
    }
    D.tri = S.tri ? 1 : 0;
    for (int k = 0; k < 9; k++) {
      D.Tf[k] = (float)S.Tinv[k];
      D.Ad[k] = S.A[k];
      D.Td[k] = S.Tinv[k];
    }
    for (int e = 0; e < 3; e++)
      for (int d = 0; d < 3; d++) D.Jg[3 * e + d] = (float)(S.Ainv[3 * e + d] * S.M[d]);
    for (int d = 0; d < 3; d++) D.reach[d] = (float)(S.a / S.wplane[d]);
    D.a2 = (float)(S.a * S.a);
    D.inv_a = (float)(1.0 / S.a);
    D.inv_a2 = (float)(1.0 / (S.a * S.a));
    D.inv_a3 = (float)(1.0 / (S.a * S.a * S.a));
    D.self_coef = (float)(soft(S.p, 0.0) / S.a);
    for (int k = 0; k < S.p; k++) D.gca[k] = (float)(S.gc[k] / S.a);
    for (int k = 0; k + 1 < S.p; k++) D.gdca[k] = (float)(2.0 * (k + 1) * S.gc[k + 1] / (S.a * S.a * S.a));
    for (int k = 0; k <= S.p; k++) D.jc[k] = (float)S.jc[k];
    {
      double bp[4][8];
      bspline_pieces(S.p, bp);
      for (int i = 0; i < 4; i++)
        for (int k = 0; k < 8; k++) D.bsp[i][k] = (float)bp[i][k];
    }
    {
      double om[4];
      omega_half(S.p, om);
      // the ball kernels prefilter the grid with omega' (and apply the raw
      // samples) for p = 4 only; for p = 6, 8 the large omega' (omega'_0 = 3.0,
      // 6.0) would cost FP32 digits, so they apply K itself (identity prefilter)
      D.pre_r = S.prefilter ? S.p / 2 - 1 : 0;
      for (int k = 0; k < 4; k++) D.om[k] = S.prefilter ? (k < S.p / 2 ? (float)om[k] : 0.f) : (k == 0 ? 1.f : 0.f);
    }
    // footprints of the binning columns on the level-1 grid (anterpolation by columns)
    for (int d = 0; d < 3; d++) {
      const int k = S.M[d] / S.C[d];
      const bool aligned = S.pbc[d] && S.M[d] % S.C[d] == 0 && (k & (k - 1)) == 0;
      D.ashift[d] = -1;
      if (aligned)
        for (D.ashift[d] = 0; (1 << D.ashift[d]) < k; D.ashift[d]++) {
        }
      D.aratio[d] = (float)((double)S.M[d] / (double)S.C[d]);
      D.ainv[d] = (float)((double)S.C[d] / (double)S.M[d]);
      if (d < 2)
        D.afoot[d] = aligned ? k + S.p - 1 : (int)std::floor((1.0 + 4e-4) * (double)S.M[d] / (double)S.C[d]) + S.p + 1;
    }
    for (int st = 0; st < counts[s]; st += kChunk) atom_items.push_back({s, st, std::min(kChunk, counts[s] - st)});
    if (counts[s] == 0) atom_items.push_back({s, 0, 0});
    D.nitem = (int)atom_items.size() - D.item0;
    atom_off += counts[s];
    cell_off += S.C[0] * S.C[1] * S.C[2];
    maxcomp = std::max(maxcomp, S.ncomp);
    for (int l = 1; l <= S.ncomp; l++) {
      LevDev L;
      std::memset(&L, 0, sizeof(L));
      const LevelHost& Lv = S.lev[l - 1];
      L.sys = s;
      L.level = l;
      for (int d = 0; d < 3; d++) {
        L.n[d] = Lv.n[d];
        L.lo[d] = Lv.lo[d];
        L.per[d] = Lv.per[d];
        L.R[d] = Lv.R[d];
        L.blo[d] = Lv.blo[d];
        L.bsz[d] = Lv.bsz[d];
      }
      L.kind = Lv.kind;
      L.scale = Lv.scale;
      long long npts = (long long)Lv.n[0] * Lv.n[1] * Lv.n[2];
      L.q_off = grid_off;
      grid_off += align_up(npts, 64);
      L.e_off = grid_off;
      grid_off += align_up(npts, 64);
      L.p_off = -1;
      if (L.kind == 0) {
        // halo-padded copy of q~^l read by the ball kernels: halos R_x, R_y and
        // hz = R_z rounded up to 4 floats; y and z extents rounded up to whole tiles
        L.hz = S.hzb;
        L.pn[0] = L.n[0] + 2 * L.R[0];
        L.pn[1] = (int)align_up(L.n[1], kBallTY) + 2 * L.R[1];
        L.pn[2] = (int)align_up(L.n[2], kBallTZ) + 2 * L.hz;
        L.p_off = grid_off;
        grid_off += align_up((long long)L.pn[0] * L.pn[1] * L.pn[2], 64);
      }
      hlev.push_back(L);
    }
  }
  total_atoms = atom_off;
  total_cells = cell_off;
  grid_floats = grid_off;
  // spectral level method: eligibility, log2 sizes and complex work buffers of the levels
  spec_ok = false;
  spec_complex = 0;
  for (LevDev& L : hlev) {
    L.f_off = L.sp_off = L.tw_off = -1;
    for (int d = 0; d < 3; d++) L.lg[d] = 0;
  }
  if (single && nsys == 1) {
    const SysHost& S = sys[0];
    bool ok = S.pbc[0] && S.pbc[1] && S.pbc[2] && !S.tri && S.ncomp >= 1 && !S.kball.empty();
    for (int l = 1; ok && l <= S.ncomp; l++) {
      const LevDev& L = hlev[hs[0].lev0 + l - 1];
      ok = L.kind == 0;
      for (int d = 0; d < 3 && ok; d++) ok = L.n[d] >= 2 && L.n[d] <= kSpecNmax && (L.n[d] & (L.n[d] - 1)) == 0;
    }
    spec_ok = ok;
    if (ok)
      for (int l = 1; l <= S.ncomp; l++) {
        LevDev& L = hlev[hs[0].lev0 + l - 1];
        L.f_off = spec_complex;
        spec_complex += (long long)L.n[0] * L.n[1] * L.n[2];
        for (int d = 0; d < 3; d++)
          while ((1 << L.lg[d]) < L.n[d]) L.lg[d]++;
      }
  }
  if (!spec_ok) level_method = 0;
  // stencil pools
  std::vector<float> kp;
  std::vector<int> wp;
  {
    std::vector<int> lev0_of(nsys);
    for (int s = 0; s < nsys; s++) lev0_of[s] = hs[s].lev0;
    assemble_pools(lev0_of, kp, wp);
  }
  // work lists
  anterp_items.clear();
  ball_items.clear();
  pad_items.clear();
  box_items.clear();
  vb_off.assign(nsys + 1, 0);
  vx_off.assign(nsys + 1, 0);
  rmax = 0;
  ryz[0] = ryz[1] = 0;
  for (int s = 0; s < nsys; s++) {
    const SysHost& S = sys[s];
    vb_off[s] = (int)ball_items.size();
    vx_off[s] = (int)box_items.size();
    for (int l = 1; l <= S.ncomp; l++) {
      int li = hs[s].lev0 + l - 1;
      const LevDev& L = hlev[li];
      if (L.kind == 0) {
        for (int x = 0; x < L.n[0]; x++)
          for (int y = 0; y < L.n[1]; y += kBallTY)
            for (int z = 0; z < L.n[2]; z += kBallTZ) ball_items.push_back({li, x, y, z});
        rmax = std::max(rmax, std::max(L.R[2] + (L.R[2] & 1), S.wmax));  // column half-widths are even
        ryz[0] = std::max(ryz[0], L.R[1]);
        ryz[1] = std::max(ryz[1], L.hz);
        for (int x = 0; x < L.pn[0]; x += kPadTX)
          for (int y = 0; y < L.pn[1]; y += kPadTY)
            for (int z = 0; z < L.pn[2]; z += kPadTZ) pad_items.push_back({li, x, y, z});
      } else {
        long long npts = (long long)L.n[0] * L.n[1] * L.n[2];
        // staged boxes in batch plans (many levels at once); a single system's few outputs per
        // level finish sooner with a warp per output (the lanes split the box entries)
        hlev[li].box_tile = (!single && npts <= kBoxStage) ? 1 : 0;
        const int chunk = hlev[li].box_tile ? kBoxThreads : kBoxChunk;
        for (long long st = 0; st < npts; st += chunk)
          box_items.push_back({li, (int)st, (int)std::min<long long>(chunk, npts - st)});
      }
    }
  }
  vb_off[nsys] = (int)ball_items.size();
  vx_off[nsys] = (int)box_items.size();
  spec_z_items.clear();
  spec_y_items.clear();
  spec_x_items.clear();
  if (spec_ok)
    for (int l = 1; l <= sys[0].ncomp; l++) {
      const int li = hs[0].lev0 + l - 1;
      const LevDev& L = hlev[li];
      const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
      const int tz = std::min(n1, kSpecTile / n2), ty = std::min(n2, kSpecTile / n1), tx = std::min(n2, kSpecTile / n0);
      for (int x = 0; x < n0; x++)
        for (int y = 0; y < n1; y += tz) spec_z_items.push_back({li, x, y, std::min(tz, n1 - y)});
      for (int x = 0; x < n0; x++)
        for (int z = 0; z < n2; z += ty) spec_y_items.push_back({li, x, z, std::min(ty, n2 - z)});
      for (int y = 0; y < n1; y++)
        for (int z = 0; z < n2; z += tx) spec_x_items.push_back({li, y, z, std::min(tx, n2 - z)});
    }
  restrict_steps.assign(std::max(0, maxcomp - 1), std::vector<TileItem>());
  prolong_steps.assign(std::max(0, maxcomp - 1), std::vector<TileItem>());
  for (int l = 1; l < maxcomp; l++) {
    for (int s = 0; s < nsys; s++) {
      if (sys[s].ncomp <= l) continue;
      int fi = hs[s].lev0 + l - 1, ci = fi + 1;
      const LevDev& F = hlev[fi];
      const LevDev& Cc = hlev[ci];
      for (int x = 0; x < Cc.n[0]; x += kResTX)
        for (int y = 0; y < Cc.n[1]; y += kResTY)
          for (int z = 0; z < Cc.n[2]; z += kResTZ) restrict_steps[l - 1].push_back({ci, x, y, z});
      for (int x = 0; x < F.n[0]; x += kProTX)
        for (int y = 0; y < F.n[1]; y += kProTY)
          for (int z = 0; z < F.n[2]; z += kProTZ) prolong_steps[l - 1].push_back({fi, x, y, z});
    }
  }
  // device tables
  std::vector<int> voff(2 * (nsys + 1));
  for (int s = 0; s <= nsys; s++) {
    voff[s] = vb_off[s];
    voff[nsys + 1 + s] = (int)ball_items.size() + vx_off[s];
  }
  // the spectral method's virial partials: one per x item of system 0, then the box items
  voff_spec.assign(2 * (nsys + 1), 0);
  for (int s = 0; s <= nsys; s++) {
    voff_spec[s] = s == 0 ? 0 : (int)spec_x_items.size();
    voff_spec[nsys + 1 + s] = (int)spec_x_items.size() + vx_off[s];
  }
  // column partials of the anterpolation: C_x C_y afoot_x afoot_y n_z floats per system
  apart_floats = 0;
  for (int s = 0; s < nsys; s++) {
    hs[s].apart = apart_floats;
    if (sys[s].ncomp < 1) continue;
    apart_floats += (long long)hs[s].C[0] * hs[s].C[1] * hs[s].afoot[0] * hs[s].afoot[1] * hlev[hs[s].lev0].n[2];
  }
  hsys = hs;
  build_anterp_items(anterp_tz);
  {
    // virial partials of the largest system: per-warp short-range items plus ball and box items
    long long most = 0;
    for (int s = 0; s < nsys; s++) {
      long long tot = (long long)hs[s].nitem * kChunkWarps +
                      std::max<long long>(vb_off[s + 1] - vb_off[s], s == 0 ? (long long)spec_x_items.size() : 0) +
                      (vx_off[s + 1] - vx_off[s]);
      most = std::max(most, tot);
    }
    vslices = (int)std::min<long long>(kVirialSlices, std::max<long long>(1, (most + 1023) / 1024));
  }
  int rc = upload(kp, wp, voff, err);
  if (rc) return rc;
  spec_n.clear();
  spec_sp.clear();
  if (spec_ok && sys[0].prefilter) {
    // scratch of the device-path spectra (msm_plan_set_cell): every level's separable sums
    const SysHost& S = sys[0];
    for (int l = 1; l <= S.ncomp; l++) {
      spec_n.push_back(hlev[hs[0].lev0 + l - 1].n[0]);
      spec_sp.push_back(hlev[hs[0].lev0 + l - 1].sp_off);
    }
    const long long nxb = 2 * S.B[0] + 1, nyb = 2 * S.B[1] + 1;
    long long na = 0, nb = 0;
    for (int nl : spec_n) {
      const long long h = nl / 2 + 1;
      na += 7 * nxb * nyb * h;
      nb += 7 * nxb * h * h;
    }
    nb += 7 * nxb * nyb * (2 * S.B[2] + 1);  // the raw samples, after the y sums
    cudaFree(d_spec_scr_a);
    cudaFree(d_spec_scr_b);
    d_spec_scr_a = d_spec_scr_b = nullptr;
    if (cudaMalloc((void**)&d_spec_scr_a, sizeof(float) * na) != cudaSuccess ||
        cudaMalloc((void**)&d_spec_scr_b, sizeof(float) * nb) != cudaSuccess)
      return fail(err, MSM_ERR_CUDA, "cudaMalloc of the spectra scratch failed");
  }
  // workspace layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1), 256);
    return o;
  };
  const size_t N = (size_t)std::max(total_atoms, 1);
  const int ntiles = (total_cells + 4095) / 4096;
  L_status = take(256);
  L_cell_count = take(sizeof(int) * total_cells);
  L_cell_start = take(sizeof(int) * (total_cells + 1));
  L_scan_tiles = take(sizeof(int) * std::max(ntiles, 1));
  L_cell_id = take(sizeof(int) * N);
  L_slot = take(sizeof(int) * N);
  L_bucket = take(sizeof(int2) * N);
  L_perm = take(sizeof(int) * N);
  L_iperm = take(sizeof(int) * N);
  L_scell = take(sizeof(int) * N);
  L_xq = take(sizeof(float4) * N);
  L_uq = take(sizeof(float4) * N);
  L_phi_sr = take(sizeof(float) * N);
  L_phi_lr = take(sizeof(float) * N);
  L_f_sr = take(sizeof(float4) * N);
  L_f_lr = take(sizeof(float4) * N);
  L_res = take(sizeof(float4) * N);
  L_part_e = take(sizeof(double) * atom_items.size());
  L_part_q = take(sizeof(double) * 2 * atom_items.size());
  L_part_w0 = take(sizeof(double) * 6 * kChunkWarps * atom_items.size());
  L_part_wg = take(sizeof(double) * 6 * std::max<size_t>(std::max(ball_items.size(), spec_x_items.size()) + box_items.size(), 1));
  L_part_vs = take(sizeof(double) * 6 * 64 * (size_t)nsys);
  L_grid = take(sizeof(float) * std::max<long long>(grid_floats, 1));
  L_vjp_u = take(sizeof(float4) * N);
  L_vjp_h = take(sizeof(float4) * N);
  L_io_pos = take(sizeof(float) * 3 * N);
  L_io_q = take(sizeof(float) * N);
  L_io_dpos = take(sizeof(float) * 3 * N);
  L_io_dq = take(sizeof(float) * N);
  L_io_e = take(sizeof(double) * 11 * (size_t)std::max(nsys, 1));
  // sized whenever the footprints fit the column kernel, whatever z-extent the tuning picks later
  L_apart = take(sizeof(float) * (size_t)(ant_fmax[0] <= kAntFootMax && ant_fmax[1] <= kAntFootMax ? apart_floats : 0));
  L_spec = take(sizeof(float2) * (size_t)spec_complex);
  ws_bytes = off;
  return MSM_OK;
}

template <class T>
static int up(const std::vector<T>& h, T** d, std::string* err) {
  cudaFree(*d);
  *d = nullptr;
  size_t b = sizeof(T) * std::max<size_t>(h.size(), 1);
  if (cudaMalloc((void**)d, b) != cudaSuccess) return fail(err, MSM_ERR_CUDA, "cudaMalloc of plan tables failed");
  if (!h.empty() && cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(err, MSM_ERR_CUDA, "cudaMemcpy of plan tables failed");
  return MSM_OK;
}

// anterpolation work lists for z-extent tz (16, 32, 64): tiles of kAnterpTX x
// kAnterpTY x tz level-1 points (dipole anterpolation, and every anterpolation
// when a footprint is too wide for the column kernel), and the column items
// (binning column, z-segment of tz points) with the sum items of k_anterp_sum
void Engine::build_anterp_items(int tz) {
  anterp_items.clear();
  acol_items.clear();
  asum_items.clear();
  int fmax[2] = {0, 0};
  for (int s = 0; s < nsys; s++) {
    if (sys[s].ncomp < 1) continue;
    const int li = hsys[s].lev0;
    const LevDev& L = hlev[li];
    for (int x = 0; x < L.n[0]; x += kAnterpTX)
      for (int y = 0; y < L.n[1]; y += kAnterpTY)
        for (int z = 0; z < L.n[2]; z += tz) anterp_items.push_back({li, x, y, z});
    const SysDev& D = hsys[s];
    for (int cx = 0; cx < D.C[0]; cx++)
      for (int cy = 0; cy < D.C[1]; cy++)
        for (int z = 0; z < L.n[2]; z += tz) acol_items.push_back({li, cx, cy, z});
    for (int x = 0; x < L.n[0]; x++)
      for (int y = 0; y < L.n[1]; y += kAntSumY)
        for (int z = 0; z < L.n[2]; z += kAntSumZ) asum_items.push_back({li, x, y, z});
    fmax[0] = std::max(fmax[0], D.afoot[0]);
    fmax[1] = std::max(fmax[1], D.afoot[1]);
  }
  ant_fmax[0] = fmax[0];
  ant_fmax[1] = fmax[1];
  ant_wstride = 0;
  if (!acol_items.empty() && fmax[0] <= kAntFootMax && fmax[1] <= kAntFootMax) {
    const int ws = anterp_cols_wstride(fmax[0], fmax[1], tz, p);
    if (sizeof(float) * kAntWarps * (size_t)ws <= 100 * 1024) ant_wstride = ws;
  }
  anterp_tz = tz;
}

int Engine::set_anterp_tz(int tz, std::string* err) {
  if (tz != 16 && tz != 32 && tz != 64) return fail(err, MSM_ERR_INVALID_ARG, "anterpolation tile must be 16, 32 or 64");
  if (tz == anterp_tz) return MSM_OK;
  build_anterp_items(tz);
  int rc = up(anterp_items, &d_anterp_items, err);
  if (!rc) rc = up(acol_items, &d_acol_items, err);
  if (!rc) rc = up(asum_items, &d_asum_items, err);
  return rc;
}

void Engine::anterp(const Work& w, const Tables& t, cudaStream_t s) const {
  if (ant_wstride > 0)
    launch_anterp_cols(w, t, d_acol_items, (int)acol_items.size(), d_asum_items, (int)asum_items.size(), anterp_tz,
                       ant_wstride, s, p);
  else
    launch_anterp(w, t, d_anterp_items, (int)anterp_items.size(), s, p, anterp_tz);
}

void Engine::stencils(const Work& w, const Tables& t, cudaStream_t s, bool virial) {
  if (level_method == 1) {
    launch_spectral(w, t, d_spec_z, (int)spec_z_items.size(), d_spec_y, (int)spec_y_items.size(), d_spec_x,
                    (int)spec_x_items.size(), virial ? w.part_wg : nullptr, s);
    if (virial) spec_virial_ready = true;
  } else {
    launch_pad(w, t, d_pad_items, (int)pad_items.size(), p == 4 ? 1 : 0, s);
    launch_stencil_ball(w, t, d_ball_items, (int)ball_items.size(), rmax, ryz, any_tri, s);
  }
  launch_stencil_box(w, t, d_box_items, (int)box_items.size(), s);
}

void Engine::grid_virial(const Work& w, const Tables& t, const double* grad, double* virial, cudaStream_t s) {
  if (level_method == 1) {
    if (!spec_virial_ready)
      launch_spectral_virial(w, t, d_spec_z, (int)spec_z_items.size(), d_spec_y, (int)spec_y_items.size(), d_spec_x,
                             (int)spec_x_items.size(), w.part_wg, s);
    spec_virial_ready = true;
    launch_virial_box(w, t, d_box_items, (int)box_items.size(), (int)spec_x_items.size(), s);
    launch_virial_out(w, t, nsys, vslices, d_voff_spec, grad, virial, s);
    return;
  }
  const int nb = (int)ball_items.size();
  launch_virial_ball(w, t, d_ball_items, nb, rmax, ryz, 0, p == 4 && !any_tri, any_tri, s);
  launch_virial_box(w, t, d_box_items, (int)box_items.size(), nb, s);
  launch_virial_out(w, t, nsys, vslices, d_voff, grad, virial, s);
}

int Engine::set_level_method(int method, std::string* err) {
  if (method != 0 && method != 1) return fail(err, MSM_ERR_INVALID_ARG, "level method must be 0 (ball) or 1 (spectral)");
  if (method == 1 && !spec_ok)
    return fail(err, MSM_ERR_UNSUPPORTED,
                "the spectral level method needs a single-system plan with a fully periodic rectangular cell and ball "
                "levels of 2 .. 256 points per axis");
  level_method = method;
  spec_virial_ready = false;
  have_fwd = false;
  return MSM_OK;
}

int Engine::upload(const std::vector<float>& kp, const std::vector<int>& wp, const std::vector<int>& voff,
                   std::string* err) {
  int rc;
  if ((rc = up(hsys, &d_sys, err))) return rc;
  if ((rc = up(hlev, &d_lev, err))) return rc;
  if ((rc = up(kp, &d_kpool, err))) return rc;
  if ((rc = up(wp, &d_wpool, err))) return rc;
  kpool_n = kp.size();
  wpool_n = wp.size();
  if ((rc = up(atom_items, &d_atom_items, err))) return rc;
  if ((rc = up(anterp_items, &d_anterp_items, err))) return rc;
  if ((rc = up(acol_items, &d_acol_items, err))) return rc;
  if ((rc = up(asum_items, &d_asum_items, err))) return rc;
  if ((rc = up(ball_items, &d_ball_items, err))) return rc;
  if ((rc = up(box_items, &d_box_items, err))) return rc;
  if ((rc = up(pad_items, &d_pad_items, err))) return rc;
  if ((rc = up(voff, &d_voff, err))) return rc;
  if ((rc = up(voff_spec, &d_voff_spec, err))) return rc;
  if ((rc = up(spec_z_items, &d_spec_z, err))) return rc;
  if ((rc = up(spec_y_items, &d_spec_y, err))) return rc;
  if ((rc = up(spec_x_items, &d_spec_x, err))) return rc;
  std::vector<TileItem> all;
  restrict_off.assign(restrict_steps.size() + 1, 0);
  for (size_t i = 0; i < restrict_steps.size(); i++) {
    restrict_off[i] = (int)all.size();
    all.insert(all.end(), restrict_steps[i].begin(), restrict_steps[i].end());
  }
  restrict_off[restrict_steps.size()] = (int)all.size();
  if ((rc = up(all, &d_res_items, err))) return rc;
  std::vector<TileItem> pro;
  prolong_off.assign(prolong_steps.size() + 1, 0);
  for (size_t i = 0; i < prolong_steps.size(); i++) {
    prolong_off[i] = (int)pro.size();
    pro.insert(pro.end(), prolong_steps[i].begin(), prolong_steps[i].end());
  }
  prolong_off[prolong_steps.size()] = (int)pro.size();
  if ((rc = up(pro, &d_pro_items, err))) return rc;
  // second stream for the short-range kernel, which overlaps the grid chain
  if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess) {
    if (err) *err = "stream or event creation failed";
    return MSM_ERR_CUDA;
  }
  return MSM_OK;
}

// A new cell for a single-system plan with a tilted cell (msm_plan_set_cell):
// the cell geometry, the SysDev fields that follow from it and the stencils
// (host rebuild with the plan's sizes). The ball columns' centres may move;
// the new halo and widths must fit the plan's (MSM_ERR_CAPACITY otherwise).
int Engine::set_cell_tilted(const double* cell, cudaStream_t s, std::string* err) {
  SysHost& S = sys[0];
  double A[9], Ai[9];
  for (int i = 0; i < 9; i++) A[i] = cell[i];
  const double det = inv3(A, Ai);
  if (!(det > 0.0)) return fail(err, MSM_ERR_INVALID_ARG, "cell rows must form a right-handed basis");
  int Snew[3];
  for (int d = 0; d < 3; d++) {
    double c2 = 0.0;
    for (int e = 0; e < 3; e++) c2 += Ai[3 * e + d] * Ai[3 * e + d];
    Snew[d] = std::max(0, (int)std::ceil(2.0 * S.a * S.M[d] * std::sqrt(c2)) - 1);
    if (Snew[d] > S.R[d] - S.hw)
      return fail(err, MSM_ERR_CAPACITY, "cell compressed or tilted beyond the plan's stencil radius");
  }
  const SysHost keep = S;
  for (int i = 0; i < 9; i++) {
    S.A[i] = A[i];
    S.Ainv[i] = Ai[i];
  }
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) S.Tinv[3 * i + j] = S.Ainv[3 * j + i];
  for (int d = 0; d < 3; d++) {
    const double* u = S.A + 3 * ((d + 1) % 3);
    const double* v = S.A + 3 * ((d + 2) % 3);
    const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
    S.wplane[d] = det / std::sqrt(cx * cx + cy * cy + cz * cz);
    S.L[d] = std::sqrt(A[3 * d] * A[3 * d] + A[3 * d + 1] * A[3 * d + 1] + A[3 * d + 2] * A[3 * d + 2]);
    S.h1[d] = S.L[d] / S.M[d];
    S.S[d] = Snew[d];
    S.edge[d] = S.wplane[d] / S.C[d];
    S.nnbr[d] = (int)std::ceil(S.a / S.edge[d]);
  }
  const int hz_old = keep.hzb, rmax_old = rmax;
  fill_stencils(S, false);
  if (S.has_ball && (S.hzb > hz_old || S.wmax > rmax_old)) {
    S = keep;
    fill_stencils(S, false);
    return fail(err, MSM_ERR_CAPACITY, "the new cell's stencil columns do not fit the plan's halo");
  }
  S.hzb = hz_old;  // the stored rows keep the plan's halo
  SysDev& D = hsys[0];
  for (int d = 0; d < 3; d++) {
    D.Ld[d] = S.L[d];
    D.edged[d] = S.edge[d];
    D.edge[d] = (float)S.edge[d];
    D.invL[d] = (float)(1.0 / S.L[d]);
    D.inv_h1[d] = (float)(1.0 / S.h1[d]);
    D.Lf[d] = (float)S.L[d];
    D.h1f[d] = (float)S.h1[d];
    D.nnbr[d] = S.nnbr[d];
    D.reach[d] = (float)(S.a / S.wplane[d]);
  }
  for (int k = 0; k < 9; k++) {
    D.Tf[k] = (float)S.Tinv[k];
    D.Ad[k] = S.A[k];
    D.Td[k] = S.Tinv[k];
  }
  for (int e = 0; e < 3; e++)
    for (int d = 0; d < 3; d++) D.Jg[3 * e + d] = (float)(S.Ainv[3 * e + d] * S.M[d]);
  int rc = set_cell_host(S.L, s, err, false);
  if (rc) return rc;
  launch_set_sys(d_sys, D, s);
  return MSM_OK;
}

int Engine::set_cell_host(const double Lnew[3], cudaStream_t s, std::string* err, bool refill) {
  SysHost& S = sys[0];
  (void)Lnew;  // the caller has set S.L and S.h1
  if (refill) fill_stencils(S, false);
  std::vector<int> lev0_of(1, hsys[0].lev0);
  std::vector<float> kp;
  std::vector<int> wp;
  assemble_pools(lev0_of, kp, wp);
  if (kp.size() != kpool_n || wp.size() != wpool_n) return fail(err, MSM_ERR_CAPACITY, "stencil pools changed size");
  if (!h_kstage) {
    if (cudaMallocHost((void**)&h_kstage, sizeof(float) * kpool_n) != cudaSuccess ||
        cudaMallocHost((void**)&h_wstage, sizeof(int) * wpool_n) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_stage, cudaEventDisableTiming) != cudaSuccess)
      return fail(err, MSM_ERR_CUDA, "pinned staging buffers for the stencils could not be allocated");
  } else if (cudaEventSynchronize(ev_stage) != cudaSuccess) {  // the previous copy has left the buffers
    return fail(err, MSM_ERR_CUDA, "cudaEventSynchronize failed");
  }
  std::memcpy(h_kstage, kp.data(), sizeof(float) * kpool_n);
  std::memcpy(h_wstage, wp.data(), sizeof(int) * wpool_n);
  if (cudaMemcpyAsync(d_kpool, h_kstage, sizeof(float) * kpool_n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_wpool, h_wstage, sizeof(int) * wpool_n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaEventRecord(ev_stage, s) != cudaSuccess)
    return fail(err, MSM_ERR_CUDA, "stencil upload failed");
  return MSM_OK;
}

Engine::~Engine() {
  if (ev_stage) cudaEventSynchronize(ev_stage);
  if (h_kstage) cudaFreeHost(h_kstage);
  if (h_wstage) cudaFreeHost(h_wstage);
  if (ev_stage) cudaEventDestroy(ev_stage);
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (ev_grad) cudaEventDestroy(ev_grad);
  if (copy) cudaStreamDestroy(copy);
  if (side) cudaStreamDestroy(side);
  cudaFree(d_sys);
  cudaFree(d_lev);
  cudaFree(d_kpool);
  cudaFree(d_wpool);
  cudaFree(d_atom_items);
  cudaFree(d_anterp_items);
  cudaFree(d_acol_items);
  cudaFree(d_asum_items);
  cudaFree(d_ball_items);
  cudaFree(d_box_items);
  cudaFree(d_pad_items);
  cudaFree(d_voff);
  cudaFree(d_voff_spec);
  cudaFree(d_spec_z);
  cudaFree(d_spec_y);
  cudaFree(d_spec_x);
  cudaFree(d_spec_scr_a);
  cudaFree(d_spec_scr_b);
  cudaFree(d_res_items);
  cudaFree(d_pro_items);
  cudaFree(d_energy_scratch);
  cudaFree(d_virial_scratch);
}

Work Engine::resolve(void* ws) const {
  char* b = (char*)ws;
  Work w;
  w.status = (int*)(b + L_status);
  w.cell_count = (int*)(b + L_cell_count);
  w.cell_start = (int*)(b + L_cell_start);
  w.scan_tiles = (int*)(b + L_scan_tiles);
  w.cell_id = (int*)(b + L_cell_id);
  w.slot = (int*)(b + L_slot);
  w.bucket = (int2*)(b + L_bucket);
  w.perm = (int*)(b + L_perm);
  w.iperm = (int*)(b + L_iperm);
  w.scell = (int*)(b + L_scell);
  w.xq = (float4*)(b + L_xq);
  w.uq = (float4*)(b + L_uq);
  w.phi_sr = (float*)(b + L_phi_sr);
  w.phi_lr = (float*)(b + L_phi_lr);
  w.f_sr = (float4*)(b + L_f_sr);
  w.f_lr = (float4*)(b + L_f_lr);
  w.res = (float4*)(b + L_res);
  w.part_e = (float2*)(b + L_part_e);
  w.io_pos = (float*)(b + L_io_pos);
  w.io_q = (float*)(b + L_io_q);
  w.io_dpos = (float*)(b + L_io_dpos);
  w.io_dq = (float*)(b + L_io_dq);
  w.io_e = (double*)(b + L_io_e);
  w.part_q = (float2*)(b + L_part_q);
  w.part_w0 = (double*)(b + L_part_w0);
  w.part_wg = (double*)(b + L_part_wg);
  w.part_vs = (double*)(b + L_part_vs);
  w.grid = (float*)(b + L_grid);
  w.vjp_u = (float4*)(b + L_vjp_u);
  w.vjp_h = (float4*)(b + L_vjp_h);
  w.apart = (float*)(b + L_apart);
  w.spec = (float2*)(b + L_spec);
  return w;
}

Tables Engine::tables() const {
  Tables t;
  t.sys = d_sys;
  t.lev = d_lev;
  t.kpool = d_kpool;
  t.wpool = d_wpool;
  return t;
}

}  // namespace msm
