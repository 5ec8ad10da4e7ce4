/*
 * msm_oracle.c -- plain, slow, FP64 CPU oracle of the B-spline multilevel
 * summation method (MSM) described in arXiv 2510.05961 (msmJAX).
 *
 * TEST INFRASTRUCTURE ONLY. The product library never links, loads or calls
 * this file and shares no header, helper, table or constant with it. Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark use it.
 *
 * Each function names the passage of the paper it restates. The arithmetic is
 * FP64 with plain ordered loops (build with -ffp-contract=off, no fast-math);
 * OpenMP only splits loops whose iterations write disjoint outputs, so every
 * output is summed in the same order with or without threads. The one FP32
 * routine is the cell binning, which follows the FP32 cell-index contract bit
 * for bit (see or_bin).
 *
 * Parity status: every function below is pinned by a CPU test against values
 * that do not come from this file (closed forms, direct sums, Ewald sums, the
 * rock-salt Madelung constant, finite differences, exact invariants).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXLEV 20

/* status bits of or_bin */
#define OR_ST_OUTSIDE 1
#define OR_ST_NONFINITE 2
#define OR_MAXHW 96  /* largest omega' half-width a plan may use */
#define OR_PI 3.14159265358979323846

typedef struct {
  /* inputs */
  double L[3];          /* orthorhombic cell edge lengths */
  int pbc[3];           /* 1 periodic, 0 open */
  double h;             /* target level-1 spacing */
  int grid_override[3]; /* >0: level-1 interval count along that axis */
  double a;             /* level-zero cutoff r_cut^(0) */
  int p;                /* B-spline order (even) */
  int levels;           /* L, 0 = rule below */
  int qi_mode;          /* 0 minimal quasi-interpolation, 1 exact interpolation (or_omega_exact) */
  /* derived by or_plan_init */
  int nlev;             /* number of grid levels L (top level included) */
  int ncomp;            /* levels whose grids are evaluated (nlev, or nlev-1 when the top is dropped) */
  int top_kept;         /* 1 when the top level's stencil is applied (all axes open, a slab or a wire) */
  int M[3];             /* level-1 interval counts */
  double h1[3];         /* level-1 spacings L/M */
  int lo[OR_MAXLEV][3]; /* first grid index per level (index 0 = level 1) */
  int n[OR_MAXLEV][3];  /* grid points per level */
  int S[3];             /* kernel-sample radius of the level stencils */
  int R[3];             /* stencil radius S + hw */
  int hw;               /* half-width of omega': p/2 - 1 (qi_mode 0) or the truncation of or_omega_exact */
  int C[3];             /* binning cells per axis (periodic: M / 2^k, edge <= a/2 (x, y), a/4 (z);
                           open: floor(2L/a) (x, y), floor(4L/a) (z)) */
  double edge[3];       /* binning cell edges */
  int nnbr[3];          /* neighbour-cell reach ceil(a/edge) */
  float invLf[3];       /* (float)(1/L): binning contract */
  /* general (triclinic) cells, Sec. 3.2.2's transform to the unit cube */
  double A[9];          /* input: cell rows a, b, c (row-major); all zero = diag(L) */
  int tri;              /* derived: 1 when A has off-diagonal entries */
  double Ainv[9];       /* A^-1 */
  double Tinv[9];       /* A^-T: fractional coordinates s = A^-T r */
  float Tf[9];          /* (float) A^-T: binning contract of general cells */
  double wplane[3];     /* distances between opposite cell faces, V / |a_e x a_f| */
} or_plan;

/* ------------------------------------------------------------------------ */
/* Softening and splitting, Sec. 3.4, Eq. coulomb_splitting_with_softener.   */
/* ------------------------------------------------------------------------ */

/* c_k = binom(2k,k)/4^k, the magnitude of the k-th Taylor coefficient of
 * s^(-1/2) about s = 1: binom(-1/2,k)(s-1)^k = c_k (1-s)^k. */
static double coef_ck(int k) {
  double c = 1.0;
  for (int j = 1; j <= k; j++) c *= (2.0 * j - 1.0) / (2.0 * j);
  return c;
}

/* gamma(rho): 1/rho for rho >= 1; for rho < 1 the degree p-1 Taylor
 * polynomial of s^(-1/2) about s = 1, evaluated at s = rho^2 (Sec. 3.4). */
double or_gamma(int p, double rho) {
  if (rho >= 1.0) return 1.0 / rho;
  double s = 1.0 - rho * rho, acc = 0.0, pw = 1.0;
  for (int k = 0; k <= p - 1; k++) {
    acc += coef_ck(k) * pw;
    pw *= s;
  }
  return acc;
}

/* d gamma / d rho. */
double or_dgamma(int p, double rho) {
  if (rho >= 1.0) return -1.0 / (rho * rho);
  double s = 1.0 - rho * rho, acc = 0.0, pw = 1.0;
  for (int k = 1; k <= p - 1; k++) {
    acc += coef_ck(k) * k * pw;
    pw *= s;
  }
  return acc * (-2.0 * rho);
}

/* Partial kernel k_l(r), l = 0 .. nlev (Eq. coulomb_splitting_with_softener):
 *   k_0 = 1/r - gamma(r/a)/a,
 *   k_l = gamma(r/(2^(l-1) a))/(2^(l-1) a) - gamma(r/(2^l a))/(2^l a), 1 <= l <= L-1,
 *   k_L = gamma(r/(2^(L-1) a))/(2^(L-1) a).
 * Where gamma = 1/rho in both terms the difference is exactly zero, so
 * k_l(r) = 0 for r >= 2^l a (l < L); that zero is returned as such. */
double or_kl(int p, double a, int nlev, int l, double r) {
  if (l == 0) {
    if (r >= a) return 0.0;
    return 1.0 / r - or_gamma(p, r / a) / a;
  }
  double s1 = ldexp(a, l - 1);
  if (l == nlev) return or_gamma(p, r / s1) / s1;
  double s2 = ldexp(a, l);
  if (r >= s2) return 0.0;
  return or_gamma(p, r / s1) / s1 - or_gamma(p, r / s2) / s2;
}

/* d k_l / d r. */
double or_dkl(int p, double a, int nlev, int l, double r) {
  if (l == 0) {
    if (r >= a) return 0.0;
    return -1.0 / (r * r) - or_dgamma(p, r / a) / (a * a);
  }
  double s1 = ldexp(a, l - 1);
  if (l == nlev) return or_dgamma(p, r / s1) / (s1 * s1);
  double s2 = ldexp(a, l);
  if (r >= s2) return 0.0;
  return or_dgamma(p, r / s1) / (s1 * s1) - or_dgamma(p, r / s2) / (s2 * s2);
}

/* ------------------------------------------------------------------------ */
/* Slab geometry (x, y periodic with edges Lx, Ly; z open): the 2-D lattice  */
/* sums the exact slab top level and the 2-D Ewald pin need.                 */
/* ------------------------------------------------------------------------ */

/* 2-D Ewald split of sum_R 1/|r + R| over R = (i Lx, j Ly, 0) at r = (x, y, z)
 * (the textbook slab Ewald sum):
 *   real space  sum_R erfc(alpha s)/s,  s = |r + R| (R = 0 left out if skip0),
 *   reciprocal  (pi/A) sum_(G != 0) cos(G.rho)/|G| [e^(|G| z) erfc(|G|/(2 alpha) + alpha z)
 *                                                  + e^(-|G| z) erfc(|G|/(2 alpha) - alpha z)],
 *   G = 0       -(2 pi/A) [z erf(alpha z) + exp(-alpha^2 z^2)/(alpha sqrt(pi))],
 * A = Lx Ly, G = 2 pi (i/Lx, j/Ly). The lattice sum itself diverges; this is
 * it without the infinite constant of the G = 0 term, which multiplies the
 * squared total charge and so vanishes for neutral systems. Truncation: real
 * space to |r + R| < 7/alpha, reciprocal space to |G| < 14 alpha (terms below
 * 1e-21 relative). */
/* e^(g z) erfc(g/(2 alpha) + alpha z) without overflow: for a positive erfc
 * argument x it is exp(-g^2/(4 alpha^2) - alpha^2 z^2) erfcx(x), erfcx(x) =
 * e^(x^2) erfc(x) taken directly below x = 10 and from its asymptotic series
 * 1/(x sqrt(pi)) sum_n (-1)^n (2n-1)!!/(2 x^2)^n above (12 terms). */
static double ewald2d_term(double g, double z, double alpha) {
  double x = g / (2.0 * alpha) + alpha * z;
  if (x <= 0.0) return exp(g * z) * erfc(x);
  double ex;
  if (x < 10.0) {
    ex = exp(x * x) * erfc(x);
  } else {
    double t = 1.0, sum = 1.0, inv = 1.0 / (2.0 * x * x);
    for (int k = 1; k <= 12; k++) {
      t *= -(2.0 * k - 1.0) * inv;
      sum += t;
    }
    ex = sum / (x * sqrt(OR_PI));
  }
  return exp(-g * g / (4.0 * alpha * alpha) - alpha * alpha * z * z) * ex;
}

double or_ewald2d_pair(double Lx, double Ly, double x, double y, double z, double alpha, int skip0) {
  const double A = Lx * Ly, rc = 7.0 / alpha, gc = 14.0 * alpha;
  double acc = 0.0;
  int ni = (int)ceil((rc + fabs(x)) / Lx) + 1, nj = (int)ceil((rc + fabs(y)) / Ly) + 1;
  for (int i = -ni; i <= ni; i++)
    for (int j = -nj; j <= nj; j++) {
      if (skip0 && i == 0 && j == 0) continue;
      double dx = x + i * Lx, dy = y + j * Ly;
      double s = sqrt(dx * dx + dy * dy + z * z);
      if (s < rc) acc += erfc(alpha * s) / s;
    }
  int mi = (int)ceil(gc * Lx / (2.0 * OR_PI)) + 1, mj = (int)ceil(gc * Ly / (2.0 * OR_PI)) + 1;
  double rec = 0.0;
  for (int i = -mi; i <= mi; i++)
    for (int j = -mj; j <= mj; j++) {
      if (i == 0 && j == 0) continue;
      double gx = 2.0 * OR_PI * i / Lx, gy = 2.0 * OR_PI * j / Ly;
      double g = sqrt(gx * gx + gy * gy);
      if (g >= gc) continue;
      double t = ewald2d_term(g, z, alpha) + ewald2d_term(g, -z, alpha);
      rec += cos(gx * x + gy * y) / g * t;
    }
  acc += OR_PI / A * rec;
  acc -= 2.0 * OR_PI / A * (z * erf(alpha * z) + exp(-alpha * alpha * z * z) / (alpha * sqrt(OR_PI)));
  return acc;
}

/* 2-D Ewald sum of a neutral slab: phi_i = sum_j q_j psi(r_j - r_i) with psi
 * the pair sum above (R = 0 left out for j = i) minus 2 alpha/sqrt(pi) q_i;
 * E = 1/2 sum q phi. alpha <= 0 picks 6 / min(Lx, Ly). */
void or_ewald2d(double Lx, double Ly, int n, const double* pos, const double* q, double alpha, double* E,
                double* phi) {
  if (alpha <= 0.0) alpha = 6.0 / (Lx < Ly ? Lx : Ly);
#pragma omp parallel for schedule(dynamic, 4)
  for (int i = 0; i < n; i++) {
    double ph = 0.0;
    for (int j = 0; j < n; j++) {
      double dx = pos[3 * j] - pos[3 * i], dy = pos[3 * j + 1] - pos[3 * i + 1], dz = pos[3 * j + 2] - pos[3 * i + 2];
      dx -= Lx * floor(dx / Lx + 0.5);
      dy -= Ly * floor(dy / Ly + 0.5);
      ph += q[j] * or_ewald2d_pair(Lx, Ly, dx, dy, dz, alpha, j == i);
    }
    phi[i] = ph - 2.0 * alpha / sqrt(OR_PI) * q[i];
  }
  double e = 0.0;
  for (int i = 0; i < n; i++) e += 0.5 * q[i] * phi[i];
  *E = e;
}

/* Top-level kernel of a slab (reading of the top level for x, y periodic and
 * z open): the level-L kernel k_L summed over the 2-D lattice, at the pure z
 * offset z. With k_L = 1/r - h_L, h_L(r) = 1/r - gamma(r/a_L)/a_L (zero for
 * r >= a_L, a_L = 2^(L-1) a), the 1/r part is the 2-D Ewald sum above and
 * the h_L part a finite direct sum; at z = 0 the R = 0 term is the limit
 * (erfc(alpha r) - 1)/r + gamma(r/a_L)/a_L -> -2 alpha/sqrt(pi) + gamma(0)/a_L. */
double or_slab_top(int p, double a, int nlev, double Lx, double Ly, double z) {
  const double aL = ldexp(a, nlev - 1), alpha = 6.0 / (Lx < Ly ? Lx : Ly);
  const int zero = fabs(z) < 1e-300;
  double v = or_ewald2d_pair(Lx, Ly, 0.0, 0.0, z, alpha, zero);
  if (zero) v += -2.0 * alpha / sqrt(OR_PI) + or_gamma(p, 0.0) / aL;
  int ni = (int)ceil(aL / Lx) + 1, nj = (int)ceil(aL / Ly) + 1;
  for (int i = -ni; i <= ni; i++)
    for (int j = -nj; j <= nj; j++) {
      if (zero && i == 0 && j == 0) continue;
      double r = sqrt((i * Lx) * (i * Lx) + (j * Ly) * (j * Ly) + z * z);
      if (r < aL) v -= 1.0 / r - or_gamma(p, r / aL) / aL;
    }
  return v;
}

/* ------------------------------------------------------------------------ */
/* Wires (one periodic axis): 1-D Ewald sum and the wire top-level kernel.   */
/* ------------------------------------------------------------------------ */

#define OR_EULER_GAMMA 0.57721566490153286061

/* n-point Gauss-Legendre rule on [-1, 1]: nodes are the roots of P_n, found by
 * Newton's method from cos(pi (i - 1/4) / (n + 1/2)); P_n and P_(n-1) from the
 * three-term recurrence, P_n' = n (x P_n - P_(n-1)) / (x^2 - 1), weights
 * 2 / ((1 - x^2) P_n'^2). */
#define OR_GLN 12
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; i++) {
    double t = cos(OR_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

/* Ein(x) = int_0^x (1 - e^-t)/t dt = sum_(k>=1) (-1)^(k+1) x^k / (k k!)
 * (an entire function; E1(x) = -gamma - ln x + Ein(x)), for 0 <= x < 4. */
static double ein_series(double x) {
  double term = x, sum = x;
  for (int k = 2; k < 200; k++) {
    term *= -x / k;
    double add = term / k;
    sum += add;
    if (fabs(add) < 1e-18 * fabs(sum)) break;
  }
  return sum;
}

/* E1(x) for x >= 1 by the continued fraction
 * E1(x) = e^-x / (x + 1 - 1^2/(x + 3 - 2^2/(x + 5 - ...))), modified Lentz. */
static double e1_cfrac(double x) {
  const double tiny = 1e-300;
  double b = x + 1.0, c = 1.0 / tiny, d = 1.0 / b, h = d;
  for (int k = 1; k < 1000; k++) {
    double an = -(double)k * k;
    b += 2.0;
    d = an * d + b;
    if (fabs(d) < tiny) d = tiny;
    c = b + an / c;
    if (fabs(c) < tiny) c = tiny;
    d = 1.0 / d;
    double del = d * c;
    h *= del;
    if (fabs(del - 1.0) < 1e-16) break;
  }
  return h * exp(-x);
}

/* I(G, rho) = int_0^(alpha^2) u^-1 exp(-u rho^2 - G^2/(4u)) du (G != 0): the
 * Fourier transform along the wire of erf(alpha r)/r at transverse distance
 * rho. With u = alpha^2 e^-s it is int_0^inf exp(-alpha^2 rho^2 e^-s - b e^s) ds,
 * b = G^2/(4 alpha^2), an integrand that dies double-exponentially; the
 * range is cut where b e^s = 46 and split into panels of width 1/2, each
 * summed by a 12-point Gauss-Legendre rule. */
static double wire_fourier(double b, double c2) {
  if (b >= 46.0) return 0.0;
  double x[OR_GLN], w[OR_GLN];
  gauss_legendre(OR_GLN, x, w);
  const double smax = log(46.0 / b);
  const int np = (int)ceil(smax / 0.5);
  const double hw = 0.5 * smax / np;
  double acc = 0.0;
  for (int k = 0; k < np; k++) {
    const double mid = (2 * k + 1) * hw;
    for (int i = 0; i < OR_GLN; i++) {
      const double s = mid + hw * x[i];
      acc += w[i] * exp(-c2 * exp(-s) - b * exp(s));
    }
  }
  return acc * hw;
}

/* 1-D Ewald sum of 1/r over the lattice n L e_z at the offset (rho, z)
 * (rho = transverse distance): with the Poisson sum of the erf part along z,
 *   real space  sum_n erfc(alpha s_n)/s_n,  s_n = |(rho, z + n L)| (n = 0 left
 *               out if skip0),
 *   reciprocal  (2/L) sum_(k >= 1) cos(G_k z) I(G_k, rho), G_k = 2 pi k / L,
 *   G = 0       (1/L) [ln(alpha^2) - Ein(alpha^2 rho^2)]
 *               (= (1/L) [-gamma - ln(rho^2) - E1(alpha^2 rho^2)] for rho > 0).
 * The lattice sum diverges logarithmically; the G = 0 integral is cut at
 * small u and the cut's constant -ln(eps)/L, which depends on neither the
 * offset nor alpha, is left out (it multiplies the squared total charge and
 * vanishes for neutral systems). Truncation: real space to s < 7/alpha,
 * reciprocal space to G^2/(4 alpha^2) < 46. */
double or_ewald1d_pair(double L, double rho, double z, double alpha, int skip0) {
  const double rc = 7.0 / alpha;
  double acc = 0.0;
  const int nr = (int)ceil((rc + fabs(z)) / L) + 1;
  for (int n = -nr; n <= nr; n++) {
    if (skip0 && n == 0) continue;
    double dz = z + n * L;
    double s = sqrt(rho * rho + dz * dz);
    if (s < rc) acc += erfc(alpha * s) / s;
  }
  const double c2 = alpha * alpha * rho * rho;
  double rec = 0.0;
  for (int k = 1;; k++) {
    double g = 2.0 * OR_PI * k / L, b = g * g / (4.0 * alpha * alpha);
    if (b >= 46.0) break;
    rec += cos(g * z) * wire_fourier(b, c2);
  }
  acc += 2.0 / L * rec;
  double g0;
  if (c2 < 4.0)
    g0 = log(alpha * alpha) - ein_series(c2);
  else
    g0 = -OR_EULER_GAMMA - log(rho * rho) - e1_cfrac(c2);
  return acc + g0 / L;
}

/* 1-D Ewald sum of a neutral wire periodic along z with period L (x, y
 * open): phi_i = sum_j q_j psi(r_j - r_i) with psi the pair sum above (n = 0
 * left out for j = i) minus 2 alpha/sqrt(pi) q_i; E = 1/2 sum q phi.
 * alpha <= 0 picks 6 / L. */
void or_ewald1d(double L, int n, const double* pos, const double* q, double alpha, double* E, double* phi) {
  if (alpha <= 0.0) alpha = 6.0 / L;
#pragma omp parallel for schedule(dynamic, 4)
  for (int i = 0; i < n; i++) {
    double ph = 0.0;
    for (int j = 0; j < n; j++) {
      double dx = pos[3 * j] - pos[3 * i], dy = pos[3 * j + 1] - pos[3 * i + 1], dz = pos[3 * j + 2] - pos[3 * i + 2];
      dz -= L * floor(dz / L + 0.5);
      ph += q[j] * or_ewald1d_pair(L, sqrt(dx * dx + dy * dy), dz, alpha, j == i);
    }
    phi[i] = ph - 2.0 * alpha / sqrt(OR_PI) * q[i];
  }
  double e = 0.0;
  for (int i = 0; i < n; i++) e += 0.5 * q[i] * phi[i];
  *E = e;
}

/* Top-level kernel of a wire (reading of the top level for one periodic axis,
 * the grid there has one point per period): k_L summed over the 1-D lattice
 * n L e at the transverse distance rho, without the divergent constant; as
 * for the slab, the 1/r part is the 1-D Ewald sum and the h_L part a finite
 * direct sum, with the R = 0 limit -2 alpha/sqrt(pi) + gamma(0)/a_L at rho = 0. */
double or_wire_top(int p, double a, int nlev, double L, double rho) {
  const double aL = ldexp(a, nlev - 1), alpha = 6.0 / L;
  const int zero = rho < 1e-300;
  double v = or_ewald1d_pair(L, rho, 0.0, alpha, zero);
  if (zero) v += -2.0 * alpha / sqrt(OR_PI) + or_gamma(p, 0.0) / aL;
  const int nn = (int)ceil(aL / L) + 1;
  for (int n = -nn; n <= nn; n++) {
    if (zero && n == 0) continue;
    double r = sqrt(rho * rho + (n * L) * (n * L));
    if (r < aL) v -= 1.0 / r - or_gamma(p, r / aL) / aL;
  }
  return v;
}

/* Top-level kernel of a partially periodic system (one or two periodic
 * axes) at the sample vector v, the periodic axes' periods Lp[d] (entries of
 * open axes unused): two periodic axes give the slab kernel at the offset
 * along the open axis, one the wire kernel at the distance across it. */
static double lattice_top(const or_plan* P, const double* Lp, const double* v) {
  int per[3], opn[3], np = 0, no = 0;
  for (int d = 0; d < 3; d++) {
    if (P->pbc[d])
      per[np++] = d;
    else
      opn[no++] = d;
  }
  if (np == 2) return or_slab_top(P->p, P->a, P->nlev, Lp[per[0]], Lp[per[1]], v[opn[0]]);
  return or_wire_top(P->p, P->a, P->nlev, Lp[per[0]], sqrt(v[opn[0]] * v[opn[0]] + v[opn[1]] * v[opn[1]]));
}

/* Strain derivatives (which = 1..6 for eps_xx, yy, zz, xy, xz, yz) of the
 * lattice-summed top level: d/d eps of lattice_top with the lattice and the
 * offset strained by (1 + eps E_ab), by central differences (step 1e-5; the
 * kernel is smooth in the cell). A diagonal strain of a periodic axis scales
 * its period, of an open axis the offset; a shear that involves a periodic
 * axis has zero derivative (the lattice sum is even under the mirror of that
 * axis); a shear of two open axes (wires) moves the offset. */
static double lattice_top_deps(const or_plan* P, const double* Lp, const double* v, int which) {
  static const int ab[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  const int a = ab[which - 1][0], b = ab[which - 1][1];
  if (a != b && (P->pbc[a] || P->pbc[b])) return 0.0;
  const double e = 1e-5;
  double f[2];
  for (int k = 0; k < 2; k++) {
    const double s = k == 0 ? e : -e;
    double L2[3] = {Lp[0], Lp[1], Lp[2]}, v2[3] = {v[0], v[1], v[2]};
    if (a == b && P->pbc[a])
      L2[a] *= 1.0 + s;
    else
      v2[a] += s * v[b];
    f[k] = lattice_top(P, L2, v2);
  }
  return (f[0] - f[1]) / (2.0 * e);
}

/* ------------------------------------------------------------------------ */
/* B-spline basis, Sec. 3.3 (cardinal B-spline of order p, support p cells). */
/* ------------------------------------------------------------------------ */

/* Centred cardinal B-spline of order q, support (-q/2, q/2), written as the
 * truncated-power sum Phi_q(t) = 1/(q-1)! sum_k (-1)^k C(q,k) (t+q/2-k)_+^(q-1).
 * It is evaluated at -|t| (Phi_q is even), where only the small leading terms
 * of the sum are non-zero. */
double or_bspline(int q, double t) {
  t = -fabs(t);
  double half = 0.5 * q;
  if (t <= -half) return 0.0;
  double fact = 1.0;
  for (int j = 2; j <= q - 1; j++) fact *= j;
  double sum = 0.0, binom = 1.0;
  for (int k = 0; k <= q; k++) {
    double x = t + half - k;
    if (x > 0.0) {
      double pw = 1.0;
      for (int e = 0; e < q - 1; e++) pw *= x;
      sum += (k & 1) ? -binom * pw : binom * pw;
    }
    binom = binom * (q - k) / (k + 1);
  }
  return sum / fact;
}

/* Phi_q'(t) = Phi_{q-1}(t + 1/2) - Phi_{q-1}(t - 1/2). */
double or_dbspline(int q, double t) {
  return or_bspline(q - 1, t + 0.5) - or_bspline(q - 1, t - 0.5);
}

/* Restriction coefficients J_k, k = -p/2 .. p/2 (Eq.
 * restriction_prolongation_explicit_formulas). The paper defers the formula to
 * its Ref. HWX+16; this is the B-spline two-scale relation
 * Phi_p(x/2) = sum_k 2^(1-p) C(p, k+p/2) Phi_p(x-k). Output index k + p/2. */
void or_J(int p, double* J) {
  double binom = 1.0;
  for (int k = 0; k <= p; k++) {
    J[k] = ldexp(binom, 1 - p);
    binom = binom * (p - k) / (k + 1);
  }
}

/* Quasi-interpolation coefficients omega'_j, j = -(p/2-1) .. p/2-1 (output
 * index j + p/2 - 1), of Eq. kernel_stencil_by_conv_with_universal_coeff.
 * The paper does not print them. Reading used: the shortest symmetric sequence
 * whose symbol times the squared B-spline sampling symbol
 * b(theta) = sum_n Phi_p(n) cos(n theta) equals 1 + O(theta^p); i.e. the
 * Taylor coefficients of theta^0 .. theta^(p-2) of omega(theta) b(theta)^2 are
 * 1, 0, ..., 0. This is p/2 linear equations for the p/2 unknowns
 * omega'_0 .. omega'_(p/2-1), solved by Gaussian elimination. */
int or_omega(int p, double* w) {
  int K = p / 2;
  double beta[8], gam[8], fac[20];
  fac[0] = 1.0;
  for (int i = 1; i < 20; i++) fac[i] = fac[i - 1] * i;
  for (int k = 0; k < K; k++) {
    double s = 0.0;
    for (int m = -p / 2; m <= p / 2; m++) s += or_bspline(p, (double)m) * pow((double)m, 2.0 * k);
    beta[k] = ((k & 1) ? -1.0 : 1.0) * s / fac[2 * k];
  }
  for (int k = 0; k < K; k++) {
    gam[k] = 0.0;
    for (int i = 0; i <= k; i++) gam[k] += beta[i] * beta[k - i];
  }
  /* coefficient of theta^(2i) in omega(theta) = w_0 + 2 sum_j w_j cos(j theta):
   * A[i][j] w_j with A[i][0] = [i==0], A[i][j] = 2 (-1)^i j^(2i) / (2i)!. */
  double A[8][8], Mx[8][9];
  for (int i = 0; i < K; i++)
    for (int j = 0; j < K; j++)
      A[i][j] = (j == 0) ? (i == 0 ? 1.0 : 0.0)
                         : 2.0 * ((i & 1) ? -1.0 : 1.0) * pow((double)j, 2.0 * i) / fac[2 * i];
  for (int k = 0; k < K; k++) {
    for (int j = 0; j < K; j++) {
      double s = 0.0;
      for (int i = 0; i <= k; i++) s += A[i][j] * gam[k - i];
      Mx[k][j] = s;
    }
    Mx[k][K] = (k == 0) ? 1.0 : 0.0;
  }
  for (int c = 0; c < K; c++) {
    int piv = c;
    for (int r = c + 1; r < K; r++)
      if (fabs(Mx[r][c]) > fabs(Mx[piv][c])) piv = r;
    if (Mx[piv][c] == 0.0) return -1;
    for (int j = 0; j <= K; j++) {
      double t = Mx[c][j];
      Mx[c][j] = Mx[piv][j];
      Mx[piv][j] = t;
    }
    for (int r = 0; r < K; r++) {
      if (r == c) continue;
      double f = Mx[r][c] / Mx[c][c];
      for (int j = c; j <= K; j++) Mx[r][j] -= f * Mx[c][j];
    }
  }
  for (int j = 0; j < K; j++) {
    double v = Mx[j][K] / Mx[j][j];
    w[(K - 1) + j] = v;
    w[(K - 1) - j] = v;
  }
  return 0;
}

/* Exact-interpolation coefficients (qi_mode 1): omega' = omega * omega with
 * omega the inverse of the sampled B-spline b_n = Phi_p(n), i.e. the Fourier
 * coefficients of 1 / b(theta)^2, b(theta) = sum_n Phi_p(n) cos(n theta) > 0:
 *   omega'_n = (1/2 pi) int_(-pi)^(pi) cos(n theta) / b(theta)^2 d theta,
 * evaluated by the trapezoidal rule on 4096 points (exponentially accurate for
 * this analytic periodic integrand). Reading of the truncation: keep |n| <= hw,
 * hw the largest n with |omega'_n| >= 1e-12 |omega'_0| (FP64 resolves the
 * coefficients to about 1e-16 |omega'_0|, so a 1e-17 cut cannot be decided;
 * FP32 stencils resolve neither). w receives omega'_(-hw) .. omega'_(hw), at
 * most 2 maxhw + 1 values; returns hw, or -1 if maxhw is too small. */
int or_omega_exact(int p, double* w, int maxhw) {
  const int N = 4096, H = p / 2;
  double bn[8];
  for (int m = 0; m < H; m++) bn[m] = or_bspline(p, (double)m);
  double* f = (double*)malloc(sizeof(double) * N);
  for (int j = 0; j < N; j++) {
    double th = 2.0 * OR_PI * j / N, b = bn[0];
    for (int m = 1; m < H; m++) b += 2.0 * bn[m] * cos(m * th);
    f[j] = 1.0 / (b * b);
  }
  double c[256];
  int lim = maxhw + 1 < 255 ? maxhw + 1 : 255;
  for (int n = 0; n <= lim; n++) {
    double s = 0.0;
    for (int j = 0; j < N; j++) s += f[j] * cos(2.0 * OR_PI * (double)((long)n * j % N) / N);
    c[n] = s / N;
  }
  free(f);
  int hw = -1;
  for (int n = 0; n <= lim; n++)
    if (fabs(c[n]) >= 1e-12 * fabs(c[0])) hw = n;
  if (hw >= lim) return -1;
  for (int n = -hw; n <= hw; n++) w[n + hw] = c[n < 0 ? -n : n];
  return hw;
}

/* omega' of the plan's interpolation mode, indices -hw .. hw (w needs 2 hw + 1) */
static void plan_omega(const or_plan* P, double* w) {
  if (P->qi_mode == 1) or_omega_exact(P->p, w, P->hw);
  else or_omega(P->p, w);
}

/* ------------------------------------------------------------------------ */
/* Grid set-up (Sec. 4.1 for periodic axes; readings for open axes).         */
/* ------------------------------------------------------------------------ */

static int floordiv(int a, int b) { int q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) q--; return q; }
static int ceildiv(int a, int b) { return -floordiv(-a, b); }

/* Fills the derived fields. Returns 0, 1 (invalid argument) or 2 (unsupported).
 * Periodic axes: M = 2^round(log2(L/h)) (or the override, a power of two), all
 * periodic axes equal, spacing doubled until one point remains (Sec. 4.1), so
 * L = log2(M) + 1 and the one-point top level is not evaluated. Open axes:
 * M = ceil(L/h), level-1 indices [-p/2, M+p/2], each coarser level keeping the
 * indices that restriction can reach; with every axis open the top level is
 * evaluated with its full-range stencil. */
static void mat_inv3(const double* m, double* inv, double* det) {
  double c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8], c02 = m[3] * m[7] - m[4] * m[6];
  double d = m[0] * c00 + m[1] * c01 + m[2] * c02;
  *det = d;
  inv[0] = c00 / d;
  inv[1] = (m[2] * m[7] - m[1] * m[8]) / d;
  inv[2] = (m[1] * m[5] - m[2] * m[4]) / d;
  inv[3] = c01 / d;
  inv[4] = (m[0] * m[8] - m[2] * m[6]) / d;
  inv[5] = (m[2] * m[3] - m[0] * m[5]) / d;
  inv[6] = c02 / d;
  inv[7] = (m[1] * m[6] - m[0] * m[7]) / d;
  inv[8] = (m[0] * m[4] - m[1] * m[3]) / d;
}

/* general cells: rows a, b, c of A; lengths, A^-1, A^-T, face distances.
 * Returns 1 for a degenerate or left-handed cell, 2 for a tilted cell with
 * an open axis (not supported). */
static int plan_cell(or_plan* P) {
  int any = 0;
  for (int k = 0; k < 9; k++) if (P->A[k] != 0.0) any = 1;
  if (!any) {
    for (int d = 0; d < 3; d++) P->A[4 * d] = P->L[d];
  } else {
    for (int d = 0; d < 3; d++)
      P->L[d] = sqrt(P->A[3 * d] * P->A[3 * d] + P->A[3 * d + 1] * P->A[3 * d + 1] + P->A[3 * d + 2] * P->A[3 * d + 2]);
  }
  P->tri = 0;
  for (int k = 0; k < 9; k++) if (k % 4 != 0 && P->A[k] != 0.0) P->tri = 1;
  if (P->tri && !(P->pbc[0] && P->pbc[1] && P->pbc[2])) return 2;
  double det;
  mat_inv3(P->A, P->Ainv, &det);
  if (!(det > 0.0)) return 1;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      P->Tinv[3 * i + j] = P->Ainv[3 * j + i];
      P->Tf[3 * i + j] = (float)P->Tinv[3 * i + j];
    }
  for (int d = 0; d < 3; d++) {
    const double* u = P->A + 3 * ((d + 1) % 3);
    const double* v = P->A + 3 * ((d + 2) % 3);
    double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
    P->wplane[d] = det / sqrt(cx * cx + cy * cy + cz * cz);
  }
  return 0;
}

int or_plan_init(or_plan* P) {
  int p = P->p;
  if (p != 4 && p != 6 && p != 8) return 1;
  {
    int rc = plan_cell(P);
    if (rc) return rc;
  }
  if (P->qi_mode != 0 && P->qi_mode != 1) return 1;
  if (P->qi_mode == 1) {
    double tmp[2 * OR_MAXHW + 1];
    P->hw = or_omega_exact(p, tmp, OR_MAXHW);
    if (P->hw < 0) return 1;
  } else {
    P->hw = p / 2 - 1;
  }
  if (!(P->a > 0.0)) return 1;
  int anyper = 0, Mper = 0;
  for (int d = 0; d < 3; d++) {
    if (!(P->L[d] > 0.0)) return 1;
    int M;
    if (P->grid_override[d] > 0) {
      M = P->grid_override[d];
    } else {
      if (!(P->h > 0.0)) return 1;
      if (P->pbc[d]) {
        int e = (int)floor(log2(P->L[d] / P->h) + 0.5);
        if (e < 1) e = 1;
        if (e > 16) return 2;
        M = 1 << e;
      } else {
        M = (int)ceil(P->L[d] / P->h);
        if (M < 1) M = 1;
      }
    }
    if (P->pbc[d]) {
      if (M < 2 || (M & (M - 1)) != 0) return 2;
      if (anyper && M != Mper) return 2;
      anyper = 1;
      Mper = M;
    }
    P->M[d] = M;
    P->h1[d] = P->L[d] / M;
  }
  int hp = p / 2;
  if (anyper) {
    int nl = 1;
    while ((1 << (nl - 1)) < Mper) nl++;
    if (P->levels > 0 && P->levels != nl) return 2;
    P->nlev = nl;
    if (!(P->pbc[0] && P->pbc[1] && P->pbc[2])) {
      /* slab (two periodic axes) or wire (one): the top level, one point per
       * period along the periodic axes, is kept, with k_L summed over the
       * 2-D (or_slab_top) or 1-D (or_wire_top) lattice */
      P->top_kept = 1;
      P->ncomp = nl;
    } else {
      P->top_kept = 0;
      P->ncomp = nl - 1;
    }
  } else {
    P->top_kept = 1;
    P->nlev = P->levels;
  }
  /* level index ranges */
  for (int d = 0; d < 3; d++) {
    if (P->pbc[d]) continue;
    P->lo[0][d] = -hp;
    P->n[0][d] = P->M[d] + p + 1;
  }
  int maxlev = OR_MAXLEV;
  for (int l = 1; l < maxlev; l++) {
    for (int d = 0; d < 3; d++) {
      if (P->pbc[d]) continue;
      int lo = P->lo[l - 1][d], hi = lo + P->n[l - 1][d] - 1;
      int nlo = ceildiv(lo - hp, 2), nhi = floordiv(hi + hp, 2);
      P->lo[l][d] = nlo;
      P->n[l][d] = nhi - nlo + 1;
    }
  }
  if (!anyper && P->nlev <= 0) {
    int cap = (p + 1 > 8) ? p + 1 : 8;
    int l = 1;
    for (;; l++) {
      int ok = 1;
      for (int d = 0; d < 3; d++) if (P->n[l - 1][d] > cap) ok = 0;
      if (ok || l == OR_MAXLEV) break;
    }
    P->nlev = l;
  }
  if (P->nlev < 1 || P->nlev > OR_MAXLEV) return 2;
  if (!anyper) P->ncomp = P->nlev;
  for (int l = 0; l < OR_MAXLEV; l++)
    for (int d = 0; d < 3; d++)
      if (P->pbc[d]) {
        P->lo[l][d] = 0;
        P->n[l][d] = (l < P->nlev) ? (P->M[d] >> l) : 1;
        if (P->n[l][d] < 1) P->n[l][d] = 1;
      }
  for (int d = 0; d < 3; d++) {
    if (!P->tri) {
      P->S[d] = (int)ceil(2.0 * P->a / P->h1[d]) - 1;
    } else {
      /* tilted cell: the samples |A^T (n / M)| < 2a lie in an ellipsoid whose
       * extent along index axis d is 2a M_d sqrt((G^-1)_dd), G = A A^T, and
       * (G^-1)_dd is the squared length of the d-th column of A^-1 */
      double c2 = 0.0;
      for (int e = 0; e < 3; e++) c2 += P->Ainv[3 * e + d] * P->Ainv[3 * e + d];
      P->S[d] = (int)ceil(2.0 * P->a * P->M[d] * sqrt(c2)) - 1;
    }
    if (P->S[d] < 0) P->S[d] = 0;
    P->R[d] = P->S[d] + P->hw;
    int C;
    /* spacing of the grid planes across axis d (h_1 for a rectangular cell) */
    const double hp = P->tri ? P->wplane[d] / P->M[d] : P->h1[d];
    if (P->pbc[d]) {
      /* periodic axis: cells of k level-1 intervals, k the largest power of
       * two with k h_1 <= a/2 for x, y and <= a/4 for z (at least 1), at
       * most 512 cells; h_1 is the spacing of the grid planes */
      const double lim = (d == 2 ? 0.25 : 0.5) * P->a;
      int k = 1;
      while (2 * k <= P->M[d] && 2 * k * hp <= lim) k *= 2;
      while (P->M[d] / k > 512) k *= 2;
      C = P->M[d] / k;
    } else {
      /* open axis: floor(2 L / a) cells for x, y and floor(4 L / a) for z, 1 .. 256 */
      C = (int)floor((d == 2 ? 4.0 : 2.0) * P->L[d] / P->a);
      if (C < 1) C = 1;
      if (C > 256) C = 256;
    }
    P->C[d] = C;
    P->edge[d] = (P->tri ? P->wplane[d] : P->L[d]) / C;  /* distance between cell faces */
    P->nnbr[d] = (int)ceil(P->a / P->edge[d]);
    P->invLf[d] = (float)(1.0 / P->L[d]);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Cell binning: the FP32 cell-index contract (bit-exact with the GPU).      */
/* ------------------------------------------------------------------------ */

/* Cell of each atom and the stable counting sort by cell. Per axis, in FP32
 * with round-to-nearest and no contraction:
 *   s = x * (float)(1/L);  periodic: s = s - floorf(s), s >= 1 -> 0;
 *   open: s outside [0,1] -> status OUTSIDE (axis cell 0);
 *   c = min((int)(s * (float)C), C - 1);  cell = (cx*Cy + cy)*Cz + cz.
 * Non-finite coordinates or charges set status NONFINITE (axis cell 0).
 * Within a cell, atoms keep ascending original index. */
int or_bin(const or_plan* P, int n, const float* pos, const float* q, int* cell_id, int* cell_start,
           int* perm) {
  int status = 0;
  int ncell = P->C[0] * P->C[1] * P->C[2];
  for (int i = 0; i < n; i++) {
    int c[3];
    if (!isfinite(q[i])) status |= OR_ST_NONFINITE;
    for (int d = 0; d < 3; d++) {
      float x = pos[3 * i + d];
      c[d] = 0;
      if (!isfinite(x)) { status |= OR_ST_NONFINITE; continue; }
      float s = x * P->invLf[d];
      if (P->tri) {
        /* general cell: s_d = ((T_d0 x + T_d1 y) + T_d2 z), FP32, each product and
         * sum rounded once (T = (float) A^-T); a rectangular cell gives exactly
         * the single product above */
        const float* Tr = P->Tf + 3 * d;
        s = ((Tr[0] * pos[3 * i]) + (Tr[1] * pos[3 * i + 1])) + (Tr[2] * pos[3 * i + 2]);
        if (!isfinite(pos[3 * i]) || !isfinite(pos[3 * i + 1]) || !isfinite(pos[3 * i + 2])) {
          status |= OR_ST_NONFINITE;
          continue;
        }
      }
      if (P->pbc[d]) {
        s = s - floorf(s);
        if (s >= 1.0f) s = 0.0f;
      } else if (!(s >= 0.0f && s <= 1.0f)) {
        status |= OR_ST_OUTSIDE;
        continue;
      }
      float t = s * (float)P->C[d];
      int ci = (int)t;
      if (ci > P->C[d] - 1) ci = P->C[d] - 1;
      c[d] = ci;
    }
    cell_id[i] = (c[0] * P->C[1] + c[1]) * P->C[2] + c[2];
  }
  for (int c = 0; c <= ncell; c++) cell_start[c] = 0;
  for (int i = 0; i < n; i++) cell_start[cell_id[i] + 1]++;
  for (int c = 0; c < ncell; c++) cell_start[c + 1] += cell_start[c];
  int* cursor = (int*)malloc(sizeof(int) * (ncell > 0 ? ncell : 1));
  for (int c = 0; c < ncell; c++) cursor[c] = cell_start[c];
  for (int i = 0; i < n; i++) perm[cursor[cell_id[i]]++] = i;
  free(cursor);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Grid helpers                                                              */
/* ------------------------------------------------------------------------ */

static int lev_size(const or_plan* P, int l) { /* l is 1-based */
  return P->n[l - 1][0] * P->n[l - 1][1] * P->n[l - 1][2];
}

/* storage index of grid point m on axis d of level l, or -1 when an open axis
 * has no such point. Periodic axes wrap. */
static int gidx(const or_plan* P, int l, int d, int m) {
  int nn = P->n[l - 1][d];
  if (P->pbc[d]) {
    int r = m % nn;
    return r < 0 ? r + nn : r;
  }
  int i = m - P->lo[l - 1][d];
  return (i >= 0 && i < nn) ? i : -1;
}

/* level-1 grid coordinate u = x / h_1 of a Cartesian coordinate (periodic axes
 * wrapped into the cell first). */
static double to_u(const or_plan* P, int d, double x) {
  if (P->pbc[d]) x = x - P->L[d] * floor(x / P->L[d]);
  return x / P->h1[d];
}

/* level-1 grid coordinates of atom position r: u = M o s, s = A^-T r wrapped
 * into [0, 1) (general cells; rectangular cells use to_u per axis) */
static void atom_u(const or_plan* P, const double* r, double* u) {
  for (int d = 0; d < 3; d++) {
    if (!P->tri) {
      u[d] = to_u(P, d, r[d]);
      continue;
    }
    double sd = P->Tinv[3 * d] * r[0] + P->Tinv[3 * d + 1] * r[1] + P->Tinv[3 * d + 2] * r[2];
    sd -= floor(sd);
    u[d] = sd * P->M[d];
  }
}

/* ------------------------------------------------------------------------ */
/* Anterpolation, interpolation (Sec. 3.2.2, Alg. anterpolation_double_loop,  */
/* Eqs. grid_charge, uoneplus_interpolation_with_index_set,                  */
/* analytic_uoneplus_position_grad / _charge_grad).                           */
/* ------------------------------------------------------------------------ */

/* q~^1_m = sum_i q_i phi^1_m(r_i), phi^1_m(r) = prod_d Phi_p(u_d - m_d),
 * summed over the index set m_d in {floor(u_d)-p/2+1 .. floor(u_d)+p/2}. */
void or_anterp(const or_plan* P, int n, const double* pos, const double* q, double* grid) {
  int p = P->p, nsz = lev_size(P, 1);
  int ny = P->n[0][1], nz = P->n[0][2];
  for (int k = 0; k < nsz; k++) grid[k] = 0.0;
  for (int i = 0; i < n; i++) {
    int base[3], idx[3][8];
    double w[3][8], uu[3];
    atom_u(P, pos + 3 * i, uu);
    for (int d = 0; d < 3; d++) {
      double u = uu[d];
      base[d] = (int)floor(u) - p / 2 + 1;
      for (int j = 0; j < p; j++) {
        w[d][j] = or_bspline(p, u - (base[d] + j));
        idx[d][j] = gidx(P, 1, d, base[d] + j);
      }
    }
    for (int jx = 0; jx < p; jx++)
      for (int jy = 0; jy < p; jy++)
        for (int jz = 0; jz < p; jz++) {
          if (idx[0][jx] < 0 || idx[1][jy] < 0 || idx[2][jz] < 0) continue;
          grid[(idx[0][jx] * ny + idx[1][jy]) * nz + idx[2][jz]] += q[i] * w[0][jx] * w[1][jy] * w[2][jz];
        }
  }
}

/* phi1_i = sum_m e_m phi^1_m(r_i); grad_i = q_i sum_m e_m grad phi^1_m(r_i);
 * F1_i = -grad_i. d phi_m / d x_d = Phi_p'(u_d - m_d) / h_1d times the other two
 * factors. F1 may be NULL. */
void or_interp(const or_plan* P, int n, const double* pos, const double* q, const double* e,
               double* phi1, double* F1) {
  int p = P->p;
  int ny = P->n[0][1], nz = P->n[0][2];
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; i++) {
    int base[3], idx[3][8];
    double w[3][8], dw[3][8], uu[3];
    atom_u(P, pos + 3 * i, uu);
    for (int d = 0; d < 3; d++) {
      double u = uu[d];
      base[d] = (int)floor(u) - p / 2 + 1;
      for (int j = 0; j < p; j++) {
        w[d][j] = or_bspline(p, u - (base[d] + j));
        /* d/dx_d for rectangular cells; d/du_d for general cells (mapped below) */
        dw[d][j] = or_dbspline(p, u - (base[d] + j)) / (P->tri ? 1.0 : P->h1[d]);
        idx[d][j] = gidx(P, 1, d, base[d] + j);
      }
    }
    double ph = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int jx = 0; jx < p; jx++)
      for (int jy = 0; jy < p; jy++)
        for (int jz = 0; jz < p; jz++) {
          if (idx[0][jx] < 0 || idx[1][jy] < 0 || idx[2][jz] < 0) continue;
          double ev = e[(idx[0][jx] * ny + idx[1][jy]) * nz + idx[2][jz]];
          ph += ev * w[0][jx] * w[1][jy] * w[2][jz];
          gx += ev * dw[0][jx] * w[1][jy] * w[2][jz];
          gy += ev * w[0][jx] * dw[1][jy] * w[2][jz];
          gz += ev * w[0][jx] * w[1][jy] * dw[2][jz];
        }
    phi1[i] = ph;
    if (P->tri) {
      /* grad_r = A^-1 diag(M) grad_u (u = M o A^-T r) */
      double gu[3] = {gx, gy, gz};
      double gr[3];
      for (int e = 0; e < 3; e++)
        gr[e] = P->Ainv[3 * e] * P->M[0] * gu[0] + P->Ainv[3 * e + 1] * P->M[1] * gu[1] + P->Ainv[3 * e + 2] * P->M[2] * gu[2];
      gx = gr[0];
      gy = gr[1];
      gz = gr[2];
    }
    if (F1) {
      F1[3 * i + 0] = -q[i] * gx;
      F1[3 * i + 1] = -q[i] * gy;
      F1[3 * i + 2] = -q[i] * gz;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Restriction and prolongation, Eq. restriction_prolongation_explicit_formulas */
/* ------------------------------------------------------------------------ */

/* q~^(l+1)_m = sum_n J_(n - 2m) q~^l_n, with J_n = J_nx J_ny J_nz (l 1-based).
 * Periodic axes wrap the fine index; open axes drop indices outside the grid. */
void or_restrict(const or_plan* P, int l, const double* fine, double* coarse) {
  int p = P->p, hp = p / 2;
  double J[9];
  or_J(p, J);
  int* nc = (int*)P->n[l];
  int* nf = (int*)P->n[l - 1];
#pragma omp parallel for schedule(static)
  for (int cx = 0; cx < nc[0]; cx++)
    for (int cy = 0; cy < nc[1]; cy++)
      for (int cz = 0; cz < nc[2]; cz++) {
        int m[3] = {cx + P->lo[l][0], cy + P->lo[l][1], cz + P->lo[l][2]};
        double acc = 0.0;
        for (int kx = -hp; kx <= hp; kx++) {
          int fx = gidx(P, l, 0, 2 * m[0] + kx);
          if (fx < 0) continue;
          for (int ky = -hp; ky <= hp; ky++) {
            int fy = gidx(P, l, 1, 2 * m[1] + ky);
            if (fy < 0) continue;
            for (int kz = -hp; kz <= hp; kz++) {
              int fz = gidx(P, l, 2, 2 * m[2] + kz);
              if (fz < 0) continue;
              acc += J[kx + hp] * J[ky + hp] * J[kz + hp] * fine[(fx * nf[1] + fy) * nf[2] + fz];
            }
          }
        }
        coarse[(cx * nc[1] + cy) * nc[2] + cz] = acc;
      }
}

/* fine += I^T coarse, the transpose of or_restrict: (I^T e)_m = sum_n J_(m-2n) e_n.
 * Written as the scatter of each coarse value to the fine points it came from,
 * which is the transpose on periodic (wrapped) and open grids alike. */
void or_prolong_add(const or_plan* P, int l, const double* coarse, double* fine) {
  int p = P->p, hp = p / 2;
  double J[9];
  or_J(p, J);
  int* nc = (int*)P->n[l];
  int* nf = (int*)P->n[l - 1];
  for (int cx = 0; cx < nc[0]; cx++)
    for (int cy = 0; cy < nc[1]; cy++)
      for (int cz = 0; cz < nc[2]; cz++) {
        int m[3] = {cx + P->lo[l][0], cy + P->lo[l][1], cz + P->lo[l][2]};
        double ev = coarse[(cx * nc[1] + cy) * nc[2] + cz];
        for (int kx = -hp; kx <= hp; kx++) {
          int fx = gidx(P, l, 0, 2 * m[0] + kx);
          if (fx < 0) continue;
          for (int ky = -hp; ky <= hp; ky++) {
            int fy = gidx(P, l, 1, 2 * m[1] + ky);
            if (fy < 0) continue;
            for (int kz = -hp; kz <= hp; kz++) {
              int fz = gidx(P, l, 2, 2 * m[2] + kz);
              if (fz < 0) continue;
              fine[(fx * nf[1] + fy) * nf[2] + fz] += J[kx + hp] * J[ky + hp] * J[kz + hp] * ev;
            }
          }
        }
      }
}

/* ------------------------------------------------------------------------ */
/* Stencils K^l, Eq. kernel_stencil_by_conv_with_universal_coeff, and their  */
/* strain derivatives.                                                       */
/* ------------------------------------------------------------------------ */

/* Offset box of the stencil applied on level l (1-based): d in [lo, lo+sz).
 * Levels below the top: [-R, R] per axis. Top level kept (all axes open, a slab or a wire): the
 * full range of grid displacements. Periodic axes are folded onto [0, n_l):
 * on a periodic grid the operator sums every image of an offset. */
void or_stencil_box(const or_plan* P, int l, int* lo, int* sz) {
  for (int d = 0; d < 3; d++) {
    if (P->pbc[d]) {
      lo[d] = 0;
      sz[d] = P->n[l - 1][d];
    } else if (l == P->nlev) {
      lo[d] = -(P->n[l - 1][d] - 1);
      sz[d] = 2 * P->n[l - 1][d] - 1;
    } else {
      lo[d] = -P->R[d];
      sz[d] = 2 * P->R[d] + 1;
    }
  }
}

/* Stencil of level l (1-based) on its box (or_stencil_box), which = 0 for K^l,
 * 1..6 for dK^l/d eps_ab with ab = xx, yy, zz, xy, xz, yz. G (row-major 3x3,
 * NULL = identity) maps the grid displacement h_l o n to the sample vector
 * v = G (h_l o n), so a strained cell can be evaluated for finite differences.
 * Sample values: which 0: k_l(|v|); which > 0: k_l'(|v|) v_a v_b / |v| (0 at v = 0).
 * K_m = sum_n omega'_(mx-nx) omega'_(my-ny) omega'_(mz-nz) sample(n), applied
 * one axis at a time; periodic axes then folded onto [0, n_l). */
void or_stencil_build(const or_plan* P, int l, int which, const double* G, double* out) {
  int p = P->p, r = P->hw;
  double om[2 * OR_MAXHW + 1];
  plan_omega(P, om);
  /* unfolded output box */
  int olo[3], osz[3], slo[3], ssz[3];
  for (int d = 0; d < 3; d++) {
    if (l == P->nlev) {
      olo[d] = -(P->n[l - 1][d] - 1);
      osz[d] = 2 * P->n[l - 1][d] - 1;
    } else {
      olo[d] = -P->R[d];
      osz[d] = 2 * P->R[d] + 1;
    }
    slo[d] = olo[d] - r;
    ssz[d] = osz[d] + 2 * r;
  }
  double hl[3];
  for (int d = 0; d < 3; d++) hl[d] = ldexp(P->h1[d], l - 1);
  int ab[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  const int npbc = P->pbc[0] + P->pbc[1] + P->pbc[2];
  const int lat_top = l == P->nlev && npbc >= 1 && npbc <= 2;
  size_t ns = (size_t)ssz[0] * ssz[1] * ssz[2];
  double* smp = (double*)malloc(sizeof(double) * ns);
#pragma omp parallel for schedule(static)
  for (int ix = 0; ix < ssz[0]; ix++)
    for (int iy = 0; iy < ssz[1]; iy++)
      for (int iz = 0; iz < ssz[2]; iz++) {
        double g[3] = {hl[0] * (ix + slo[0]), hl[1] * (iy + slo[1]), hl[2] * (iz + slo[2])};
        if (P->tri) {
          /* general cell: the grid displacement n (level-l index steps) is the
           * Cartesian vector sum_d n_d 2^(l-1) / M_d a_d */
          double f[3] = {ldexp((double)(ix + slo[0]), l - 1) / P->M[0], ldexp((double)(iy + slo[1]), l - 1) / P->M[1],
                         ldexp((double)(iz + slo[2]), l - 1) / P->M[2]};
          for (int c = 0; c < 3; c++) g[c] = f[0] * P->A[c] + f[1] * P->A[3 + c] + f[2] * P->A[6 + c];
        }
        double v[3];
        for (int a = 0; a < 3; a++)
          v[a] = G ? G[3 * a + 0] * g[0] + G[3 * a + 1] * g[1] + G[3 * a + 2] * g[2] : g[a];
        double rr = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double val;
        if (lat_top) {
          /* offsets along the periodic axes are lattice vectors here: the
           * lattice sum depends on the open components only (a strain G, if
           * given, scales the periods by its diagonal) */
          double Lp[3];
          for (int d = 0; d < 3; d++) Lp[d] = P->L[d] * (G ? G[4 * d] : 1.0);
          val = which == 0 ? lattice_top(P, Lp, v) : lattice_top_deps(P, Lp, v, which);
        } else if (which == 0) {
          val = or_kl(p, P->a, P->nlev, l, rr);
        } else {
          int a = ab[which - 1][0], b = ab[which - 1][1];
          val = (rr > 0.0) ? or_dkl(p, P->a, P->nlev, l, rr) * v[a] * v[b] / rr : 0.0;
        }
        smp[((size_t)ix * ssz[1] + iy) * ssz[2] + iz] = val;
      }
  /* z pass: A[nx][ny][mz] = sum_t omega'_t smp[nx][ny][mz - t] */
  size_t nA = (size_t)ssz[0] * ssz[1] * osz[2];
  double* A = (double*)malloc(sizeof(double) * nA);
  for (int ix = 0; ix < ssz[0]; ix++)
    for (int iy = 0; iy < ssz[1]; iy++)
      for (int mz = 0; mz < osz[2]; mz++) {
        double acc = 0.0;
        for (int t = -r; t <= r; t++)
          acc += om[t + r] * smp[((size_t)ix * ssz[1] + iy) * ssz[2] + (mz + r - t)];
        A[((size_t)ix * ssz[1] + iy) * osz[2] + mz] = acc;
      }
  size_t nB = (size_t)ssz[0] * osz[1] * osz[2];
  double* B = (double*)malloc(sizeof(double) * nB);
  for (int ix = 0; ix < ssz[0]; ix++)
    for (int my = 0; my < osz[1]; my++)
      for (int mz = 0; mz < osz[2]; mz++) {
        double acc = 0.0;
        for (int t = -r; t <= r; t++)
          acc += om[t + r] * A[((size_t)ix * ssz[1] + (my + r - t)) * osz[2] + mz];
        B[((size_t)ix * osz[1] + my) * osz[2] + mz] = acc;
      }
  size_t nK = (size_t)osz[0] * osz[1] * osz[2];
  double* Kb = (double*)malloc(sizeof(double) * nK);
  for (int mx = 0; mx < osz[0]; mx++)
    for (int my = 0; my < osz[1]; my++)
      for (int mz = 0; mz < osz[2]; mz++) {
        double acc = 0.0;
        for (int t = -r; t <= r; t++)
          acc += om[t + r] * B[((size_t)(mx + r - t) * osz[1] + my) * osz[2] + mz];
        Kb[((size_t)mx * osz[1] + my) * osz[2] + mz] = acc;
      }
  /* fold periodic axes */
  int flo[3], fsz[3];
  or_stencil_box(P, l, flo, fsz);
  size_t nF = (size_t)fsz[0] * fsz[1] * fsz[2];
  for (size_t k = 0; k < nF; k++) out[k] = 0.0;
  for (int mx = 0; mx < osz[0]; mx++)
    for (int my = 0; my < osz[1]; my++)
      for (int mz = 0; mz < osz[2]; mz++) {
        int m[3] = {mx + olo[0], my + olo[1], mz + olo[2]}, f[3];
        for (int d = 0; d < 3; d++) {
          if (P->pbc[d]) {
            int r2 = m[d] % fsz[d];
            f[d] = r2 < 0 ? r2 + fsz[d] : r2;
          } else {
            f[d] = m[d] - flo[d];
          }
        }
        out[((size_t)f[0] * fsz[1] + f[1]) * fsz[2] + f[2]] += Kb[((size_t)mx * osz[1] + my) * osz[2] + mz];
      }
  free(smp);
  free(A);
  free(B);
  free(Kb);
}

/* e_m = sum_d K_d q_(m-d) (Eq. action_of_K_as_convolution) on level l; periodic
 * axes wrap, open axes drop indices outside the grid. Zero stencil entries are
 * skipped. */
void or_stencil_apply(const or_plan* P, int l, const double* K, const double* qg, double* eg) {
  int klo[3], ksz[3];
  or_stencil_box(P, l, klo, ksz);
  int* nn = (int*)P->n[l - 1];
  int* lo = (int*)P->lo[l - 1];
  size_t nK = (size_t)ksz[0] * ksz[1] * ksz[2];
  int* nzl = (int*)malloc(sizeof(int) * (nK > 0 ? nK : 1));
  size_t nnz = 0;
  for (size_t k = 0; k < nK; k++) if (K[k] != 0.0) nzl[nnz++] = (int)k;
#pragma omp parallel for schedule(dynamic, 1)
  for (int ix = 0; ix < nn[0]; ix++)
    for (int iy = 0; iy < nn[1]; iy++)
      for (int iz = 0; iz < nn[2]; iz++) {
        int m[3] = {ix + lo[0], iy + lo[1], iz + lo[2]};
        double acc = 0.0;
        for (size_t t = 0; t < nnz; t++) {
          int k = nzl[t];
          int d[3] = {k / (ksz[1] * ksz[2]) + klo[0], (k / ksz[2]) % ksz[1] + klo[1], k % ksz[2] + klo[2]};
          int sx = gidx(P, l, 0, m[0] - d[0]);
          if (sx < 0) continue;
          int sy = gidx(P, l, 1, m[1] - d[1]);
          if (sy < 0) continue;
          int sz2 = gidx(P, l, 2, m[2] - d[2]);
          if (sz2 < 0) continue;
          acc += K[k] * qg[((size_t)sx * nn[1] + sy) * nn[2] + sz2];
        }
        eg[((size_t)ix * nn[1] + iy) * nn[2] + iz] = acc;
      }
  free(nzl);
}

/* Grid part of the virial on level l: -1/2 q~^T (dK/d eps_ab) q~ for the six
 * components, computed as -1/2 sum_d dK_d C_d with the autocorrelation
 * C_d = sum_m q~_m q~_(m-d) (the same double sum, grouped by offset). */
void or_grid_virial_level(const or_plan* P, int l, const double* qg, double W6[6]) {
  int klo[3], ksz[3];
  or_stencil_box(P, l, klo, ksz);
  size_t nK = (size_t)ksz[0] * ksz[1] * ksz[2];
  double* dK = (double*)malloc(sizeof(double) * nK * 6);
  for (int c = 0; c < 6; c++) or_stencil_build(P, l, c + 1, NULL, dK + c * nK);
  double* Cd = (double*)malloc(sizeof(double) * nK);
  int* nn = (int*)P->n[l - 1];
  int* lo = (int*)P->lo[l - 1];
#pragma omp parallel for schedule(dynamic, 16)
  for (long k = 0; k < (long)nK; k++) {
    int any = 0;
    for (int c = 0; c < 6; c++) if (dK[c * nK + k] != 0.0) any = 1;
    if (!any) { Cd[k] = 0.0; continue; }
    int d[3] = {(int)(k / (ksz[1] * ksz[2])) + klo[0], (int)((k / ksz[2]) % ksz[1]) + klo[1],
                (int)(k % ksz[2]) + klo[2]};
    double acc = 0.0;
    for (int ix = 0; ix < nn[0]; ix++) {
      int sx = gidx(P, l, 0, ix + lo[0] - d[0]);
      if (sx < 0) continue;
      for (int iy = 0; iy < nn[1]; iy++) {
        int sy = gidx(P, l, 1, iy + lo[1] - d[1]);
        if (sy < 0) continue;
        for (int iz = 0; iz < nn[2]; iz++) {
          int sz2 = gidx(P, l, 2, iz + lo[2] - d[2]);
          if (sz2 < 0) continue;
          acc += qg[((size_t)ix * nn[1] + iy) * nn[2] + iz] * qg[((size_t)sx * nn[1] + sy) * nn[2] + sz2];
        }
      }
    }
    Cd[k] = acc;
  }
  for (int c = 0; c < 6; c++) {
    double acc = 0.0;
    for (size_t k = 0; k < nK; k++) acc += dK[c * nK + k] * Cd[k];
    W6[c] = -0.5 * acc;
  }
  free(dK);
  free(Cd);
}

/* ------------------------------------------------------------------------ */
/* Short-range part, Eq. U_zero.                                             */
/* ------------------------------------------------------------------------ */

/* phi0_i = sum over (j, image n) != (i, 0) with |d| < a of q_j k_0(|d|),
 * d = r_j + A n - r_i, minus the self term q_i gamma(0)/a (the sum over l >= 1
 * of k_l(0), which telescopes). Every periodic image within the cutoff counts,
 * self images included. F0_i = sum q_i q_j k_0'(|d|) d/|d|;
 * W0 = -1/2 sum_i sum_(j,n) q_i q_j k_0'(|d|) d d^T / |d| (row-major 3x3).
 * E0 = 1/2 sum_i q_i phi0_i. Candidates come from a cell list with cells of
 * edge >= a. F0, W0 may be NULL. */
/* or_short_range for a general (tilted, periodic) cell: the same sums over a
 * cell list in fractional coordinates s = A^-T r; a point within a of r_i has
 * |s_d - s_i,d| <= a / w_d (w_d the distance between the cell faces across d),
 * which bounds the cells visited; displacements d = A^T (s_j + k - s_i). */
static void short_range_tri(const or_plan* P, int n, const double* pos, const double* q, double* phi0, double* F0,
                            double* W0) {
  int p = P->p;
  double a = P->a;
  int C[3];
  for (int d = 0; d < 3; d++) {
    C[d] = (int)floor(P->wplane[d] / a);
    if (C[d] < 1) C[d] = 1;
    if (C[d] > 512) C[d] = 512;
  }
  double* sf = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
  for (int i = 0; i < n; i++)
    for (int d = 0; d < 3; d++) {
      const double* r = pos + 3 * i;
      double sd = P->Tinv[3 * d] * r[0] + P->Tinv[3 * d + 1] * r[1] + P->Tinv[3 * d + 2] * r[2];
      sd -= floor(sd);
      if (sd >= 1.0) sd -= 1.0;
      sf[3 * i + d] = sd;
    }
  int ncell = C[0] * C[1] * C[2];
  int* head = (int*)calloc((size_t)ncell + 1, sizeof(int));
  int* list = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  int* cid = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  for (int i = 0; i < n; i++) {
    int c[3];
    for (int d = 0; d < 3; d++) {
      int ci = (int)floor(sf[3 * i + d] * C[d]);
      c[d] = ci < 0 ? 0 : (ci > C[d] - 1 ? C[d] - 1 : ci);
    }
    cid[i] = (c[0] * C[1] + c[1]) * C[2] + c[2];
    head[cid[i] + 1]++;
  }
  for (int c = 0; c < ncell; c++) head[c + 1] += head[c];
  {
    int* cur = (int*)malloc(sizeof(int) * (ncell > 0 ? ncell : 1));
    for (int c = 0; c < ncell; c++) cur[c] = head[c];
    for (int i = 0; i < n; i++) list[cur[cid[i]]++] = i;
    free(cur);
  }
  double self = or_gamma(p, 0.0) / a;
  double* Wi = W0 ? (double*)malloc(sizeof(double) * 9 * (n > 0 ? n : 1)) : NULL;
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < n; i++) {
    const double* si = sf + 3 * i;
    int clo[3], chi[3];
    for (int d = 0; d < 3; d++) {
      double reach = a / P->wplane[d];
      clo[d] = (int)floor((si[d] - reach) * C[d]);
      chi[d] = (int)floor((si[d] + reach) * C[d]);
    }
    double ph = 0.0, f[3] = {0, 0, 0}, wv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int ux = clo[0]; ux <= chi[0]; ux++)
      for (int uy = clo[1]; uy <= chi[1]; uy++)
        for (int uz = clo[2]; uz <= chi[2]; uz++) {
          int u[3] = {ux, uy, uz}, cw[3], k[3];
          int zero_shift = 1;
          for (int d = 0; d < 3; d++) {
            k[d] = floordiv(u[d], C[d]);
            cw[d] = u[d] - k[d] * C[d];
            if (k[d] != 0) zero_shift = 0;
          }
          int c = (cw[0] * C[1] + cw[1]) * C[2] + cw[2];
          for (int t = head[c]; t < head[c + 1]; t++) {
            int j = list[t];
            if (j == i && zero_shift) continue;
            double ds[3], d[3];
            for (int e = 0; e < 3; e++) ds[e] = sf[3 * j + e] + k[e] - si[e];
            for (int c2 = 0; c2 < 3; c2++) d[c2] = ds[0] * P->A[c2] + ds[1] * P->A[3 + c2] + ds[2] * P->A[6 + c2];
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= a * a) continue;
            double r = sqrt(r2);
            ph += q[j] * or_kl(p, a, P->nlev, 0, r);
            double dk = or_dkl(p, a, P->nlev, 0, r);
            for (int dd = 0; dd < 3; dd++) f[dd] += q[i] * q[j] * dk * d[dd] / r;
            if (Wi)
              for (int aa = 0; aa < 3; aa++)
                for (int bb = 0; bb < 3; bb++) wv[3 * aa + bb] += -0.5 * q[i] * q[j] * dk * d[aa] * d[bb] / r;
          }
        }
    phi0[i] = ph - q[i] * self;
    if (F0)
      for (int dd = 0; dd < 3; dd++) F0[3 * i + dd] = f[dd];
    if (Wi)
      for (int k2 = 0; k2 < 9; k2++) Wi[9 * i + k2] = wv[k2];
  }
  if (W0) {
    for (int k2 = 0; k2 < 9; k2++) {
      double acc = 0.0;
      for (int i = 0; i < n; i++) acc += Wi[9 * i + k2];
      W0[k2] = acc;
    }
    free(Wi);
  }
  free(sf);
  free(head);
  free(list);
  free(cid);
}

void or_short_range(const or_plan* P, int n, const double* pos, const double* q, double* phi0, double* F0,
                    double* W0) {
  if (P->tri) {
    short_range_tri(P, n, pos, q, phi0, F0, W0);
    return;
  }
  int p = P->p;
  double a = P->a;
  int C[3];
  double e[3];
  double* w = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
  for (int d = 0; d < 3; d++) {
    C[d] = (int)floor(P->L[d] / a);
    if (C[d] < 1) C[d] = 1;
    if (C[d] > 512) C[d] = 512;
    e[d] = P->L[d] / C[d];
  }
  for (int i = 0; i < n; i++)
    for (int d = 0; d < 3; d++) {
      double x = pos[3 * i + d];
      if (P->pbc[d]) {
        x = x - P->L[d] * floor(x / P->L[d]);
        if (x >= P->L[d]) x -= P->L[d];
      }
      w[3 * i + d] = x;
    }
  int ncell = C[0] * C[1] * C[2];
  int* head = (int*)malloc(sizeof(int) * (ncell + 1));
  int* list = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  int* cid = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  for (int c = 0; c <= ncell; c++) head[c] = 0;
  for (int i = 0; i < n; i++) {
    int c[3];
    for (int d = 0; d < 3; d++) {
      int ci = (int)floor(w[3 * i + d] / e[d]);
      if (ci < 0) ci = 0;
      if (ci > C[d] - 1) ci = C[d] - 1;
      c[d] = ci;
    }
    cid[i] = (c[0] * C[1] + c[1]) * C[2] + c[2];
    head[cid[i] + 1]++;
  }
  for (int c = 0; c < ncell; c++) head[c + 1] += head[c];
  {
    int* cur = (int*)malloc(sizeof(int) * (ncell > 0 ? ncell : 1));
    for (int c = 0; c < ncell; c++) cur[c] = head[c];
    for (int i = 0; i < n; i++) list[cur[cid[i]]++] = i;
    free(cur);
  }
  double self = or_gamma(p, 0.0) / a;
  double* Wi = W0 ? (double*)malloc(sizeof(double) * 9 * (n > 0 ? n : 1)) : NULL;
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < n; i++) {
    double xi[3] = {w[3 * i], w[3 * i + 1], w[3 * i + 2]};
    int clo[3], chi[3];
    for (int d = 0; d < 3; d++) {
      clo[d] = (int)floor((xi[d] - a) / e[d]);
      chi[d] = (int)floor((xi[d] + a) / e[d]);
      if (!P->pbc[d]) {
        if (clo[d] < 0) clo[d] = 0;
        if (chi[d] > C[d] - 1) chi[d] = C[d] - 1;
      }
    }
    double ph = 0.0, f[3] = {0, 0, 0}, wv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int ux = clo[0]; ux <= chi[0]; ux++)
      for (int uy = clo[1]; uy <= chi[1]; uy++)
        for (int uz = clo[2]; uz <= chi[2]; uz++) {
          int u[3] = {ux, uy, uz}, cw[3];
          double sh[3];
          int zero_shift = 1;
          for (int d = 0; d < 3; d++) {
            int k = floordiv(u[d], C[d]);
            cw[d] = u[d] - k * C[d];
            sh[d] = k * P->L[d];
            if (k != 0) zero_shift = 0;
          }
          int c = (cw[0] * C[1] + cw[1]) * C[2] + cw[2];
          for (int t = head[c]; t < head[c + 1]; t++) {
            int j = list[t];
            if (j == i && zero_shift) continue;
            double d[3];
            for (int dd = 0; dd < 3; dd++) d[dd] = w[3 * j + dd] + sh[dd] - xi[dd];
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= a * a) continue;
            double r = sqrt(r2);
            ph += q[j] * or_kl(p, a, P->nlev, 0, r);
            double dk = or_dkl(p, a, P->nlev, 0, r);
            for (int dd = 0; dd < 3; dd++) f[dd] += q[i] * q[j] * dk * d[dd] / r;
            if (Wi)
              for (int aa = 0; aa < 3; aa++)
                for (int bb = 0; bb < 3; bb++) wv[3 * aa + bb] += -0.5 * q[i] * q[j] * dk * d[aa] * d[bb] / r;
          }
        }
    phi0[i] = ph - q[i] * self;
    if (F0)
      for (int dd = 0; dd < 3; dd++) F0[3 * i + dd] = f[dd];
    if (Wi)
      for (int k = 0; k < 9; k++) Wi[9 * i + k] = wv[k];
  }
  if (W0) {
    for (int k = 0; k < 9; k++) {
      double acc = 0.0;
      for (int i = 0; i < n; i++) acc += Wi[9 * i + k];
      W0[k] = acc;
    }
    free(Wi);
  }
  free(w);
  free(head);
  free(list);
  free(cid);
}

/* Kahan sum of 1/2 sum_i q_i phi_i. */
double or_energy(int n, const double* q, const double* phi) {
  double s = 0.0, c = 0.0;
  for (int i = 0; i < n; i++) {
    double y = 0.5 * q[i] * phi[i] - c;
    double t = s + y;
    c = (t - s) - y;
    s = t;
  }
  return s;
}

/* ------------------------------------------------------------------------ */
/* Whole method: Sec. 2 / Eq. u_oneplus_nested_eval and the derivatives of   */
/* Sec. 3.2.2.                                                               */
/* ------------------------------------------------------------------------ */

/* Grid pass: q~^1 -> restrictions -> e^l = K^l q~^l on every evaluated level
 * -> prolongation from the top down, e^l += I^T e^(l+1). qlev / elev hold the
 * grids of all evaluated levels back to back (level 1 first). */
void or_grid_pass(const or_plan* P, double* qlev, double* elev) {
  size_t off[OR_MAXLEV + 1];
  off[0] = 0;
  for (int l = 1; l <= P->ncomp; l++) off[l] = off[l - 1] + (size_t)lev_size(P, l);
  for (int l = 1; l < P->ncomp; l++) or_restrict(P, l, qlev + off[l - 1], qlev + off[l]);
  for (int l = 1; l <= P->ncomp; l++) {
    int klo[3], ksz[3];
    or_stencil_box(P, l, klo, ksz);
    size_t nK = (size_t)ksz[0] * ksz[1] * ksz[2];
    double* K = (double*)malloc(sizeof(double) * nK);
    or_stencil_build(P, l, 0, NULL, K);
    or_stencil_apply(P, l, K, qlev + off[l - 1], elev + off[l - 1]);
    free(K);
  }
  for (int l = P->ncomp - 1; l >= 1; l--) or_prolong_add(P, l, elev + off[l], elev + off[l - 1]);
}

size_t or_grid_total(const or_plan* P) {
  size_t s = 0;
  for (int l = 1; l <= P->ncomp; l++) s += (size_t)lev_size(P, l);
  return s;
}

/* Full evaluation. Outputs (any may be NULL except E): phi (n), F (n x 3),
 * W (3x3), and the level grids qlev / elev (or_grid_total doubles each). */
void or_msm(const or_plan* P, int n, const double* pos, const double* q, double* E, double* phi, double* F,
            double* W, double* qlev_out, double* elev_out) {
  size_t tot = or_grid_total(P);
  double* qlev = qlev_out ? qlev_out : (double*)malloc(sizeof(double) * (tot > 0 ? tot : 1));
  double* elev = elev_out ? elev_out : (double*)malloc(sizeof(double) * (tot > 0 ? tot : 1));
  double* phi0 = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double* phi1 = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double* F0 = (F || W) ? (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1)) : NULL;
  double* F1 = F ? (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1)) : NULL;
  double W0[9];
  or_short_range(P, n, pos, q, phi0, F0, W ? W0 : NULL);
  if (P->ncomp >= 1) {
    or_anterp(P, n, pos, q, qlev);
    or_grid_pass(P, qlev, elev);
    or_interp(P, n, pos, q, elev, phi1, F1);
  } else {
    for (int i = 0; i < n; i++) phi1[i] = 0.0;
    if (F1) for (int i = 0; i < 3 * n; i++) F1[i] = 0.0;
  }
  double* ph = phi ? phi : (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  for (int i = 0; i < n; i++) ph[i] = phi0[i] + phi1[i];
  *E = or_energy(n, q, ph);
  if (F)
    for (int i = 0; i < 3 * n; i++) F[i] = F0[i] + F1[i];
  if (W) {
    double Wg[6] = {0, 0, 0, 0, 0, 0};
    size_t off = 0;
    for (int l = 1; l <= P->ncomp; l++) {
      double w6[6];
      or_grid_virial_level(P, l, qlev + off, w6);
      for (int c = 0; c < 6; c++) Wg[c] += w6[c];
      off += (size_t)lev_size(P, l);
    }
    int map[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
    for (int k = 0; k < 9; k++) W[k] = W0[k] + Wg[map[k]];
  }
  if (!phi) free(ph);
  if (!qlev_out) free(qlev);
  if (!elev_out) free(elev);
  free(phi0);
  free(phi1);
  free(F0);
  free(F1);
}

/* ------------------------------------------------------------------------ */
/* Exact sums used as pins (not the method).                                */
/* ------------------------------------------------------------------------ */

/* Direct open-boundary Coulomb sum, Eq. generic_pair_potential_sum with k = 1/r:
 * phi_i = sum_(j != i) q_j / r_ij, F_i = q_i sum_j q_j (r_i - r_j)/r^3,
 * E = 1/2 sum q_i phi_i. */
void or_direct_open(int n, const double* pos, const double* q, double* E, double* phi, double* F) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; i++) {
    double ph = 0.0, f[3] = {0, 0, 0};
    for (int j = 0; j < n; j++) {
      if (j == i) continue;
      double d[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1], pos[3 * i + 2] - pos[3 * j + 2]};
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      ph += q[j] / r;
      for (int k = 0; k < 3; k++) f[k] += q[i] * q[j] * d[k] / (r * r * r);
    }
    phi[i] = ph;
    if (F)
      for (int k = 0; k < 3; k++) F[3 * i + k] = f[k];
  }
  *E = or_energy(n, q, phi);
}

/* Direct sum of one smooth kernel over all ordered pairs including i == j
 * (open boundaries): phi_i = sum_j q_j k_l(r_ij) for level l of a plan with
 * nlev levels. Used to pin the grid part level by level. */
void or_direct_level(int p, double a, int nlev, int l, int n, const double* pos, const double* q, double* E,
                     double* phi) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; i++) {
    double ph = 0.0;
    for (int j = 0; j < n; j++) {
      double d[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1], pos[3 * i + 2] - pos[3 * j + 2]};
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      ph += q[j] * or_kl(p, a, nlev, l, r);
    }
    phi[i] = ph;
  }
  *E = or_energy(n, q, phi);
}

/* Ewald sum for an orthorhombic periodic cell with tin-foil boundary
 * conditions (textbook form): real-space erfc(alpha r)/r over all images with
 * r < rcut, reciprocal sum over |k| <= kmax of (4 pi / V) exp(-k^2/4alpha^2)/k^2,
 * self term -2 alpha/sqrt(pi) q_i. phi, F per atom; E = 1/2 sum q phi. */
void or_ewald(const double* L, int n, const double* pos, const double* q, double alpha, double rcut,
              double kmax, double* E, double* phi, double* F) {
  double V = L[0] * L[1] * L[2];
  int im[3];
  for (int d = 0; d < 3; d++) im[d] = (int)ceil(rcut / L[d]) + 1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; i++) {
    double ph = 0.0, f[3] = {0, 0, 0};
    for (int j = 0; j < n; j++) {
      double d0[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1], pos[3 * j + 2] - pos[3 * i + 2]};
      for (int d = 0; d < 3; d++) d0[d] -= L[d] * floor(d0[d] / L[d] + 0.5);
      for (int nx = -im[0]; nx <= im[0]; nx++)
        for (int ny = -im[1]; ny <= im[1]; ny++)
          for (int nz = -im[2]; nz <= im[2]; nz++) {
            if (j == i && nx == 0 && ny == 0 && nz == 0) continue;
            double d[3] = {d0[0] + nx * L[0], d0[1] + ny * L[1], d0[2] + nz * L[2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= rcut * rcut) continue;
            double r = sqrt(r2);
            double er = erfc(alpha * r);
            ph += q[j] * er / r;
            double dpot = -er / r2 - 2.0 * alpha / sqrt(M_PI) * exp(-alpha * alpha * r2) / r; /* d/dr erfc(ar)/r */
            for (int k = 0; k < 3; k++) f[k] += q[i] * q[j] * dpot * d[k] / r;
          }
    }
    phi[i] = ph - 2.0 * alpha / sqrt(M_PI) * q[i];
    if (F)
      for (int k = 0; k < 3; k++) F[3 * i + k] = f[k];
  }
  /* reciprocal space: k = 2 pi (mx/Lx, my/Ly, mz/Lz) */
  int mm[3];
  for (int d = 0; d < 3; d++) mm[d] = (int)floor(kmax * L[d] / (2.0 * M_PI));
  double* ph_r = (double*)calloc((size_t)n, sizeof(double));
  double* f_r = (double*)calloc((size_t)3 * n, sizeof(double));
  long nkx = 2L * mm[0] + 1, nky = 2L * mm[1] + 1, nkz = 2L * mm[2] + 1;
  long nk = nkx * nky * nkz;
  /* per-k loop with per-atom work; the per-atom accumulations are done
   * afterwards in fixed k order to stay deterministic */
  double* Sre = (double*)malloc(sizeof(double) * nk);
  double* Sim = (double*)malloc(sizeof(double) * nk);
  double* Ak = (double*)malloc(sizeof(double) * nk);
#pragma omp parallel for schedule(dynamic, 8)
  for (long t = 0; t < nk; t++) {
    int mx = (int)(t / (nky * nkz)) - mm[0], my = (int)((t / nkz) % nky) - mm[1], mz = (int)(t % nkz) - mm[2];
    double k[3] = {2 * M_PI * mx / L[0], 2 * M_PI * my / L[1], 2 * M_PI * mz / L[2]};
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    if ((mx == 0 && my == 0 && mz == 0) || k2 > kmax * kmax) {
      Ak[t] = 0.0;
      Sre[t] = Sim[t] = 0.0;
      continue;
    }
    Ak[t] = 4.0 * M_PI / V * exp(-k2 / (4.0 * alpha * alpha)) / k2;
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < n; j++) {
      double kr = k[0] * pos[3 * j] + k[1] * pos[3 * j + 1] + k[2] * pos[3 * j + 2];
      sr += q[j] * cos(kr);
      si += q[j] * sin(kr);
    }
    Sre[t] = sr;
    Sim[t] = si;
  }
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; i++) {
    double ph = 0.0, f[3] = {0, 0, 0};
    for (long t = 0; t < nk; t++) {
      if (Ak[t] == 0.0) continue;
      int mx = (int)(t / (nky * nkz)) - mm[0], my = (int)((t / nkz) % nky) - mm[1], mz = (int)(t % nkz) - mm[2];
      double k[3] = {2 * M_PI * mx / L[0], 2 * M_PI * my / L[1], 2 * M_PI * mz / L[2]};
      double kr = k[0] * pos[3 * i] + k[1] * pos[3 * i + 1] + k[2] * pos[3 * i + 2];
      double c = cos(kr), s = sin(kr);
      /* Re(S(k) e^{-ik r_i}) and Im(S*(k) e^{ik r_i}) */
      double re = Sre[t] * c + Sim[t] * s;
      double imv = Sre[t] * s - Sim[t] * c;
      ph += Ak[t] * re;
      for (int d = 0; d < 3; d++) f[d] += Ak[t] * q[i] * k[d] * imv;
    }
    ph_r[i] = ph;
    for (int d = 0; d < 3; d++) f_r[3 * i + d] = f[d];
  }
  for (int i = 0; i < n; i++) {
    phi[i] += ph_r[i];
    if (F)
      for (int d = 0; d < 3; d++) F[3 * i + d] += f_r[3 * i + d];
  }
  *E = or_energy(n, q, phi);
  free(ph_r);
  free(f_r);
  free(Sre);
  free(Sim);
  free(Ak);
}

/* Ewald sum for a general periodic cell (rows a, b, c of A; tin-foil): real
 * space over lattice vectors A^T n with |r_ij + A^T n| < rcut, reciprocal
 * space over k = 2 pi sum_j m_j b_j (b_j the columns of A^-1, a_i . b_j =
 * delta_ij) with |k| <= kmax, self term -2 alpha/sqrt(pi) q_i; E = 1/2 sum q phi. */
void or_ewald_tri(const double* A, int n, const double* pos, const double* q, double alpha, double rcut, double kmax,
                  double* E, double* phi) {
  double Ai[9], det;
  mat_inv3(A, Ai, &det);
  double V = det, w[3];
  for (int d = 0; d < 3; d++) {
    const double* u = A + 3 * ((d + 1) % 3);
    const double* v = A + 3 * ((d + 2) % 3);
    double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
    w[d] = det / sqrt(cx * cx + cy * cy + cz * cz);
  }
  int im[3];
  for (int d = 0; d < 3; d++) im[d] = (int)ceil(rcut / w[d]) + 1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; i++) {
    double ph = 0.0;
    for (int j = 0; j < n; j++) {
      double ds[3];
      for (int d = 0; d < 3; d++) {
        double rd[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1], pos[3 * j + 2] - pos[3 * i + 2]};
        ds[d] = Ai[d] * rd[0] + Ai[3 + d] * rd[1] + Ai[6 + d] * rd[2];  /* (A^-T r)_d */
        ds[d] -= floor(ds[d] + 0.5);
      }
      for (int nx = -im[0]; nx <= im[0]; nx++)
        for (int ny = -im[1]; ny <= im[1]; ny++)
          for (int nz = -im[2]; nz <= im[2]; nz++) {
            if (j == i && nx == 0 && ny == 0 && nz == 0) continue;
            double f[3] = {ds[0] + nx, ds[1] + ny, ds[2] + nz}, d[3];
            for (int c = 0; c < 3; c++) d[c] = f[0] * A[c] + f[1] * A[3 + c] + f[2] * A[6 + c];
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= rcut * rcut) continue;
            double r = sqrt(r2);
            ph += q[j] * erfc(alpha * r) / r;
          }
    }
    phi[i] = ph - 2.0 * alpha / sqrt(OR_PI) * q[i];
  }
  int mm[3];
  for (int d = 0; d < 3; d++) {
    double la = sqrt(A[3 * d] * A[3 * d] + A[3 * d + 1] * A[3 * d + 1] + A[3 * d + 2] * A[3 * d + 2]);
    mm[d] = (int)floor(kmax * la / (2.0 * OR_PI)) + 1;
  }
  long nkx = 2L * mm[0] + 1, nky = 2L * mm[1] + 1, nkz = 2L * mm[2] + 1, nk = nkx * nky * nkz;
  double* Ak = (double*)malloc(sizeof(double) * nk);
  double* Sre = (double*)malloc(sizeof(double) * nk);
  double* Sim = (double*)malloc(sizeof(double) * nk);
  double (*kv)[3] = (double (*)[3])malloc(sizeof(double) * 3 * nk);
#pragma omp parallel for schedule(dynamic, 8)
  for (long t = 0; t < nk; t++) {
    int m[3] = {(int)(t / (nky * nkz)) - mm[0], (int)((t / nkz) % nky) - mm[1], (int)(t % nkz) - mm[2]};
    double k[3];
    for (int c = 0; c < 3; c++) k[c] = 2.0 * OR_PI * (m[0] * Ai[3 * c] + m[1] * Ai[3 * c + 1] + m[2] * Ai[3 * c + 2]);
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    for (int c = 0; c < 3; c++) kv[t][c] = k[c];
    if ((m[0] == 0 && m[1] == 0 && m[2] == 0) || k2 > kmax * kmax) {
      Ak[t] = 0.0;
      Sre[t] = Sim[t] = 0.0;
      continue;
    }
    Ak[t] = 4.0 * OR_PI / V * exp(-k2 / (4.0 * alpha * alpha)) / k2;
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < n; j++) {
      double kr = k[0] * pos[3 * j] + k[1] * pos[3 * j + 1] + k[2] * pos[3 * j + 2];
      sr += q[j] * cos(kr);
      si += q[j] * sin(kr);
    }
    Sre[t] = sr;
    Sim[t] = si;
  }
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; i++) {
    double ph = 0.0;
    for (long t = 0; t < nk; t++) {
      if (Ak[t] == 0.0) continue;
      double kr = kv[t][0] * pos[3 * i] + kv[t][1] * pos[3 * i + 1] + kv[t][2] * pos[3 * i + 2];
      ph += Ak[t] * (Sre[t] * cos(kr) + Sim[t] * sin(kr));
    }
    phi[i] += ph;
  }
  double e = 0.0;
  for (int i = 0; i < n; i++) e += 0.5 * q[i] * phi[i];
  *E = e;
  free(Ak);
  free(Sre);
  free(Sim);
  free(kv);
}
