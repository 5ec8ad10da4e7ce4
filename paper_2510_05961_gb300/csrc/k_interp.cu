// k_interp.cu -- particle <-> grid operations of the MSM (Sec. 3.2.2):
// anterpolation q~^1_m = sum_i q_i phi^1_m(r_i) (Eq. grid_charge,
// Alg. anterpolation_double_loop) and interpolation
// phi^(1+)_i = sum_m e^(1+)_m phi^1_m(r_i) with the position gradient
// q_i sum_m e^(1+)_m grad phi^1_m(r_i) (Eqs. uoneplus_interpolation_with_index_set,
// analytic_uoneplus_position_grad). The basis is the tensor product of
// centred cardinal B-splines of order p (Sec. 3.3), evaluated in FP32 by the
// uniform Cox-de Boor recursion on the fractional grid coordinate.
//
// Anterpolation reads the cell-sorted atoms, one warp per binning column: the
// column's partial sums over the grid points its atoms reach, then one sum per
// grid point (k_anterp_cols, k_anterp_sum); the gather by grid columns
// (k_anterp) serves dipole charges and footprints too wide for those. No
// atomics; the result is the same on every run.
#include "msm_internal.h"

namespace msm {

__host__ __device__ __forceinline__ int floordiv_i(int a, int b) {
  int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}
__device__ __forceinline__ int wrap_i(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// Weights w[j] = Phi_P(f + P/2 - 1 - j) of the grid points base + j,
// base = floor(u) - P/2 + 1, f = u - floor(u), and their u-derivatives.
// Cardinal B-spline N_m on [0, m): N_m(x) = (x N_(m-1)(x) + (m - x) N_(m-1)(x-1)) / (m-1),
// N_P'(x) = N_(P-1)(x) - N_(P-1)(x-1); Phi_P(t) = N_P(t + P/2).
template <int P, bool DERIV>
__device__ __forceinline__ void bspline_weights(float f, float (&w)[P], float (&dw)[P]) {
  float c[P];
#pragma unroll
  for (int k = 0; k < P; k++) c[k] = (k == 0) ? 1.0f : 0.0f;
  float cp[P];
#pragma unroll
  for (int m = 2; m <= P; m++) {
    if (DERIV && m == P) {
#pragma unroll
      for (int k = 0; k < P; k++) cp[k] = c[k];
    }
    const float inv = 1.0f / (float)(m - 1);
#pragma unroll
    for (int k = m - 1; k >= 0; k--) {
      float lower = (k > 0) ? c[k - 1] : 0.0f;
      c[k] = ((f + (float)k) * c[k] + ((float)(m - k) - f) * lower) * inv;
    }
  }
#pragma unroll
  for (int j = 0; j < P; j++) {
    w[j] = c[P - 1 - j];
    if (DERIV) {
      float hi = (P - 1 - j <= P - 2) ? cp[P - 1 - j] : 0.0f;
      float lo = (P - 2 - j >= 0) ? cp[P - 2 - j] : 0.0f;
      dw[j] = hi - lo;
    }
  }
}

// Weights, u-derivatives and second u-derivatives of the P grid points of
// one axis: N_P'' (x) = N_(P-2)(x) - 2 N_(P-2)(x-1) + N_(P-2)(x-2).
template <int P>
__device__ __forceinline__ void bspline_weights2(float f, float (&w)[P], float (&dw)[P], float (&d2w)[P]) {
  float c[P], cp[P], cpp[P];
#pragma unroll
  for (int k = 0; k < P; k++) c[k] = (k == 0) ? 1.0f : 0.0f;
#pragma unroll
  for (int m = 2; m <= P; m++) {
    if (m == P - 1) {
#pragma unroll
      for (int k = 0; k < P; k++) cpp[k] = c[k];  // N_(P-2)(f + k)
    }
    if (m == P) {
#pragma unroll
      for (int k = 0; k < P; k++) cp[k] = c[k];   // N_(P-1)(f + k)
    }
    const float inv = 1.0f / (float)(m - 1);
#pragma unroll
    for (int k = m - 1; k >= 0; k--) {
      float lower = (k > 0) ? c[k - 1] : 0.0f;
      c[k] = ((f + (float)k) * c[k] + ((float)(m - k) - f) * lower) * inv;
    }
  }
  auto at2 = [&](int k) { return (k >= 0 && k <= P - 3) ? cpp[k] : 0.0f; };
#pragma unroll
  for (int j = 0; j < P; j++) {
    w[j] = c[P - 1 - j];
    float hi = (P - 1 - j <= P - 2) ? cp[P - 1 - j] : 0.0f;
    float lo = (P - 2 - j >= 0) ? cp[P - 2 - j] : 0.0f;
    dw[j] = hi - lo;
    d2w[j] = at2(P - 1 - j) - 2.0f * at2(P - 2 - j) + at2(P - 3 - j);
  }
}

// Centred B-spline Phi_P(t): zero for |t| >= P/2; on |t| in [i, i+1) the
// polynomial S.bsp[i][.] (ascending powers) of the local variable |t| - i.
template <int P>
__device__ __forceinline__ float bspline_value(float t, const float (&cf)[P / 2][P]) {
  const float a = fabsf(t);
  const int i = (int)a;
  float w = 0.f;
#pragma unroll
  for (int piece = 0; piece < P / 2; piece++) {
    const float s = a - (float)piece;
    float v = cf[piece][P - 1];
#pragma unroll
    for (int k = P - 2; k >= 0; k--) v = fmaf(v, s, cf[piece][k]);
    w = (i == piece) ? v : w;
  }
  return w;
}

// Phi_P(t) and its derivative Phi_P'(t) (odd) from the same pieces.
template <int P>
__device__ __forceinline__ void bspline_value_d(float t, const float (&cf)[P / 2][P], float& v, float& dv) {
  const float a = fabsf(t);
  const int i = (int)a;
  v = 0.f;
  dv = 0.f;
#pragma unroll
  for (int piece = 0; piece < P / 2; piece++) {
    const float s = a - (float)piece;
    float pv = cf[piece][P - 1], pd = (float)(P - 1) * cf[piece][P - 1];
#pragma unroll
    for (int k = P - 2; k >= 0; k--) {
      pv = fmaf(pv, s, cf[piece][k]);
      if (k >= 1) pd = fmaf(pd, s, (float)k * cf[piece][k]);
    }
    v = (i == piece) ? pv : v;
    dv = (i == piece) ? pd : dv;
  }
  dv = t < 0.f ? -dv : dv;
}

// Anterpolation by grid columns. A block owns a tile of 16 x 8 grid columns
// (x, y) and TZ points along z (16, 32 or 64, chosen by the autotuner); each thread owns one column and sums,
// over the atoms of the cells whose B-spline support reaches that column,
// q_i Phi(m_x - u_x) Phi(m_y - u_y) times the p weights of the atom's z-base
// into a private z-array in shared memory (u: atom position in level-1 grid
// units, shifted by the period for cells visited across a periodic
// boundary). Warp w holds the columns of one parity class (x mod 2, y mod 2),
// so its lanes visit the same number of cell columns; each lane keeps four
// atom loads in flight. No atomics, no block barriers; every column sums its
// atoms in a fixed order.
constexpr int kAntNT = kAnterpTX * kAnterpTY;
static_assert(kAnterpTX == 16 && kAnterpTY == 8, "one parity class of 8 x 4 columns per warp");

//
// DIP: the same gather for point dipoles p_i = q_i u_i (us holds (u_i, q_i)
// sorted): the grid charge of a dipole is p_i . grad Phi_m(r_i), i.e. per
// column A w_z + B dw_z with A = p_x Phi_x' Phi_y / h_x + p_y Phi_x Phi_y' / h_y
// and B = p_z Phi_x Phi_y / h_z (the force vector-Jacobian product).
template <int P, int TZ, bool DIP = false>
__global__ void __launch_bounds__(kAntNT, 8) k_anterp(const SysDev* __restrict__ sys, const LevDev* __restrict__ levs,
                                                  const TileItem* __restrict__ items,
                                                  const int* __restrict__ cell_start,
                                                  const float4* __restrict__ uq, float* __restrict__ grid,
                                                  const float4* __restrict__ us = nullptr) {
  constexpr int H = P / 2;
  constexpr int PAD = P - 1;
  constexpr int NZ = TZ + 2 * PAD;
  __shared__ float col[NZ][kAntNT];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = levs[it.lev];
  const SysDev& S = sys[L.sys];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int gx = it.x0 + 2 * (lane & 7) + (warp & 1), gy = it.y0 + 2 * (lane >> 3) + (warp >> 1);
  if (gx >= L.n[0] || gy >= L.n[1]) return;
#pragma unroll
  for (int r = 0; r < NZ; r++) col[r][t] = 0.f;
  float cf[H][P];
#pragma unroll
  for (int i = 0; i < H; i++)
#pragma unroll
    for (int k = 0; k < P; k++) cf[i][k] = S.bsp[i][k];
  const int zlen = min(TZ, L.n[2] - it.z0);
  // grid indices of this column and of the tile's z-range; atom cell ranges
  const int m[3] = {gx + L.lo[0], gy + L.lo[1], it.z0 + L.lo[2]};
  const int mhi[3] = {m[0], m[1], m[2] + zlen - 1};
  int cl[3], ch[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    if (S.pbc[d] && S.M[d] % S.C[d] == 0) {
      // cells aligned with the grid (k intervals per cell): the cell of an
      // atom is floor(u / k) exactly, so the range is exact
      const int k = S.M[d] / S.C[d];
      cl[d] = floordiv_i(m[d] - H, k);
      ch[d] = floordiv_i(mhi[d] + H - 1, k);
    } else {
      // cells not aligned with the grid (open axes): the atoms reaching the
      // points [m, mhi] have u in [m - H, mhi + H), and an atom binned in cell
      // c has u C / M within 1e-4 of [c, c + 1] (s C and s M are FP32 products
      // of one s, and C <= 256 on an open axis); with the rounding of the
      // bounds below, a margin of 2e-4 cells keeps every such atom
      const float rc = (float)S.C[d] / (float)S.M[d];
      cl[d] = (int)floorf((float)(m[d] - H) * rc - 2e-4f);
      ch[d] = (int)floorf((float)(mhi[d] + H) * rc + 2e-4f);
    }
    if (!S.pbc[d]) {
      cl[d] = max(cl[d], 0);
      ch[d] = min(ch[d], S.C[d] - 1);
    }
  }
  const int Cx = S.C[0], Cy = S.C[1], Cz = S.C[2];
  for (int ux = cl[0]; ux <= ch[0]; ux++) {
    const int wx = wrap_i(ux, Cx);
    const float mx = (float)(m[0] - floordiv_i(ux, Cx) * S.M[0]);  // m_x minus the image shift
    for (int uy = cl[1]; uy <= ch[1]; uy++) {
      const int wy = wrap_i(uy, Cy);
      const float my = (float)(m[1] - floordiv_i(uy, Cy) * S.M[1]);
      const int* cs = cell_start + S.cell_off + (wx * Cy + wy) * Cz;
      int uz = cl[2];
      while (uz <= ch[2]) {
        const int kz = floordiv_i(uz, Cz), wz = uz - kz * Cz;
        const int wend = min(Cz - 1, wz + (ch[2] - uz));
        const int zsh = kz * S.M[2] - m[2];  // z-base relative to the tile's first point
        auto add = [&](const float4 u, const float4 pu) {
          const float fl = floorf(u.z);
          const int r = (int)fl + zsh - H + 1;  // first of the p z-points, tile-relative
          if constexpr (!DIP) {
            const float wxy = u.w * bspline_value<P>(mx - u.x, cf) * bspline_value<P>(my - u.y, cf);
            if (wxy != 0.f && r >= -PAD && r < zlen) {
              float wz[P], dummy[P];
              bspline_weights<P, false>(u.z - fl, wz, dummy);
#pragma unroll
              for (int jz = 0; jz < P; jz++) col[r + PAD + jz][t] = fmaf(wxy, wz[jz], col[r + PAD + jz][t]);
            }
          } else {
            float vx, dvx, vy, dvy;
            bspline_value_d<P>(mx - u.x, cf, vx, dvx);  // d/du Phi(u - m) = -Phi'(m - u)
            bspline_value_d<P>(my - u.y, cf, vy, dvy);
            // the dipole in grid units, p_u = J^T p (J = A^-1 diag(M); diag(1/h_1) for a
            // rectangular cell): p . grad_r Phi = p_u . grad_u Phi
            float px = pu.w * pu.x, py = pu.w * pu.y, pz = pu.w * pu.z;
            if (S.tri) {
              const float* J = S.Jg;
              const float ux = J[0] * px + J[3] * py + J[6] * pz, uy = J[1] * px + J[4] * py + J[7] * pz,
                          uz = J[2] * px + J[5] * py + J[8] * pz;
              px = ux;
              py = uy;
              pz = uz;
            } else {
              px *= S.inv_h1[0];
              py *= S.inv_h1[1];
              pz *= S.inv_h1[2];
            }
            const float A = -(px * dvx * vy + py * vx * dvy);
            const float B = pz * vx * vy;
            if ((A != 0.f || B != 0.f) && r >= -PAD && r < zlen) {
              float wz[P], dwz[P];
              bspline_weights<P, true>(u.z - fl, wz, dwz);
#pragma unroll
              for (int jz = 0; jz < P; jz++)
                col[r + PAD + jz][t] = fmaf(A, wz[jz], fmaf(B, dwz[jz], col[r + PAD + jz][t]));
            }
          }
        };
        int je = cs[wend + 1];
        int j = cs[wz];
        if (!MSM_CHECK(S, j >= S.atom_off && je <= S.atom_off + S.n)) je = j;
        const float4 none = make_float4(0.f, 0.f, 0.f, 0.f);
        for (; j + 3 < je; j += 4) {  // four loads in flight
          const float4 u0 = uq[j], u1 = uq[j + 1], u2 = uq[j + 2], u3 = uq[j + 3];
          if constexpr (DIP) {
            const float4 p0 = us[j], p1 = us[j + 1], p2 = us[j + 2], p3 = us[j + 3];
            add(u0, p0);
            add(u1, p1);
            add(u2, p2);
            add(u3, p3);
          } else {
            add(u0, none);
            add(u1, none);
            add(u2, none);
            add(u3, none);
          }
        }
        for (; j < je; j++) add(uq[j], DIP ? us[j] : none);
        uz += wend - wz + 1;
      }
    }
  }
  float* out = grid + L.q_off + ((long long)gx * L.n[1] + gy) * L.n[2] + it.z0;
  for (int z = 0; z < zlen; z++) out[z] = col[z + PAD][t];
}

template <int P>
__global__ void __launch_bounds__(kChunk) k_interp(const SysDev* __restrict__ sys, const LevDev* __restrict__ levs,
                                                   const AtomItem* __restrict__ items, const float4* __restrict__ uq,
                                                   const float* __restrict__ grid, float* __restrict__ phi_lr,
                                                   float4* __restrict__ f_lr, int want_f) {
  constexpr int H = P / 2;
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  int local = it.start + threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  int k = S.atom_off + local;
  if (S.ncomp < 1) {
    phi_lr[k] = 0.0f;
    if (want_f) f_lr[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const LevDev& L = levs[S.lev0];
  float4 u4 = uq[k];
  float uu[3] = {u4.x, u4.y, u4.z};
  float w[3][P], dw[3][P];
  int ix[3][P];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    float fl = floorf(uu[d]);
    int base = (int)fl - H + 1;
    bspline_weights<P, true>(uu[d] - fl, w[d], dw[d]);
#pragma unroll
    for (int j = 0; j < P; j++) {
      int m = base + j;
      ix[d][j] = L.per[d] ? (m & (L.n[d] - 1)) : m - L.lo[d];  // periodic grid counts are powers of two
    }
  }
  const float* e = grid + L.e_off;
#if MSM_CHECKS
  for (int d = 0; d < 3; d++)
    for (int j = 0; j < P; j++)
      if (!MSM_CHECK(S, ix[d][j] >= 0 && ix[d][j] < L.n[d])) ix[d][j] = 0;
#endif
  float ph = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
  for (int jx = 0; jx < P; jx++) {
#pragma unroll
    for (int jy = 0; jy < P; jy++) {
      const float* row = e + ((long long)ix[0][jx] * L.n[1] + ix[1][jy]) * L.n[2];
      float sz = 0.f, dsz = 0.f;
#pragma unroll
      for (int jz = 0; jz < P; jz++) {
        float ev = __ldg(row + ix[2][jz]);
        sz = fmaf(w[2][jz], ev, sz);
        dsz = fmaf(dw[2][jz], ev, dsz);
      }
      float wxy = w[0][jx] * w[1][jy];
      ph = fmaf(wxy, sz, ph);
      gx = fmaf(dw[0][jx] * w[1][jy], sz, gx);
      gy = fmaf(w[0][jx] * dw[1][jy], sz, gy);
      gz = fmaf(wxy, dsz, gz);
    }
  }
  phi_lr[k] = ph;
  // field -grad phi^(1+) at the atom (the force is q_i times it); a tilted cell
  // maps the grid derivatives by A^-1 diag(M)
  if (want_f) {
    if (S.tri) {
      const float* J = S.Jg;
      f_lr[k] = make_float4(-(J[0] * gx + J[1] * gy + J[2] * gz), -(J[3] * gx + J[4] * gy + J[5] * gz),
                            -(J[6] * gx + J[7] * gy + J[8] * gz), 0.f);
    } else {
      f_lr[k] = make_float4(-gx * S.inv_h1[0], -gy * S.inv_h1[1], -gz * S.inv_h1[2], 0.f);
    }
  }
}

// ------------------------------------------- anterpolation by binning columns
// Anterpolation runs from the cell-sorted atoms in two launches, with no
// atomics and a fixed summation order:
//  (1) k_anterp_cols: one warp per (binning column, z-segment of tz level-1
//      points). The warp owns the grid columns its atoms can reach (the
//      column's footprint, afoot[0] x afoot[1]) over the segment, in shared
//      memory, and walks the column's atoms in sorted order: the lanes first
//      evaluate the B-spline weights of 32 atoms at once (q w_x w_y for the
//      p^2 (x, y) pairs, w_z), then the warp adds the p^3 products of one atom
//      at a time, each lane a fixed set of (i, j, k) offsets, so the lanes of
//      one atom write distinct points. The footprint is then written out as
//      the column's partial sums.
//  (2) k_anterp_sum: every level-1 point adds the partial sums of the binning
//      columns whose footprint holds it, in order of the column index.
// Along an axis, the footprint of binning cell c starts at cell_lo(c):
// c k - p/2 + 1 when the cells are aligned with the grid (k = M / C = 2^ashift
// level-1 intervals per cell; an atom of cell c has floor(u) in [ck, ck + k)),
// else floor((c - 2e-4) M / C) - p/2 + 1 (an atom binned in cell c has u C / M
// within 1e-4 of [c, c + 1]); its width afoot is k + p - 1, or
// floor((1 + 4e-4) M / C) + p + 1, set by the planner.
template <int P>
__device__ __forceinline__ int cell_lo(const SysDev& S, int d, int c) {
  constexpr int H = P / 2;
  if (S.ashift[d] >= 0) return (c << S.ashift[d]) - H + 1;
  return (int)floorf(((float)c - 2e-4f) * S.aratio[d]) - H + 1;
}

// shared-memory layout of one warp's footprint: point (fx, fy, z) of the
// segment at fx * xs + fy * zp + z + p - 1, with p - 1 rows of padding on both
// sides of the segment (the parts of an atom's support outside it land there),
// zp >= tz + 2p - 2. For p = 4, lane l adds the products (i, j, k) with
// 4 i + j = l / 2 and k = l % 2 + {0, 2}: zp = 2 mod 16 and xs = 8 mod 32 put
// the 32 lanes' offsets 8 i + zp j + k in 32 distinct banks; other orders use
// zp = 4 mod 16 and xs = 16 mod 32 (their lanes take (ij, k) = divmod(l + 32 r, p))
__host__ __device__ inline int ant_zp(int tz, int p) {
  int zp = tz + 2 * p - 2;
  const int want = p == 4 ? 2 : 4;
  return zp + ((want - zp % 16) + 16) % 16;
}
__host__ __device__ inline int ant_xs(int fy_n, int tz, int p) {
  const int xs = fy_n * ant_zp(tz, p);
  const int want = p == 4 ? 8 : 16;
  return xs + ((want - xs % 32) + 32) % 32;
}
// staging of 32 atoms: q w_x w_y (p^2 + 1 per atom), w_z (p + 1 per atom), base offsets
__host__ __device__ inline int ant_stage_floats(int p) { return 32 * (p * p + 1) + 32 * (p + 1) + 32; }

template <int P>
__global__ void __launch_bounds__(kAntWarps * 32, 4) k_anterp_cols(const SysDev* __restrict__ sys,
                                                                const LevDev* __restrict__ levs,
                                                                const TileItem* __restrict__ items, int nitems,
                                                                int tz, int wstride,
                                                                const int* __restrict__ cell_start,
                                                                const float4* __restrict__ uq,
                                                                float* __restrict__ apart) {
  constexpr int H = P / 2, P3 = P * P * P, R = (P3 + 31) / 32, SQ = P * P + 1, SZ = P + 1;
  extern __shared__ __align__(16) float smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int iw = blockIdx.x * kAntWarps + wib;
  if (iw >= nitems) return;  // whole warps only; no block barriers below
  const TileItem it = items[iw];
  const LevDev& L = levs[it.lev];
  const SysDev& S = sys[L.sys];
  const int Fx = S.afoot[0], Fy = S.afoot[1];
  const int ZP = ant_zp(tz, P), XS = ant_xs(Fy, tz, P);
  float* acc = smem + (size_t)wib * wstride;
  float* sq = acc + ((Fx * XS + 3) & ~3);  // q w_x w_y of 32 atoms
  float* sz = sq + 32 * SQ;                // w_z of 32 atoms
  int* sb = reinterpret_cast<int*>(sz + 32 * SZ);  // base offset of each atom in acc
  for (int e = 4 * lane; e < Fx * XS; e += 128) *reinterpret_cast<float4*>(acc + e) = make_float4(0.f, 0.f, 0.f, 0.f);
  const int cx = it.x0, cy = it.y0, z0 = it.z0;
  const int lox = cell_lo<P>(S, 0, cx), loy = cell_lo<P>(S, 1, cy);
  const int zlen = min(tz, L.n[2] - z0);
  const int mz0 = z0 + L.lo[2];
  // z-cells of the column whose atoms reach the points [mz0, mz0 + zlen)
  int cl, ch;
  if (S.ashift[2] >= 0) {
    cl = (mz0 - H) >> S.ashift[2];
    ch = (mz0 + zlen - 1 + H - 1) >> S.ashift[2];
  } else {
    const float rc = S.ainv[2];
    cl = (int)floorf((float)(mz0 - H) * rc - 2e-4f);
    ch = (int)floorf((float)(mz0 + zlen - 1 + H) * rc + 2e-4f);
  }
  if (!S.pbc[2]) {
    cl = max(cl, 0);
    ch = min(ch, S.C[2] - 1);
  }
  const int Cy = S.C[1], Cz = S.C[2];
  const int* cs = cell_start + S.cell_off + (cx * Cy + cy) * Cz;
  int uz = cl;
  while (uz <= ch) {
    const int kz = floordiv_i(uz, Cz), wz = uz - kz * Cz;
    const int wend = min(Cz - 1, wz + (ch - uz));
    const int zsh = kz * S.M[2] - mz0 - H + 1;  // z base relative to the segment: floor(u_z) + zsh
    int j = cs[wz], je = cs[wend + 1];
    if (!MSM_CHECK(S, j >= S.atom_off && je <= S.atom_off + S.n)) je = j;
    // the next chunk's atoms are loaded while this chunk is added (one memory
    // round trip per run instead of one per chunk)
    float4 un = lane < je - j ? uq[j + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (; j < je; j += 32) {
      const int na = min(32, je - j);
      const float4 u = un;
      if (lane < je - j - 32) un = uq[j + 32 + lane];
      __syncwarp();  // the previous chunk's staging has been read
      if (lane < na) {
        const float flx = floorf(u.x), fly = floorf(u.y), flz = floorf(u.z);
        const int bx = (int)flx - H + 1 - lox, by = (int)fly - H + 1 - loy, bz = (int)flz + zsh;
        float qq = u.w;
        int base = bx * XS + by * ZP + bz + P - 1;
        // every atom of the column lies inside its footprint; one outside is
        // skipped (and reported by the checked build) instead of written; an
        // atom whose support misses the segment adds nothing to it
        if (!(bx >= 0 && bx <= Fx - P && by >= 0 && by <= Fy - P)) {
          (void)MSM_CHECK(S, false);
          qq = 0.f;
          base = 0;
        } else if (bz < 1 - P || bz >= zlen) {
          qq = 0.f;
          base = 0;
        }
        float wx[P], wy[P], w3[P], dummy[P];
        bspline_weights<P, false>(u.x - flx, wx, dummy);
        bspline_weights<P, false>(u.y - fly, wy, dummy);
        bspline_weights<P, false>(u.z - flz, w3, dummy);
#pragma unroll
        for (int i = 0; i < P; i++) {
          const float qx = qq * wx[i];
#pragma unroll
          for (int jj = 0; jj < P; jj++) sq[lane * SQ + i * P + jj] = qx * wy[jj];
        }
        if constexpr (P == 4) {
          // w_z as (w0, w2, w1, w3): a lane reads its two values k0, k0 + 2 with one 8-byte load
          sz[lane * 4 + 0] = w3[0];
          sz[lane * 4 + 1] = w3[2];
          sz[lane * 4 + 2] = w3[1];
          sz[lane * 4 + 3] = w3[3];
        } else {
#pragma unroll
          for (int k = 0; k < P; k++) sz[lane * SZ + k] = w3[k];
        }
        sb[lane] = base;
      }
      __syncwarp();
      if constexpr (P == 4) {
        const int ij = lane >> 1, k0 = lane & 1;
        const int off = (ij >> 2) * XS + (ij & 3) * ZP + k0;
        for (int a = 0; a < na; a++) {
          float* dst = acc + sb[a] + off;
          const float w = sq[a * SQ + ij];
          const float2 z2 = *reinterpret_cast<const float2*>(sz + a * 4 + 2 * k0);
          dst[0] = fmaf(w, z2.x, dst[0]);
          dst[2] = fmaf(w, z2.y, dst[2]);
          __syncwarp();  // lanes of the next atom may write the points this one wrote
        }
      } else {
        for (int a = 0; a < na; a++) {
          const int base = sb[a];
          const float* qa = sq + a * SQ;
          const float* za = sz + a * SZ;
#pragma unroll
          for (int r = 0; r < R; r++) {
            const int c = lane + 32 * r;
            if (P3 % 32 != 0 && c >= P3) continue;
            const int ij = c / P, k = c % P;
            float* dst = acc + base + (ij / P) * XS + (ij % P) * ZP + k;
            *dst = fmaf(qa[ij], za[k], *dst);
          }
          __syncwarp();  // lanes of the next atom may write the points this one wrote
        }
      }
    }
    uz += wend - wz + 1;
  }
  __syncwarp();
  float* out = apart + S.apart + (long long)(cx * Cy + cy) * (Fx * Fy) * L.n[2] + z0;
  for (int fx = 0; fx < Fx; fx++)
    for (int fy = 0; fy < Fy; fy++) {
      const float* src = acc + fx * XS + fy * ZP + P - 1;
      float* dst = out + (long long)(fx * Fy + fy) * L.n[2];
      for (int z = lane; z < zlen; z += 32) dst[z] = src[z];
    }
}

// binning cells of one axis whose footprint may hold level-1 coordinate m:
// candidates [c_a, c_b] (a cell c of a periodic axis may lie outside [0, C):
// it stands for c mod C shifted by whole periods)
template <int P>
__device__ __forceinline__ void foot_cells(const SysDev& S, int d, int m, int F, int& ca, int& cb) {
  constexpr int H = P / 2;
  if (S.ashift[d] >= 0) {
    ca = (m + H - F) >> S.ashift[d];
    cb = (m + H - 1) >> S.ashift[d];
  } else {
    ca = max((int)floorf((float)(m + H - F) * S.ainv[d]) - 1, 0);
    cb = min((int)floorf((float)(m + H) * S.ainv[d]) + 1, S.C[d] - 1);
  }
}

// One block per kAntSumY level-1 grid columns (gx, gy .. gy + kAntSumY - 1) and
// chunk of kAntSumZ points along z, kAntSumZ threads per column: the threads of
// a column test the candidate (binning column, footprint offset) pairs that may
// hold it in parallel, then each sums the valid ones for its z in the
// candidates' order.
template <int P>
__global__ void __launch_bounds__(kAntSumZ * kAntSumY, 8) k_anterp_sum(const SysDev* __restrict__ sys,
                                                                    const LevDev* __restrict__ levs,
                                                                    const TileItem* __restrict__ items,
                                                                    const float* __restrict__ apart,
                                                                    float* __restrict__ grid) {
  constexpr int NC = kAntFootMax * kAntFootMax;
  __shared__ long long off[kAntSumY][NC];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = levs[it.lev];
  const SysDev& S = sys[L.sys];
  const int col = threadIdx.x / kAntSumZ, tz = threadIdx.x % kAntSumZ;
  const int gx = it.x0, gy = it.y0 + col;
  const long long nz = L.n[2];
  const int Fx = S.afoot[0], Fy = S.afoot[1], Cx = S.C[0], Cy = S.C[1];
  const int mx = gx + L.lo[0], my = gy + L.lo[1];
  int xa, xb, ya, yb;
  foot_cells<P>(S, 0, mx, Fx, xa, xb);
  foot_cells<P>(S, 1, my, Fy, ya, yb);
  const int ny = yb - ya + 1, nc = min((xb - xa + 1) * ny, NC);
  for (int t = tz; t < nc; t += kAntSumZ) {
    const int c = xa + t / ny, e = ya + t % ny;
    const int fx = mx - cell_lo<P>(S, 0, c), fy = my - cell_lo<P>(S, 1, e);
    long long o = -1;
    if (fx >= 0 && fx < Fx && fy >= 0 && fy < Fy) {
      const int wx = S.pbc[0] ? (c & (Cx - 1)) : c;  // C is a power of two on a periodic axis
      const int wy = S.pbc[1] ? (e & (Cy - 1)) : e;
      o = S.apart + ((long long)(wx * Cy + wy) * (Fx * Fy) + fx * Fy + fy) * nz;
    }
    off[col][t] = o;
  }
  __syncthreads();
  const int z = it.z0 + tz;
  if (gy >= L.n[1] || z >= L.n[2]) return;
  // sixteen loads in flight before their sum (in the candidates' order; a
  // footprint of 5 grid columns per axis has 9 candidates, so one round trip)
  float v = 0.f;
  for (int t0 = 0; t0 < nc; t0 += 16) {
    float x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const long long o = t0 + k < nc ? off[col][t0 + k] : -1;
      x[k] = o >= 0 ? __ldg(apart + o + z) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 16; k++) v += x[k];
  }
  grid[L.q_off + ((long long)gx * L.n[1] + gy) * nz + z] = v;
}

template <int P>
static void run_anterp(const Work& w, const Tables& t, const TileItem* items, int nitems, cudaStream_t s, int tz) {
  if (tz == 16) k_anterp<P, 16><<<nitems, kAntNT, 0, s>>>(t.sys, t.lev, items, w.cell_start, w.uq, w.grid);
  else if (tz == 64) k_anterp<P, 64><<<nitems, kAntNT, 0, s>>>(t.sys, t.lev, items, w.cell_start, w.uq, w.grid);
  else k_anterp<P, 32><<<nitems, kAntNT, 0, s>>>(t.sys, t.lev, items, w.cell_start, w.uq, w.grid);
}

template <int P>
static void run_anterp_dipole(const Work& w, const Tables& t, const TileItem* items, int nitems, cudaStream_t s,
                              int tz, const float4* us) {
  if (tz == 16) k_anterp<P, 16, true><<<nitems, kAntNT, 0, s>>>(t.sys, t.lev, items, w.cell_start, w.uq, w.grid, us);
  else if (tz == 64) k_anterp<P, 64, true><<<nitems, kAntNT, 0, s>>>(t.sys, t.lev, items, w.cell_start, w.uq, w.grid, us);
  else k_anterp<P, 32, true><<<nitems, kAntNT, 0, s>>>(t.sys, t.lev, items, w.cell_start, w.uq, w.grid, us);
}

void launch_anterp_dipole(const Work& w, const Tables& t, const TileItem* items, int nitems, cudaStream_t s, int p,
                          int tz, const float4* us) {
  if (nitems <= 0) return;
  switch (p) {
    case 4: run_anterp_dipole<4>(w, t, items, nitems, s, tz, us); break;
    case 6: run_anterp_dipole<6>(w, t, items, nitems, s, tz, us); break;
    default: run_anterp_dipole<8>(w, t, items, nitems, s, tz, us); break;
  }
}

// Hessian of the interpolated potential at every atom times its upstream
// vector, (grad grad phi^(1+)(r_i)) u_i (second derivatives of the tensor
// B-spline basis), and u_i . E_i from the stored field parts; in place over
// the short-range field array: fout[k] = ((H u)_grid, u . E).
template <int P>
__global__ void __launch_bounds__(kChunk) k_interp_hess(const SysDev* __restrict__ sys, const LevDev* __restrict__ levs,
                                                        const AtomItem* __restrict__ items,
                                                        const float4* __restrict__ uq, const float* __restrict__ grid,
                                                        const float4* __restrict__ us, const float4* f_lr,
                                                        float4* fsr_inout) {
  constexpr int H = P / 2;
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  int local = it.start + threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  int k = S.atom_off + local;
  const float4 u = us[k];
  const float4 ea = fsr_inout[k], eb = f_lr[k];
  const float uE = u.x * (ea.x + eb.x) + u.y * (ea.y + eb.y) + u.z * (ea.z + eb.z);
  float hx = 0.f, hy = 0.f, hz = 0.f;
  if (S.ncomp >= 1) {
    const LevDev& L = levs[S.lev0];
    float4 u4 = uq[k];
    float uu[3] = {u4.x, u4.y, u4.z};
    float w[3][P], dw[3][P], d2w[3][P];
    int ix[3][P];
#pragma unroll
    for (int d = 0; d < 3; d++) {
      float fl = floorf(uu[d]);
      int base = (int)fl - H + 1;
      bspline_weights2<P>(uu[d] - fl, w[d], dw[d], d2w[d]);
#pragma unroll
      for (int j = 0; j < P; j++) {
        int m = base + j;
        ix[d][j] = L.per[d] ? (m & (L.n[d] - 1)) : m - L.lo[d];  // periodic grid counts are powers of two
      }
    }
    const float* e = grid + L.e_off;
    float gxx = 0.f, gyy = 0.f, gzz = 0.f, gxy = 0.f, gxz = 0.f, gyz = 0.f;
#pragma unroll
    for (int jx = 0; jx < P; jx++) {
#pragma unroll
      for (int jy = 0; jy < P; jy++) {
        const float* row = e + ((long long)ix[0][jx] * L.n[1] + ix[1][jy]) * L.n[2];
        float sz = 0.f, dsz = 0.f, d2sz = 0.f;
#pragma unroll
        for (int jz = 0; jz < P; jz++) {
          float ev = __ldg(row + ix[2][jz]);
          sz = fmaf(w[2][jz], ev, sz);
          dsz = fmaf(dw[2][jz], ev, dsz);
          d2sz = fmaf(d2w[2][jz], ev, d2sz);
        }
        gxx = fmaf(d2w[0][jx] * w[1][jy], sz, gxx);
        gyy = fmaf(w[0][jx] * d2w[1][jy], sz, gyy);
        gzz = fmaf(w[0][jx] * w[1][jy], d2sz, gzz);
        gxy = fmaf(dw[0][jx] * dw[1][jy], sz, gxy);
        gxz = fmaf(dw[0][jx] * w[1][jy], dsz, gxz);
        gyz = fmaf(w[0][jx] * dw[1][jy], dsz, gyz);
      }
    }
    if (S.tri) {
      // grad_r grad_r G = J H_u J^T (J = A^-1 diag(M)): (H u) = J (H_u (J^T u))
      const float* J = S.Jg;
      const float vx = J[0] * u.x + J[3] * u.y + J[6] * u.z, vy = J[1] * u.x + J[4] * u.y + J[7] * u.z,
                  vz = J[2] * u.x + J[5] * u.y + J[8] * u.z;
      const float wx = gxx * vx + gxy * vy + gxz * vz, wy = gxy * vx + gyy * vy + gyz * vz,
                  wz = gxz * vx + gyz * vy + gzz * vz;
      hx = J[0] * wx + J[1] * wy + J[2] * wz;
      hy = J[3] * wx + J[4] * wy + J[5] * wz;
      hz = J[6] * wx + J[7] * wy + J[8] * wz;
    } else {
      const float ax = S.inv_h1[0], ay = S.inv_h1[1], az = S.inv_h1[2];
      gxx *= ax * ax;
      gyy *= ay * ay;
      gzz *= az * az;
      gxy *= ax * ay;
      gxz *= ax * az;
      gyz *= ay * az;
      hx = gxx * u.x + gxy * u.y + gxz * u.z;
      hy = gxy * u.x + gyy * u.y + gyz * u.z;
      hz = gxz * u.x + gyz * u.y + gzz * u.z;
    }
  }
  fsr_inout[k] = make_float4(hx, hy, hz, uE);
}

void launch_interp_hess(const Work& w, const Tables& t, const AtomItem* items, int nitems, const float4* us,
                        cudaStream_t s, int p) {
  switch (p) {
    case 4: k_interp_hess<4><<<nitems, kChunk, 0, s>>>(t.sys, t.lev, items, w.uq, w.grid, us, w.f_lr, w.f_sr); break;
    case 6: k_interp_hess<6><<<nitems, kChunk, 0, s>>>(t.sys, t.lev, items, w.uq, w.grid, us, w.f_lr, w.f_sr); break;
    default: k_interp_hess<8><<<nitems, kChunk, 0, s>>>(t.sys, t.lev, items, w.uq, w.grid, us, w.f_lr, w.f_sr); break;
  }
}

// tz: the z-extent of the tiles the items were built for (16, 32 or 64)
void launch_anterp(const Work& w, const Tables& t, const TileItem* items, int nitems, cudaStream_t s, int p, int tz) {
  if (nitems <= 0) return;
  switch (p) {
    case 4: run_anterp<4>(w, t, items, nitems, s, tz); break;
    case 6: run_anterp<6>(w, t, items, nitems, s, tz); break;
    default: run_anterp<8>(w, t, items, nitems, s, tz); break;
  }
}

template <int P>
static void run_anterp_cols(const Work& w, const Tables& t, const TileItem* cols, int ncol, const TileItem* sums,
                            int nsum, int tz, int wstride, cudaStream_t s) {
  const size_t bytes = sizeof(float) * kAntWarps * (size_t)wstride;
  static size_t attr = 0;
  if (bytes > 48 * 1024 && bytes > attr &&
      cudaFuncSetAttribute(k_anterp_cols<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
    attr = bytes;
  if (ncol > 0)
    k_anterp_cols<P><<<(ncol + kAntWarps - 1) / kAntWarps, kAntWarps * 32, bytes, s>>>(
        t.sys, t.lev, cols, ncol, tz, wstride, w.cell_start, w.uq, w.apart);
  if (nsum > 0) k_anterp_sum<P><<<nsum, kAntSumZ * kAntSumY, 0, s>>>(t.sys, t.lev, sums, w.apart, w.grid);
}

// floats of shared memory per warp of k_anterp_cols for footprints up to fx_max x fy_max
int anterp_cols_wstride(int fx_max, int fy_max, int tz, int p) {
  return ((fx_max * ant_xs(fy_max, tz, p) + 3) & ~3) + ant_stage_floats(p);
}

void launch_anterp_cols(const Work& w, const Tables& t, const TileItem* cols, int ncol, const TileItem* sums,
                        int nsum, int tz, int wstride, cudaStream_t s, int p) {
  switch (p) {
    case 4: run_anterp_cols<4>(w, t, cols, ncol, sums, nsum, tz, wstride, s); break;
    case 6: run_anterp_cols<6>(w, t, cols, ncol, sums, nsum, tz, wstride, s); break;
    default: run_anterp_cols<8>(w, t, cols, ncol, sums, nsum, tz, wstride, s); break;
  }
}

void launch_interp(const Work& w, const Tables& t, const AtomItem* items, int nitems, bool forces,
                   cudaStream_t s, int p) {
  switch (p) {
    case 4: k_interp<4><<<nitems, kChunk, 0, s>>>(t.sys, t.lev, items, w.uq, w.grid, w.phi_lr, w.f_lr, forces); break;
    case 6: k_interp<6><<<nitems, kChunk, 0, s>>>(t.sys, t.lev, items, w.uq, w.grid, w.phi_lr, w.f_lr, forces); break;
    default: k_interp<8><<<nitems, kChunk, 0, s>>>(t.sys, t.lev, items, w.uq, w.grid, w.phi_lr, w.f_lr, forces); break;
  }
}

}  // namespace msm
