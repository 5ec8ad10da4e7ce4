// k_interp.cu -- particle <-> grid operations of the MSM (Sec. 3.2.2):
// anterpolation q~^1_m = sum_i q_i phi^1_m(r_i) (Eq. grid_charge,
// Alg. anterpolation_double_loop) and interpolation
// phi^(1+)_i = sum_m e^(1+)_m phi^1_m(r_i) with the position gradient
// q_i sum_m e^(1+)_m grad phi^1_m(r_i) (Eqs. uoneplus_interpolation_with_index_set,
// analytic_uoneplus_position_grad). The basis is the tensor product of
// centred cardinal B-splines of order p (Sec. 3.3), evaluated in FP32 by the
// uniform Cox-de Boor recursion on the fractional grid coordinate.
//
// Anterpolation is tile-owned: each block owns an 8^3 tile of the level-1
// grid, gathers the atoms of the cells whose B-spline support reaches the
// tile, and each thread sums one z-column of the tile over those atoms in a
// fixed order. No global atomics; the result is the same on every run.
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

template <int P>
__global__ void __launch_bounds__(64) k_anterp(const SysDev* __restrict__ sys, const LevDev* __restrict__ levs,
                                               const TileItem* __restrict__ items,
                                               const int* __restrict__ cell_start, const float4* __restrict__ uq,
                                               float* __restrict__ grid) {
  constexpr int T = kAnterpT;
  constexpr int CAP = 128;
  constexpr int H = P / 2;
  __shared__ float sw[CAP][3 * T];
  __shared__ int s_wtot[2];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = levs[it.lev];
  const SysDev& S = sys[L.sys];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tid / T, ty = tid % T;
  int st0[3] = {it.x0, it.y0, it.z0};
  int m0[3], m1[3], cl[3], ch[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    int e = st0[d] + T;
    if (e > L.n[d]) e = L.n[d];
    m0[d] = st0[d] + L.lo[d];
    m1[d] = e - 1 + L.lo[d];
    if (S.pbc[d] && S.M[d] % S.C[d] == 0) {
      // cells aligned with the grid (k intervals per cell, powers of two): the
      // cell of an atom is floor(u / k) exactly, so the range is exact
      const int k = S.M[d] / S.C[d];
      cl[d] = floordiv_i(m0[d] - H, k);
      ch[d] = floordiv_i(m1[d] + H - 1, k);
    } else {
      cl[d] = floordiv_i((m0[d] - H) * S.C[d], S.M[d]) - 1;
      ch[d] = floordiv_i((m1[d] + H) * S.C[d], S.M[d]) + 1;
    }
    if (!S.pbc[d]) {
      if (cl[d] < 0) cl[d] = 0;
      if (ch[d] > S.C[d] - 1) ch[d] = S.C[d] - 1;
    }
  }
  float acc[T];
#pragma unroll
  for (int z = 0; z < T; z++) acc[z] = 0.0f;
  int batch = 0;

  auto accumulate = [&](int nb) {
    for (int a = 0; a < nb; a++) {
      float wxy = sw[a][tx] * sw[a][T + ty];
      if (wxy != 0.0f) {
#pragma unroll
        for (int z = 0; z < T; z++) acc[z] = fmaf(wxy, sw[a][2 * T + z], acc[z]);
      }
    }
  };

  const int Cy = S.C[1], Cz = S.C[2];
  for (int ux = cl[0]; ux <= ch[0]; ux++) {
    int wx = wrap_i(ux, S.C[0]);
    int shx = floordiv_i(ux, S.C[0]) * S.M[0];
    for (int uy = cl[1]; uy <= ch[1]; uy++) {
      int wy = wrap_i(uy, Cy);
      int shy = floordiv_i(uy, Cy) * S.M[1];
      int uz = cl[2];
      while (uz <= ch[2]) {
        int wz = wrap_i(uz, Cz);
        int kz = floordiv_i(uz, Cz);
        int run = Cz - 1 - wz;
        if (uz + run > ch[2]) run = ch[2] - uz;
        int shz = kz * S.M[2];
        int cfirst = S.cell_off + (wx * Cy + wy) * Cz + wz;
        int ab = cell_start[cfirst], ae = cell_start[cfirst + run + 1];
        for (int base = ab; base < ae; base += 64) {
          int idx = base + tid;
          bool keep = false;
          float wv[3][P], dummy[P];
          int bb[3];
          if (idx < ae) {
            float4 u4 = uq[idx];
            float uu[3] = {u4.x, u4.y, u4.z};
            int sh[3] = {shx, shy, shz};
            keep = true;
#pragma unroll
            for (int d = 0; d < 3; d++) {
              float fl = floorf(uu[d]);
              int b = (int)fl + sh[d];
              bb[d] = b;
              if (b < m0[d] - H || b > m1[d] + H - 1) keep = false;
              bspline_weights<P, false>(uu[d] - fl, wv[d], dummy);
            }
            if (keep) {
#pragma unroll
              for (int j = 0; j < P; j++) wv[0][j] *= u4.w;
            }
          }
          unsigned bal = __ballot_sync(0xffffffffu, keep);
          int rank = __popc(bal & ((1u << lane) - 1u));
          if (lane == 0) s_wtot[warp] = __popc(bal);
          __syncthreads();
          int tot = s_wtot[0] + s_wtot[1];
          int before = (warp == 1) ? s_wtot[0] : 0;
          if (batch + tot > CAP) {
            accumulate(batch);
            __syncthreads();
            batch = 0;
          }
          if (keep) {
            int slotp = batch + before + rank;
#pragma unroll
            for (int d = 0; d < 3; d++) {
#pragma unroll
              for (int t = 0; t < T; t++) {
                int j = m0[d] + t - bb[d] + H - 1;
                float v = 0.0f;
#pragma unroll
                for (int jj = 0; jj < P; jj++) v = (j == jj) ? wv[d][jj] : v;
                sw[slotp][d * T + t] = v;
              }
            }
          }
          batch += tot;
          __syncthreads();
        }
        uz += run + 1;
      }
    }
  }
  accumulate(batch);
  int gx = it.x0 + tx, gy = it.y0 + ty;
  if (gx < L.n[0] && gy < L.n[1]) {
    float* out = grid + L.q_off + ((long long)gx * L.n[1] + gy) * L.n[2] + it.z0;
#pragma unroll
    for (int z = 0; z < T; z++)
      if (it.z0 + z < L.n[2]) out[z] = acc[z];
  }
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
      ix[d][j] = L.per[d] ? wrap_i(m, L.n[d]) : m - L.lo[d];
    }
  }
  const float* e = grid + L.e_off;
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
  if (want_f) {
    float qq = u4.w;
    f_lr[k] = make_float4(-qq * gx * S.inv_h1[0], -qq * gy * S.inv_h1[1], -qq * gz * S.inv_h1[2], 0.f);
  }
}

void launch_anterp(const Work& w, const Tables& t, const TileItem* items, int nitems, cudaStream_t s, int p) {
  if (nitems <= 0) return;
  switch (p) {
    case 4: k_anterp<4><<<nitems, 64, 0, s>>>(t.sys, t.lev, items, w.cell_start, w.uq, w.grid); break;
    case 6: k_anterp<6><<<nitems, 64, 0, s>>>(t.sys, t.lev, items, w.cell_start, w.uq, w.grid); break;
    default: k_anterp<8><<<nitems, 64, 0, s>>>(t.sys, t.lev, items, w.cell_start, w.uq, w.grid); break;
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
