// k_grid.cu -- grid <-> grid translation operators of the MSM (Sec. 2 and
// Eq. restriction_prolongation_explicit_formulas):
//   restriction   q~^(l+1)_m = sum_n J_(n-2m) q~^l_n,
//   prolongation  e^l_m     += sum_n J_(m-2n) e^(l+1)_n   (the transpose),
// with the separable J_n = J_nx J_ny J_nz (B-spline two-scale coefficients,
// J_k = 2^(1-p) C(p, k+p/2)). Periodic axes wrap; open axes drop points
// outside the level's index range. Restriction: one thread per coarse point;
// prolongation: one block per fine tile, separable passes in shared memory.
// All systems of a batch in one launch per level step.
#include "msm_internal.h"

namespace msm {

__device__ __forceinline__ int wrap_g(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}
__device__ __forceinline__ int floordiv_g(int a, int b) {
  int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// storage index of grid coordinate m on axis d of a level, or -1 (open axis,
// outside the level's index range)
__device__ __forceinline__ int grid_index(const LevDev& L, int d, int m) {
  if (L.per[d]) return wrap_g(m, L.n[d]);
  const int s = m - L.lo[d];
  return (s >= 0 && s < L.n[d]) ? s : -1;
}

// Restriction, one thread per coarse point: (p+1)^3 taps read from L1.
template <int P>
__global__ void __launch_bounds__(kGridChunk) k_restrict(const SysDev* __restrict__ sys,
                                                         const LevDev* __restrict__ levs,
                                                         const RangeItem* __restrict__ items,
                                                         float* __restrict__ grid) {
  constexpr int H = P / 2;
  RangeItem it = items[blockIdx.x];
  if ((int)threadIdx.x >= it.count) return;
  const LevDev& Cl = levs[it.lev];
  const LevDev& Fl = levs[it.lev - 1];
  const SysDev& S = sys[Cl.sys];
  int idx = it.start + threadIdx.x;
  int cz = idx % Cl.n[2], cy = (idx / Cl.n[2]) % Cl.n[1], cx = idx / (Cl.n[2] * Cl.n[1]);
  int c[3] = {cx, cy, cz};
  int fi[3][P + 1];
  float jw[P + 1];
#pragma unroll
  for (int k = 0; k <= P; k++) jw[k] = S.jc[k];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    int m = c[d] + Cl.lo[d];
#pragma unroll
    for (int k = 0; k <= P; k++) {
      int f = 2 * m + (k - H);
      if (Fl.per[d]) {
        fi[d][k] = f & (Fl.n[d] - 1);  // periodic level sizes are powers of two
      } else {
        int s = f - Fl.lo[d];
        fi[d][k] = (s >= 0 && s < Fl.n[d]) ? s : -1;
      }
    }
  }
  const float* src = grid + Fl.q_off;
  float acc = 0.f;
#pragma unroll
  for (int kx = 0; kx <= P; kx++) {
    if (fi[0][kx] < 0) continue;
    float ay = 0.f;
#pragma unroll
    for (int ky = 0; ky <= P; ky++) {
      if (fi[1][ky] < 0) continue;
      const float* row = src + ((long long)fi[0][kx] * Fl.n[1] + fi[1][ky]) * Fl.n[2];
      float az = 0.f;
#pragma unroll
      for (int kz = 0; kz <= P; kz++)
        if (fi[2][kz] >= 0) az = fmaf(jw[kz], __ldg(row + fi[2][kz]), az);
      ay = fmaf(jw[ky], az, ay);
    }
    acc = fmaf(jw[kx], ay, acc);
  }
  grid[Cl.q_off + idx] = acc;
}

// Prolongation, one block per fine tile of kProTX x kProTY x kProTZ points:
// e^l_m += sum_n J_(m - 2n) e^(l+1)_n. The block stages the coarse points the
// tile reads (wrapped or zero) and applies the transposed filter along z, y
// and x in turn; each fine point takes the at most H + 1 coarse points with
// |m - 2n| <= H per axis.
template <int P>
__global__ void __launch_bounds__(256) k_prolong(const SysDev* __restrict__ sys, const LevDev* __restrict__ levs,
                                                 const TileItem* __restrict__ items, float* __restrict__ grid) {
  constexpr int H = P / 2, NT = 256;
  constexpr int CX = kProTX / 2 + H + 1, CY = kProTY / 2 + H + 1, CZ = kProTZ / 2 + H + 1;
  __shared__ float crs[CX * CY * CZ];
  __shared__ float pz[CX * CY * kProTZ];
  __shared__ float py[CX * kProTY * kProTZ];
  __shared__ int ix[CX], iy[CY], iz[CZ];
  const TileItem it = items[blockIdx.x];
  const LevDev& Fl = levs[it.lev];
  const LevDev& Cl = levs[it.lev + 1];
  const SysDev& S = sys[Fl.sys];
  const int t = threadIdx.x;
  // first coarse coordinate per axis: ceil((m0 - H) / 2), m0 the tile's first fine coordinate
  const int m0[3] = {it.x0 + Fl.lo[0], it.y0 + Fl.lo[1], it.z0 + Fl.lo[2]};
  int n0[3];
#pragma unroll
  for (int d = 0; d < 3; d++) n0[d] = -floordiv_g(-(m0[d] - H), 2);
  for (int e = t; e < CX; e += NT) ix[e] = grid_index(Cl, 0, n0[0] + e);
  for (int e = t; e < CY; e += NT) iy[e] = grid_index(Cl, 1, n0[1] + e);
  for (int e = t; e < CZ; e += NT) iz[e] = grid_index(Cl, 2, n0[2] + e);
  float jw[P + 1];
#pragma unroll
  for (int k = 0; k <= P; k++) jw[k] = S.jc[k];
  __syncthreads();
  const float* src = grid + Cl.e_off;
  for (int e = t; e < CX * CY * CZ; e += NT) {
    const int z = e % CZ, y = (e / CZ) % CY, x = e / (CZ * CY);
    const int a = ix[x], b = iy[y], c = iz[z];
    crs[e] = (a >= 0 && b >= 0 && c >= 0) ? src[((long long)a * Cl.n[1] + b) * Cl.n[2] + c] : 0.f;
  }
  __syncthreads();
  // weight of staged coarse index u for fine offset i along an axis: J_(m0 + i - 2 (n0 + u))
  auto w = [&](int d, int i, int u) {
    const int k = m0[d] + i - 2 * (n0[d] + u);
    return (k >= -H && k <= H) ? jw[k + H] : 0.f;
  };
  for (int e = t; e < CX * CY * kProTZ; e += NT) {
    const int z = e % kProTZ, xy = e / kProTZ;
    const int u0 = (m0[2] + z - H - 2 * n0[2] + 1) >> 1;  // ceil((m - H) / 2) - n0: first u with k <= H
    float v = 0.f;
#pragma unroll
    for (int u = 0; u <= H; u++)
      if (u0 + u < CZ) v = fmaf(w(2, z, u0 + u), crs[xy * CZ + u0 + u], v);
    pz[e] = v;
  }
  __syncthreads();
  for (int e = t; e < CX * kProTY * kProTZ; e += NT) {
    const int z = e % kProTZ, y = (e / kProTZ) % kProTY, x = e / (kProTZ * kProTY);
    const int u0 = (m0[1] + y - H - 2 * n0[1] + 1) >> 1;
    float v = 0.f;
#pragma unroll
    for (int u = 0; u <= H; u++)
      if (u0 + u < CY) v = fmaf(w(1, y, u0 + u), pz[(x * CY + u0 + u) * kProTZ + z], v);
    py[e] = v;
  }
  __syncthreads();
  for (int e = t; e < kProTX * kProTY * kProTZ; e += NT) {
    const int z = e % kProTZ, y = (e / kProTZ) % kProTY, x = e / (kProTZ * kProTY);
    const int fx = it.x0 + x, fy = it.y0 + y, fz = it.z0 + z;
    if (fx >= Fl.n[0] || fy >= Fl.n[1] || fz >= Fl.n[2]) continue;
    const int u0 = (m0[0] + x - H - 2 * n0[0] + 1) >> 1;
    float v = 0.f;
#pragma unroll
    for (int u = 0; u <= H; u++)
      if (u0 + u < CX) v = fmaf(w(0, x, u0 + u), py[((u0 + u) * kProTY + y) * kProTZ + z], v);
    grid[Fl.e_off + ((long long)fx * Fl.n[1] + fy) * Fl.n[2] + fz] += v;
  }
}

void launch_restrict(const Work& w, const Tables& t, const RangeItem* items, int nitems, cudaStream_t s, int p) {
  if (nitems <= 0) return;
  switch (p) {
    case 4: k_restrict<4><<<nitems, kGridChunk, 0, s>>>(t.sys, t.lev, items, w.grid); break;
    case 6: k_restrict<6><<<nitems, kGridChunk, 0, s>>>(t.sys, t.lev, items, w.grid); break;
    default: k_restrict<8><<<nitems, kGridChunk, 0, s>>>(t.sys, t.lev, items, w.grid); break;
  }
}

void launch_prolong(const Work& w, const Tables& t, const TileItem* items, int nitems, cudaStream_t s, int p) {
  if (nitems <= 0) return;
  switch (p) {
    case 4: k_prolong<4><<<nitems, 256, 0, s>>>(t.sys, t.lev, items, w.grid); break;
    case 6: k_prolong<6><<<nitems, 256, 0, s>>>(t.sys, t.lev, items, w.grid); break;
    default: k_prolong<8><<<nitems, 256, 0, s>>>(t.sys, t.lev, items, w.grid); break;
  }
}

}  // namespace msm
