// k_grid.cu -- grid <-> grid translation operators of the MSM (Sec. 2 and
// Eq. restriction_prolongation_explicit_formulas):
//   restriction   q~^(l+1)_m = sum_n J_(n-2m) q~^l_n,
//   prolongation  e^l_m     += sum_n J_(m-2n) e^(l+1)_n   (the transpose),
// with the separable J_n = J_nx J_ny J_nz (B-spline two-scale coefficients,
// J_k = 2^(1-p) C(p, k+p/2)). Periodic axes wrap; open axes drop points
// outside the level's index range. Both run as one block per tile with three
// separable 1-D passes in shared memory.
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

// Copies the box of points (ix[x], iy[y], iz[z]) of a level grid into shared
// memory (z fastest), zero where an index is -1. Every load of a thread is
// issued before its first store, so each thread waits for one memory round
// trip instead of one per point.
template <int NX, int NY, int NZ, int NT>
__device__ __forceinline__ void stage_box(float* __restrict__ dst, const float* __restrict__ src, const int* ix,
                                          const int* iy, const int* iz, int n1, int n2) {
  constexpr int N = NX * NY * NZ, R = (N + NT - 1) / NT;
  float v[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int e = (int)threadIdx.x + r * NT;
    v[r] = 0.f;
    if (e < N) {
      const int z = e % NZ, y = (e / NZ) % NY, x = e / (NZ * NY);
      const int a = ix[x], b = iy[y], c = iz[z];
      if (a >= 0 && b >= 0 && c >= 0) v[r] = __ldg(src + ((long long)a * n1 + b) * n2 + c);
    }
  }
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int e = (int)threadIdx.x + r * NT;
    if (e < N) dst[e] = v[r];
  }
}

// Restriction, one block per coarse tile of kResTX x kResTY x kResTZ points,
// as three 1-D passes: the block stages the fine points its tile reads
// (2 T + p - 1 per axis, wrapped or zero), then applies J along x, y and z in
// turn in shared memory. Coarse offset i along an axis reads the staged fine
// offsets 2 i + k, k = 0 .. p, with weight J_(k - p/2).
template <int P>
__global__ void __launch_bounds__(kResNT) k_restrict(const SysDev* __restrict__ sys, const LevDev* __restrict__ levs,
                                                     const TileItem* __restrict__ items, float* __restrict__ grid) {
  constexpr int H = P / 2, NT = kResNT;
  constexpr int FX = 2 * kResTX + P - 1, FY = 2 * kResTY + P - 1, FZ = 2 * kResTZ + P - 1;
  __shared__ float fine[FX * FY * FZ];      // staged fine points; later the output of the y pass
  __shared__ float ax[kResTX * FY * FZ];    // output of the x pass
  __shared__ int ix[FX], iy[FY], iz[FZ];
  const TileItem it = items[blockIdx.x];
  const LevDev& Cl = levs[it.lev];
  const LevDev& Fl = levs[it.lev - 1];
  const SysDev& S = sys[Cl.sys];
  const int t = threadIdx.x;
  // first staged fine coordinate per axis: 2 m0 - p/2, m0 the tile's first coarse coordinate
  const int f0[3] = {2 * (it.x0 + Cl.lo[0]) - H, 2 * (it.y0 + Cl.lo[1]) - H, 2 * (it.z0 + Cl.lo[2]) - H};
  for (int e = t; e < FX; e += NT) ix[e] = grid_index(Fl, 0, f0[0] + e);
  for (int e = t; e < FY; e += NT) iy[e] = grid_index(Fl, 1, f0[1] + e);
  for (int e = t; e < FZ; e += NT) iz[e] = grid_index(Fl, 2, f0[2] + e);
  float jw[P + 1];
#pragma unroll
  for (int k = 0; k <= P; k++) jw[k] = S.jc[k];
  __syncthreads();
  const float* src = grid + Fl.q_off;
  stage_box<FX, FY, FZ, NT>(fine, src, ix, iy, iz, Fl.n[1], Fl.n[2]);
  __syncthreads();
  for (int e = t; e < kResTX * FY * FZ; e += NT) {
    const int yz = e % (FY * FZ), i = e / (FY * FZ);
    const float* f = fine + 2 * i * (FY * FZ) + yz;
    float v = 0.f;
#pragma unroll
    for (int k = 0; k <= P; k++) v = fmaf(jw[k], f[k * (FY * FZ)], v);
    ax[e] = v;
  }
  __syncthreads();
  float* ay = fine;  // kResTX x kResTY x FZ
  for (int e = t; e < kResTX * kResTY * FZ; e += NT) {
    const int z = e % FZ, ij = e / FZ, j = ij % kResTY, i = ij / kResTY;
    const float* f = ax + (i * FY + 2 * j) * FZ + z;
    float v = 0.f;
#pragma unroll
    for (int k = 0; k <= P; k++) v = fmaf(jw[k], f[k * FZ], v);
    ay[e] = v;
  }
  __syncthreads();
  for (int e = t; e < kResTX * kResTY * kResTZ; e += NT) {
    const int kz = e % kResTZ, ij = e / kResTZ, j = ij % kResTY, i = ij / kResTY;
    const int cx = it.x0 + i, cy = it.y0 + j, cz = it.z0 + kz;
    if (cx >= Cl.n[0] || cy >= Cl.n[1] || cz >= Cl.n[2]) continue;
    const float* f = ay + ij * FZ + 2 * kz;
    float v = 0.f;
#pragma unroll
    for (int k = 0; k <= P; k++) v = fmaf(jw[k], f[k], v);
    grid[Cl.q_off + ((long long)cx * Cl.n[1] + cy) * Cl.n[2] + cz] = v;
  }
}

// Prolongation, one block per fine tile of kProTX x kProTY x kProTZ points:
// e^l_m += sum_n J_(m - 2n) e^(l+1)_n. The block stages the coarse points the
// tile reads (wrapped or zero) and applies the transposed filter along z, y
// and x in turn. A fine point m takes the coarse points n = n_1(m) + u,
// n_1(m) = ceil((m - p/2) / 2), u = 0 .. p/2: J_(p/2 - 2u) when m - p/2 is
// even, J_(p/2 - 1 - 2u) (u < p/2) when it is odd.
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
  // first coarse coordinate per axis: n_1(m0), m0 the tile's first fine coordinate
  const int m0[3] = {it.x0 + Fl.lo[0], it.y0 + Fl.lo[1], it.z0 + Fl.lo[2]};
  int n0[3];
#pragma unroll
  for (int d = 0; d < 3; d++) n0[d] = (m0[d] - H + 1) >> 1;
  for (int e = t; e < CX; e += NT) ix[e] = grid_index(Cl, 0, n0[0] + e);
  for (int e = t; e < CY; e += NT) iy[e] = grid_index(Cl, 1, n0[1] + e);
  for (int e = t; e < CZ; e += NT) iz[e] = grid_index(Cl, 2, n0[2] + e);
  // weights by tap u and the parity of m - p/2 (the odd case has p/2 taps)
  float we[H + 1], wo[H + 1];
#pragma unroll
  for (int u = 0; u <= H; u++) {
    we[u] = S.jc[2 * H - 2 * u];
    wo[u] = u < H ? S.jc[2 * H - 1 - 2 * u] : 0.f;
  }
  __syncthreads();
  // the fine values this thread adds to, loaded before the staging so that both round trips overlap
  constexpr int RO = kProTX * kProTY * kProTZ / NT;
  static_assert(RO * NT == kProTX * kProTY * kProTZ, "whole outputs per thread");
  float old[RO];
  long long dst[RO];
#pragma unroll
  for (int r = 0; r < RO; r++) {
    const int e = t + r * NT;
    const int z = e % kProTZ, y = (e / kProTZ) % kProTY, x = e / (kProTZ * kProTY);
    const int fx = it.x0 + x, fy = it.y0 + y, fz = it.z0 + z;
    dst[r] = -1;
    old[r] = 0.f;
    if (fx < Fl.n[0] && fy < Fl.n[1] && fz < Fl.n[2]) {
      dst[r] = Fl.e_off + ((long long)fx * Fl.n[1] + fy) * Fl.n[2] + fz;
      old[r] = grid[dst[r]];
    }
  }
  const float* src = grid + Cl.e_off;
  stage_box<CX, CY, CZ, NT>(crs, src, ix, iy, iz, Cl.n[1], Cl.n[2]);
  __syncthreads();
  // fine offset i along axis d: first staged coarse index u0 = n_1(m0 + i) - n0 and the parity
  // of m0 + i - p/2; u0 + p/2 < T/2 + p/2 + 1 stays inside the staged range
  auto taps = [&](int d, int i, int& u0) {
    const int m = m0[d] + i - H;
    u0 = ((m + 1) >> 1) - n0[d];
    return (m & 1) != 0;
  };
  for (int e = t; e < CX * CY * kProTZ; e += NT) {
    const int z = e % kProTZ, xy = e / kProTZ;
    int u0;
    const bool odd = taps(2, z, u0);
    const float* c = crs + xy * CZ + u0;
    float v = 0.f;
#pragma unroll
    for (int u = 0; u <= H; u++) v = fmaf(odd ? wo[u] : we[u], c[u], v);
    pz[e] = v;
  }
  __syncthreads();
  for (int e = t; e < CX * kProTY * kProTZ; e += NT) {
    const int z = e % kProTZ, y = (e / kProTZ) % kProTY, x = e / (kProTZ * kProTY);
    int u0;
    const bool odd = taps(1, y, u0);
    const float* c = pz + (x * CY + u0) * kProTZ + z;
    float v = 0.f;
#pragma unroll
    for (int u = 0; u <= H; u++) v = fmaf(odd ? wo[u] : we[u], c[u * kProTZ], v);
    py[e] = v;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RO; r++) {
    if (dst[r] < 0) continue;
    const int e = t + r * NT;
    const int z = e % kProTZ, y = (e / kProTZ) % kProTY, x = e / (kProTZ * kProTY);
    int u0;
    const bool odd = taps(0, x, u0);
    const float* c = py + (u0 * kProTY + y) * kProTZ + z;
    float v = 0.f;
#pragma unroll
    for (int u = 0; u <= H; u++) v = fmaf(odd ? wo[u] : we[u], c[u * (kProTY * kProTZ)], v);
    grid[dst[r]] = old[r] + v;
  }
}

void launch_restrict(const Work& w, const Tables& t, const TileItem* items, int nitems, cudaStream_t s, int p) {
  if (nitems <= 0) return;
  switch (p) {
    case 4: k_restrict<4><<<nitems, kResNT, 0, s>>>(t.sys, t.lev, items, w.grid); break;
    case 6: k_restrict<6><<<nitems, kResNT, 0, s>>>(t.sys, t.lev, items, w.grid); break;
    default: k_restrict<8><<<nitems, kResNT, 0, s>>>(t.sys, t.lev, items, w.grid); break;
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
