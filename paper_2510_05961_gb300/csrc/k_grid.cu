// k_grid.cu -- grid <-> grid translation operators of the MSM (Sec. 2 and
// Eq. restriction_prolongation_explicit_formulas):
//   restriction   q~^(l+1)_m = sum_n J_(n-2m) q~^l_n,
//   prolongation  e^l_m     += sum_n J_(m-2n) e^(l+1)_n   (the transpose),
// with the separable J_n = J_nx J_ny J_nz (B-spline two-scale coefficients,
// J_k = 2^(1-p) C(p, k+p/2)). Periodic axes wrap; open axes drop points
// outside the level's index range. One thread per output point, all systems
// of a batch in one launch per level step.
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
        fi[d][k] = wrap_g(f, Fl.n[d]);
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

template <int P>
__global__ void __launch_bounds__(kGridChunk) k_prolong(const SysDev* __restrict__ sys,
                                                        const LevDev* __restrict__ levs,
                                                        const RangeItem* __restrict__ items,
                                                        float* __restrict__ grid) {
  constexpr int H = P / 2;
  constexpr int NC = H + 1;  // coarse points that reach one fine point, at most
  RangeItem it = items[blockIdx.x];
  if ((int)threadIdx.x >= it.count) return;
  const LevDev& Fl = levs[it.lev];
  const LevDev& Cl = levs[it.lev + 1];
  const SysDev& S = sys[Fl.sys];
  int idx = it.start + threadIdx.x;
  int fz = idx % Fl.n[2], fy = (idx / Fl.n[2]) % Fl.n[1], fx = idx / (Fl.n[2] * Fl.n[1]);
  int f[3] = {fx, fy, fz};
  int ci[3][NC];
  float cw[3][NC];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    int m = f[d] + Fl.lo[d];
    int n0 = -floordiv_g(-(m - H), 2);  // ceil((m - H) / 2)
#pragma unroll
    for (int t = 0; t < NC; t++) {
      int n = n0 + t;
      int k = m - 2 * n;  // in [-H, H] when valid
      int s;
      if (k < -H || k > H) {
        s = -1;
      } else if (Cl.per[d]) {
        s = wrap_g(n, Cl.n[d]);
      } else {
        s = n - Cl.lo[d];
        if (s < 0 || s >= Cl.n[d]) s = -1;
      }
      ci[d][t] = s;
      cw[d][t] = (s >= 0) ? S.jc[k + H] : 0.f;
    }
  }
  const float* src = grid + Cl.e_off;
  float acc = 0.f;
#pragma unroll
  for (int tx = 0; tx < NC; tx++) {
    if (ci[0][tx] < 0) continue;
    float ay = 0.f;
#pragma unroll
    for (int ty = 0; ty < NC; ty++) {
      if (ci[1][ty] < 0) continue;
      const float* row = src + ((long long)ci[0][tx] * Cl.n[1] + ci[1][ty]) * Cl.n[2];
      float az = 0.f;
#pragma unroll
      for (int tz = 0; tz < NC; tz++)
        if (ci[2][tz] >= 0) az = fmaf(cw[2][tz], __ldg(row + ci[2][tz]), az);
      ay = fmaf(cw[1][ty], az, ay);
    }
    acc = fmaf(cw[0][tx], ay, acc);
  }
  grid[Fl.e_off + idx] += acc;
}

void launch_restrict(const Work& w, const Tables& t, const RangeItem* items, int nitems, cudaStream_t s, int p) {
  if (nitems <= 0) return;
  switch (p) {
    case 4: k_restrict<4><<<nitems, kGridChunk, 0, s>>>(t.sys, t.lev, items, w.grid); break;
    case 6: k_restrict<6><<<nitems, kGridChunk, 0, s>>>(t.sys, t.lev, items, w.grid); break;
    default: k_restrict<8><<<nitems, kGridChunk, 0, s>>>(t.sys, t.lev, items, w.grid); break;
  }
}

void launch_prolong(const Work& w, const Tables& t, const RangeItem* items, int nitems, cudaStream_t s, int p) {
  if (nitems <= 0) return;
  switch (p) {
    case 4: k_prolong<4><<<nitems, kGridChunk, 0, s>>>(t.sys, t.lev, items, w.grid); break;
    case 6: k_prolong<6><<<nitems, kGridChunk, 0, s>>>(t.sys, t.lev, items, w.grid); break;
    default: k_prolong<8><<<nitems, kGridChunk, 0, s>>>(t.sys, t.lev, items, w.grid); break;
  }
}

}  // namespace msm
