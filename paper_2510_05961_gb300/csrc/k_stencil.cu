// k_stencil.cu -- the per-level grid-to-grid kernel sum of the MSM,
// e^l_m = sum_d K^l_d q~^l_(m-d) (Eq. action_of_K_as_convolution), and the
// grid part of the virial, W = -1/2 sum_l sum_d (dK^l/d eps)_d C^l_d with the
// autocorrelation C^l_d = sum_m q~^l_m q~^l_(m-d).
//
// Ball kernels (levels whose stencil support is a ball of radius R that does
// not overlap itself under the periodic wrap): one block per output tile of
// 1 x 32 x 32 points; the block streams the 2R+1 input x-planes of the tile's
// halo through shared memory (cp.async, double buffered, periodic wrap or
// zero fill done by the copy addresses) together with the matching x-slab of
// the stencil. Each thread owns 16 consecutive z outputs in registers and,
// per (dx, dy) stencil column of half-width w, loads 16 + 2w plane values and
// 2w + 1 stencil values and issues 16 (2w + 1) FFMA from registers; w picks
// an unrolled variant, so the ball shape costs nothing for empty columns.
// The arithmetic is FP32 on the CUDA cores: the contraction has no dense
// reduction axis, and a Toeplitz recast for the tensor cores would multiply
// the work by (16 + 2R)/(2R + 1) per axis while TF32 loses the accuracy the
// method needs.
//
// The virial kernel is the same loop with the roles swapped: per column a
// thread forms its partial C_(dx,dy,dz) for the 2w + 1 dz values and
// contracts it at once with the six strain-derivative weights (stored with
// the half-space symmetry C_d = C_-d folded in). Box kernels serve the small
// levels with folded (dense) stencils and the top level of open systems.
#include "msm_internal.h"

namespace msm {

constexpr int BZ = kBallBZ;
constexpr int TY = kBallTY;
constexpr int TZ = kBallTZ;
constexpr int NT = kBallThreads;

__device__ __forceinline__ int wrap_s(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc, bool valid) {
  unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  int bytes = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gsrc), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ------------------------------------------------------------------ columns
template <int W>
__device__ __forceinline__ void ball_column(float (&acc)[BZ], const float* __restrict__ qrow,
                                            const float* __restrict__ kc) {
  float qv[BZ + 2 * W];
#pragma unroll
  for (int t = 0; t < BZ + 2 * W; t++) qv[t] = qrow[t - W];
#pragma unroll
  for (int j = 0; j <= 2 * W; j++) {
    const float kv = kc[j - W];
#pragma unroll
    for (int o = 0; o < BZ; o++) acc[o] = fmaf(kv, qv[o - j + 2 * W], acc[o]);
  }
}

template <int W>
__device__ __forceinline__ void virial_column(float (&w6)[6], const float (&qown)[BZ],
                                              const float* __restrict__ qrow, const float* __restrict__ kc,
                                              int kstride) {
  float qv[BZ + 2 * W];
#pragma unroll
  for (int t = 0; t < BZ + 2 * W; t++) qv[t] = qrow[t - W];
#pragma unroll
  for (int j = 0; j <= 2 * W; j++) {
    float c = 0.f;
#pragma unroll
    for (int o = 0; o < BZ; o++) c = fmaf(qown[o], qv[o - j + 2 * W], c);
#pragma unroll
    for (int k = 0; k < 6; k++) w6[k] = fmaf(kc[k * kstride + j - W], c, w6[k]);
  }
}

template <int W, int WMAX>
struct Col {
  static __device__ __forceinline__ void stencil(int w, float (&acc)[BZ], const float* q, const float* k) {
    if (w == W)
      ball_column<W>(acc, q, k);
    else
      Col<W + 1, WMAX>::stencil(w, acc, q, k);
  }
  static __device__ __forceinline__ void virial(int w, float (&w6)[6], const float (&qown)[BZ], const float* q,
                                                const float* k, int ks) {
    if (w == W)
      virial_column<W>(w6, qown, q, k, ks);
    else
      Col<W + 1, WMAX>::virial(w, w6, qown, q, k, ks);
  }
};
template <int WMAX>
struct Col<WMAX, WMAX> {
  static __device__ __forceinline__ void stencil(int, float (&acc)[BZ], const float* q, const float* k) {
    ball_column<WMAX>(acc, q, k);
  }
  static __device__ __forceinline__ void virial(int, float (&w6)[6], const float (&qown)[BZ], const float* q,
                                                const float* k, int ks) {
    virial_column<WMAX>(w6, qown, q, k, ks);
  }
};

// ------------------------------------------------------------------ staging
// shared-memory carve-up: two plane buffers, two stencil slabs, two column tables
__device__ __forceinline__ float* sm_plane(float* smem, int plane_sz, int b) { return smem + b * plane_sz; }
__device__ __forceinline__ float* sm_kslab(float* smem, int plane_sz, int kslab_sz, int b) {
  return smem + 2 * plane_sz + b * kslab_sz;
}
__device__ __forceinline__ int* sm_wsl(float* smem, int plane_sz, int kslab_sz, int wsl_sz, int b) {
  return reinterpret_cast<int*>(smem + 2 * plane_sz + 2 * kslab_sz) + b * wsl_sz;
}

// Issue the copies of input plane x = x0 - dx (rows y0-Ry .. y0+TY-1+Ry,
// columns z0-Rz .. z0+TZ-1+Rz) and of the stencil x-slab of this dx.
__device__ __forceinline__ void stage(const LevDev& L, const TileItem& it, int step, const float* __restrict__ src,
                                      const float* __restrict__ kpool, long long kslab_off, int nkcomp,
                                      long long kcomp_stride, const int* __restrict__ wpool, long long w_off,
                                      float* plane, float* kslab, int* wsl, int stride) {
  const int Rx = L.R[0], Ry = L.R[1], Rz = L.R[2];
  const int rows = TY + 2 * Ry, cols = TZ + 2 * Rz;
  const int dx = step - Rx;
  int xs = it.x0 - dx;
  bool xok = true;
  if (L.per[0]) xs = wrap_s(xs, L.n[0]);
  else xok = (xs >= 0 && xs < L.n[0]);
  const int n1 = L.n[1], n2 = L.n[2];
  for (int e = threadIdx.x; e < rows * cols; e += NT) {
    int r = e / cols, c = e - r * cols;
    int ys = it.y0 - Ry + r, zs = it.z0 - Rz + c;
    bool ok = xok;
    if (L.per[1]) ys = wrap_s(ys, n1);
    else ok = ok && ys >= 0 && ys < n1;
    if (L.per[2]) zs = wrap_s(zs, n2);
    else ok = ok && zs >= 0 && zs < n2;
    const float* g = ok ? src + ((long long)xs * n1 + ys) * n2 + zs : src;
    cp_async4(plane + r * stride + c, g, ok);
  }
  const int ksz = (2 * Ry + 1) * (2 * Rz + 1);
  for (int k = 0; k < nkcomp; k++) {
    const float* ks = kpool + kslab_off + k * kcomp_stride + (long long)step * ksz;
    for (int e = threadIdx.x; e < ksz; e += NT) cp_async4(kslab + k * ksz + e, ks + e, true);
  }
  for (int e = threadIdx.x; e < 2 * Ry + 1; e += NT)
    cp_async4(wsl + e, wpool + w_off + (long long)step * (2 * Ry + 1) + e, true);
  cp_async_commit();
}

template <int WMAX>
__global__ void __launch_bounds__(NT) k_stencil_ball(const LevDev* __restrict__ levs,
                                                     const TileItem* __restrict__ items,
                                                     const float* __restrict__ kpool, const int* __restrict__ wpool,
                                                     float* __restrict__ grid, int plane_sz, int kslab_sz,
                                                     int wsl_sz, int stride) {
  extern __shared__ float smem[];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = levs[it.lev];
  const int Rx = L.R[0], Ry = L.R[1], Rz = L.R[2];
  const int ty = threadIdx.x % TY, zb = threadIdx.x / TY;
  const float* src = grid + L.q_off;
  float acc[BZ];
#pragma unroll
  for (int o = 0; o < BZ; o++) acc[o] = 0.f;
  const int nsteps = 2 * Rx + 1;
  const int ksz = (2 * Ry + 1) * (2 * Rz + 1);
  stage(L, it, 0, src, kpool, L.k_off, 1, 0, wpool, L.w_off, sm_plane(smem, plane_sz, 0), sm_kslab(smem, plane_sz, kslab_sz, 0), sm_wsl(smem, plane_sz, kslab_sz, wsl_sz, 0), stride);
  for (int step = 0; step < nsteps; step++) {
    cp_async_wait_all();
    __syncthreads();
    const int b = step & 1;
    if (step + 1 < nsteps)
      stage(L, it, step + 1, src, kpool, L.k_off, 1, 0, wpool, L.w_off, sm_plane(smem, plane_sz, b ^ 1),
            sm_kslab(smem, plane_sz, kslab_sz, b ^ 1), sm_wsl(smem, plane_sz, kslab_sz, wsl_sz, b ^ 1), stride);
    const float* plane = sm_plane(smem, plane_sz, b);
    const float* kslab = sm_kslab(smem, plane_sz, kslab_sz, b);
    const int* wsl = sm_wsl(smem, plane_sz, kslab_sz, wsl_sz, b);
    for (int dy = -Ry; dy <= Ry; dy++) {
      const int w = wsl[dy + Ry];
      if (w < 0) continue;
      const float* qrow = plane + (ty - dy + Ry) * stride + zb * BZ + Rz;
      const float* kc = kslab + (dy + Ry) * (2 * Rz + 1) + Rz;
      Col<0, WMAX>::stencil(w, acc, qrow, kc);
    }
    (void)ksz;
  }
  const int y = it.y0 + ty;
  if (y < L.n[1]) {
    float* out = grid + L.e_off + ((long long)it.x0 * L.n[1] + y) * L.n[2];
    const int z0 = it.z0 + zb * BZ;
#pragma unroll
    for (int o = 0; o < BZ; o++)
      if (z0 + o < L.n[2]) out[z0 + o] = acc[o] * L.scale;
  }
}

template <int WMAX>
__global__ void __launch_bounds__(NT) k_virial_ball(const LevDev* __restrict__ levs,
                                                    const TileItem* __restrict__ items,
                                                    const float* __restrict__ kpool, const int* __restrict__ wpool,
                                                    const float* __restrict__ grid, double* __restrict__ part,
                                                    int plane_sz, int kslab_sz, int wsl_sz, int stride) {
  extern __shared__ float smem[];
  __shared__ double red[NT / 32][6];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = levs[it.lev];
  const int Rx = L.R[0], Ry = L.R[1], Rz = L.R[2];
  const int ty = threadIdx.x % TY, zb = threadIdx.x / TY;
  const float* src = grid + L.q_off;
  const int ksz = (2 * Ry + 1) * (2 * Rz + 1);
  const long long kcs = (long long)(2 * Rx + 1) * ksz;  // one component of the dense box
  float qown[BZ];
  {
    const int y = it.y0 + ty, z0 = it.z0 + zb * BZ;
#pragma unroll
    for (int o = 0; o < BZ; o++)
      qown[o] = (y < L.n[1] && z0 + o < L.n[2]) ? src[((long long)it.x0 * L.n[1] + y) * L.n[2] + z0 + o] : 0.f;
  }
  float w6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int nsteps = 2 * Rx + 1;
  stage(L, it, 0, src, kpool, L.dk_off, 6, kcs, wpool, L.wh_off, sm_plane(smem, plane_sz, 0), sm_kslab(smem, plane_sz, kslab_sz, 0), sm_wsl(smem, plane_sz, kslab_sz, wsl_sz, 0), stride);
  for (int step = 0; step < nsteps; step++) {
    cp_async_wait_all();
    __syncthreads();
    const int b = step & 1;
    if (step + 1 < nsteps)
      stage(L, it, step + 1, src, kpool, L.dk_off, 6, kcs, wpool, L.wh_off, sm_plane(smem, plane_sz, b ^ 1),
            sm_kslab(smem, plane_sz, kslab_sz, b ^ 1), sm_wsl(smem, plane_sz, kslab_sz, wsl_sz, b ^ 1), stride);
    const float* plane = sm_plane(smem, plane_sz, b);
    const float* kslab = sm_kslab(smem, plane_sz, kslab_sz, b);
    const int* wsl = sm_wsl(smem, plane_sz, kslab_sz, wsl_sz, b);
    for (int dy = -Ry; dy <= Ry; dy++) {
      const int w = wsl[dy + Ry];
      if (w < 0) continue;
      const float* qrow = plane + (ty - dy + Ry) * stride + zb * BZ + Rz;
      const float* kc = kslab + (dy + Ry) * (2 * Rz + 1) + Rz;
      Col<0, WMAX>::virial(w, w6, qown, qrow, kc, ksz);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 6; c++) {
    double v = -0.5 * (double)L.scale * (double)w6[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int w = 0; w < NT / 32; w++) v += red[w][threadIdx.x];
    part[6 * (long long)blockIdx.x + threadIdx.x] = v;
  }
}

// ------------------------------------------------------------------ boxes
__global__ void __launch_bounds__(kBoxChunk) k_stencil_box(const LevDev* __restrict__ levs,
                                                           const RangeItem* __restrict__ items,
                                                           const float* __restrict__ kpool,
                                                           float* __restrict__ grid) {
  RangeItem it = items[blockIdx.x];
  if ((int)threadIdx.x >= it.count) return;
  const LevDev& L = levs[it.lev];
  int idx = it.start + threadIdx.x;
  int m[3] = {idx / (L.n[1] * L.n[2]), (idx / L.n[2]) % L.n[1], idx % L.n[2]};
  const float* q = grid + L.q_off;
  const float* K = kpool + L.k_off;
  float acc = 0.f;
  for (int a = 0; a < L.bsz[0]; a++) {
    int sx = m[0] - (a + L.blo[0]);
    if (L.per[0]) sx = wrap_s(sx, L.n[0]);
    else if (sx < 0 || sx >= L.n[0]) continue;
    for (int b = 0; b < L.bsz[1]; b++) {
      int sy = m[1] - (b + L.blo[1]);
      if (L.per[1]) sy = wrap_s(sy, L.n[1]);
      else if (sy < 0 || sy >= L.n[1]) continue;
      const float* krow = K + ((long long)a * L.bsz[1] + b) * L.bsz[2];
      const float* qrow = q + ((long long)sx * L.n[1] + sy) * L.n[2];
      for (int c = 0; c < L.bsz[2]; c++) {
        int sz = m[2] - (c + L.blo[2]);
        if (L.per[2]) sz = wrap_s(sz, L.n[2]);
        else if (sz < 0 || sz >= L.n[2]) continue;
        acc = fmaf(__ldg(krow + c), qrow[sz], acc);
      }
    }
  }
  grid[L.e_off + idx] = acc * L.scale;
}

__global__ void __launch_bounds__(kBoxChunk) k_virial_box(const LevDev* __restrict__ levs,
                                                          const RangeItem* __restrict__ items,
                                                          const float* __restrict__ kpool,
                                                          const float* __restrict__ grid,
                                                          double* __restrict__ part) {
  __shared__ double red[kBoxChunk / 32][6];
  RangeItem it = items[blockIdx.x];
  const LevDev& L = levs[it.lev];
  float w6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if ((int)threadIdx.x < it.count) {
    int idx = it.start + threadIdx.x;
    int m[3] = {idx / (L.n[1] * L.n[2]), (idx / L.n[2]) % L.n[1], idx % L.n[2]};
    const float* q = grid + L.q_off;
    const float qm = q[idx];
    const long long cs = (long long)L.bsz[0] * L.bsz[1] * L.bsz[2];
    const float* K = kpool + L.dk_off;
    for (int a = 0; a < L.bsz[0]; a++) {
      int sx = m[0] - (a + L.blo[0]);
      if (L.per[0]) sx = wrap_s(sx, L.n[0]);
      else if (sx < 0 || sx >= L.n[0]) continue;
      for (int b = 0; b < L.bsz[1]; b++) {
        int sy = m[1] - (b + L.blo[1]);
        if (L.per[1]) sy = wrap_s(sy, L.n[1]);
        else if (sy < 0 || sy >= L.n[1]) continue;
        const long long kr = ((long long)a * L.bsz[1] + b) * L.bsz[2];
        const float* qrow = q + ((long long)sx * L.n[1] + sy) * L.n[2];
        for (int c = 0; c < L.bsz[2]; c++) {
          int sz = m[2] - (c + L.blo[2]);
          if (L.per[2]) sz = wrap_s(sz, L.n[2]);
          else if (sz < 0 || sz >= L.n[2]) continue;
          float cq = qm * qrow[sz];
#pragma unroll
          for (int k = 0; k < 6; k++) w6[k] = fmaf(__ldg(K + k * cs + kr + c), cq, w6[k]);
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 6; c++) {
    double v = -0.5 * (double)L.scale * (double)w6[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int w = 0; w < kBoxChunk / 32; w++) v += red[w][threadIdx.x];
    part[6 * (long long)blockIdx.x + threadIdx.x] = v;
  }
}

// ------------------------------------------------------------------ launchers
static void ball_smem(int ryz_max[2], int ncomp, int& plane_sz, int& kslab_sz, int& wsl_sz, int& stride,
                      size_t& bytes) {
  const int Ry = ryz_max[0], Rz = ryz_max[1];
  stride = (TZ + 2 * Rz) | 1;
  plane_sz = (TY + 2 * Ry) * stride;
  kslab_sz = ncomp * (2 * Ry + 1) * (2 * Rz + 1);
  wsl_sz = 2 * Ry + 1;
  bytes = sizeof(float) * (2 * (size_t)plane_sz + 2 * (size_t)kslab_sz) + sizeof(int) * 2 * (size_t)wsl_sz;
}

template <int WMAX>
static void run_ball(const Work& w, const Tables& t, const TileItem* items, int nitems, int ryz_max[2],
                     cudaStream_t s) {
  int plane_sz, kslab_sz, wsl_sz, stride;
  size_t bytes;
  ball_smem(ryz_max, 1, plane_sz, kslab_sz, wsl_sz, stride, bytes);
  cudaFuncSetAttribute(k_stencil_ball<WMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  k_stencil_ball<WMAX><<<nitems, NT, bytes, s>>>(t.lev, items, t.kpool, t.wpool, w.grid, plane_sz, kslab_sz, wsl_sz,
                                                 stride);
}

template <int WMAX>
static void run_virial_ball(const Work& w, const Tables& t, const TileItem* items, int nitems, int ryz_max[2],
                            int part_off, cudaStream_t s) {
  int plane_sz, kslab_sz, wsl_sz, stride;
  size_t bytes;
  ball_smem(ryz_max, 6, plane_sz, kslab_sz, wsl_sz, stride, bytes);
  cudaFuncSetAttribute(k_virial_ball<WMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  k_virial_ball<WMAX><<<nitems, NT, bytes, s>>>(t.lev, items, t.kpool, t.wpool, w.grid,
                                                w.part_wg + 6 * (long long)part_off, plane_sz, kslab_sz, wsl_sz,
                                                stride);
}

void launch_stencil_ball(const Work& w, const Tables& t, const TileItem* items, int nitems, int rmax,
                         int ryz_max[2], cudaStream_t s) {
  if (nitems <= 0) return;
  if (rmax <= 8) run_ball<8>(w, t, items, nitems, ryz_max, s);
  else if (rmax <= 12) run_ball<12>(w, t, items, nitems, ryz_max, s);
  else if (rmax <= 16) run_ball<16>(w, t, items, nitems, ryz_max, s);
  else run_ball<24>(w, t, items, nitems, ryz_max, s);
}

void launch_virial_ball(const Work& w, const Tables& t, const TileItem* items, int nitems, int rmax,
                        int ryz_max[2], int part_off, cudaStream_t s) {
  if (nitems <= 0) return;
  if (rmax <= 8) run_virial_ball<8>(w, t, items, nitems, ryz_max, part_off, s);
  else if (rmax <= 12) run_virial_ball<12>(w, t, items, nitems, ryz_max, part_off, s);
  else if (rmax <= 16) run_virial_ball<16>(w, t, items, nitems, ryz_max, part_off, s);
  else run_virial_ball<24>(w, t, items, nitems, ryz_max, part_off, s);
}

void launch_stencil_box(const Work& w, const Tables& t, const RangeItem* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return;
  k_stencil_box<<<nitems, kBoxChunk, 0, s>>>(t.lev, items, t.kpool, w.grid);
}

void launch_virial_box(const Work& w, const Tables& t, const RangeItem* items, int nitems, int part_off,
                       cudaStream_t s) {
  if (nitems <= 0) return;
  k_virial_box<<<nitems, kBoxChunk, 0, s>>>(t.lev, items, t.kpool, w.grid, w.part_wg + 6 * (long long)part_off);
}

}  // namespace msm
