// k_stencil.cu -- the per-level grid-to-grid kernel sum of the MSM,
// e^l_m = sum_d K^l_d q~^l_(m-d) (Eq. action_of_K_as_convolution), and the
// grid part of the virial, W = -1/2 sum_l sum_d (dK^l/d eps)_d C^l_d with the
// autocorrelation C^l_d = sum_m q~^l_m q~^l_(m-d).
//
// Ball levels (support a ball of radius R that does not overlap itself under
// the periodic wrap). Since K^l = omega'^3 * s^l with s^l the raw samples of
// k_l on the grid (Eq. kernel_stencil_by_conv_with_universal_coeff), the ball
// kernels compute e^l = s^l * (omega'^3 * q~^l): the samples have a smaller
// ball (|h o n| < 2a, about two thirds of K's nonzeros) and the 3-tap-per-axis
// prefilter is fused into a pad kernel that writes a halo-padded copy of the
// prefiltered grid (periodic images or zeros in the halo), so every tile's
// input box is a plain rectangle. The samples are even in x and in y, so one
// block per output tile of 1 x 32 x 32 points streams the input x-planes in
// mirrored pairs x0 - dx, x0 + dx (dx = 0 .. R; 16-byte cp.async rows, one
// stage buffer: the block waits for each pair, and twice as many resident
// blocks as with double buffering hide the copies; measured faster) together
// with the stencil x-slab of +dx, stored column by column
// with dz aligned to 16 bytes. Each thread owns 16 consecutive z outputs in
// registers; per column (dx, dy >= 0) of half-width w it sums the 16 + 2w
// windows of the 1, 2 or 4 rows (x0 -+ dx, y -+ dy) that share the column,
// loads the 2w + 1 stencil values with 128-bit shared loads and issues
// 16 (2w + 1) FFMA from registers: a quarter of the FMAs of the plain sum.
// w (rounded up to an even value by the planner) selects an unrolled variant,
// so the ball shape costs little for short columns and nothing for empty ones.
// The arithmetic is FP32 on the CUDA cores: the sum has no dense
// reduction axis, and a Toeplitz recast for the tensor cores would multiply
// the work by (16 + 2R)/(2R + 1) per axis while TF32 loses the accuracy the
// method needs.
//
// The ball virial kernel is the same loop with the roles swapped: per column a
// thread forms its partial C'_(dx,dy,dz) = sum_m q~_m q'_(m-d) for the 2w + 1 dz
// values and at once contracts it with the six strain-derivative samples
// (q~^T dK q~ = sum_d ds_d C'_d for dK = omega'^3 * ds; stored with the
// half-space symmetry C'_d = C'_-d folded in). With raw samples the six
// factor through one weight column (ds_ab = g v_a v_b, v = h o d), so the
// contraction takes three dz moments of g C' per column.
//
// Box levels (small periodic levels whose stencil wraps onto itself, folded
// onto the grid, and the top level of open systems): one warp per output, the
// lanes splitting the stencil entries, then a shuffle reduction.
#include "msm_internal.h"

namespace msm {

constexpr int BZ = kBallBZ;
constexpr int TY = kBallTY;
constexpr int TZ = kBallTZ;
constexpr int NT = kBallThreads;
constexpr int kWslMax = 64;  // column table entries per stage buffer (2 R_y + 1 <= 49)

__device__ __forceinline__ int wrap_s(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ------------------------------------------------------------------ halo padding
// Halo-padded copy of the omega'-prefiltered grid, q'_m = sum_t omega'_tx
// omega'_ty omega'_tz q~_(m-t) (periodic axes wrap, open axes read zeros outside
// the grid). The ball kernels apply the raw kernel samples s to q', which equals
// K * q~ since K = omega'^3 * s (Eq. kernel_stencil_by_conv_with_universal_coeff)
// and convolution is associative.
// index of grid point c along an axis of n points: periodic axes wrap (the
// halo may reach past one period on small grids), open axes give -1 outside
__device__ __forceinline__ int pad_axis(int c, int n, int per) {
  if (per) {
    while (c < 0) c += n;
    while (c >= n) c -= n;
    return c;
  }
  return (c >= 0 && c < n) ? c : -1;
}

// One block per tile of kPadTX x-planes x kPadTY rows x kPadTZ columns of
// the padded grid, one thread per (row, column). The block walks the source
// x-planes the tile needs: it stages the plane's (rows +- r) x (columns +- r)
// patch in shared memory (wrapped or zero source indices, fixed per tile),
// applies the (2r+1)^2 y-z taps, and keeps the last 2r+1 filtered planes in
// registers for the x taps. r = 0 (no prefilter) makes it a halo copy.
template <int PR>
__global__ void __launch_bounds__(kPadTY * kPadTZ) k_pad(const SysDev* __restrict__ sys,
                                                         const LevDev* __restrict__ levs,
                                                         const TileItem* __restrict__ items, float* __restrict__ grid) {
  constexpr int NT = kPadTY * kPadTZ;
  constexpr int PW = kPadTZ + 2 * PR;
  constexpr int NE = (kPadTY + 2 * PR) * PW;
  constexpr int NL = (NE + NT - 1) / NT;
  __shared__ float patch[NE];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = levs[it.lev];
  const SysDev& S = sys[L.sys];
  const int tz = threadIdx.x % kPadTZ, ty = threadIdx.x / kPadTZ;
  const int py = it.y0 + ty, pz = it.z0 + tz;
  const bool own = py < L.pn[1] && pz < L.pn[2];
  float om[PR + 1];
#pragma unroll
  for (int k = 0; k <= PR; k++) om[k] = S.om[k];
  // in-plane source offset of each patch element this thread stages (-1: zero)
  int soff[NL];
#pragma unroll
  for (int u = 0; u < NL; u++) {
    const int e = threadIdx.x + u * NT;
    soff[u] = -1;
    if (e < NE) {
      const int sy = pad_axis(it.y0 + e / PW - PR - L.R[1], L.n[1], L.per[1]);
      const int sz = pad_axis(it.z0 + e % PW - PR - L.hz, L.n[2], L.per[2]);
      if (sy >= 0 && sz >= 0) soff[u] = sy * L.n[2] + sz;
    }
  }
  const float* q = grid + L.q_off;
  const long long plane = (long long)L.n[1] * L.n[2];
  float g[2 * PR + 1];
#pragma unroll
  for (int k = 0; k <= 2 * PR; k++) g[k] = 0.f;
  const int xend = min(it.x0 + kPadTX, L.pn[0]);
  // source plane xs feeds outputs px = xs + Rx - PR .. xs + Rx + PR
  for (int xs = it.x0 - L.R[0] - PR, step = 0; xs <= xend - 1 - L.R[0] + PR; xs++, step++) {
    const int sx = pad_axis(xs, L.n[0], L.per[0]);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NL; u++) {
      const int e = threadIdx.x + u * NT;
      if (e < NE) patch[e] = (sx >= 0 && soff[u] >= 0) ? __ldg(q + sx * plane + soff[u]) : 0.f;
    }
    __syncthreads();
    float v = 0.f;
#pragma unroll
    for (int a = 0; a <= 2 * PR; a++) {
      float row = 0.f;
#pragma unroll
      for (int b = 0; b <= 2 * PR; b++) row = fmaf(om[b < PR ? PR - b : b - PR], patch[(ty + a) * PW + tz + b], row);
      v = fmaf(om[a < PR ? PR - a : a - PR], row, v);
    }
#pragma unroll
    for (int k = 0; k < 2 * PR; k++) g[k] = g[k + 1];
    g[2 * PR] = v;
    if (step >= 2 * PR && own) {
      float o = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * PR; k++) o = fmaf(om[k < PR ? PR - k : k - PR], g[k], o);
      const int px = xs + L.R[0] - PR;
      grid[L.p_off + ((long long)px * L.pn[1] + py) * L.pn[2] + pz] = o;
    }
  }
}

// ------------------------------------------------------------------ columns
template <int W>
__device__ __forceinline__ void ball_column(float (&acc)[BZ], const float* __restrict__ qrow,
                                            const float* __restrict__ kc) {
  constexpr int A = (W + 3) & ~3;
  constexpr int NQ = BZ + 2 * A;
  constexpr int NK = 2 * A + 4;
  float qv[NQ], kv[NK];
#pragma unroll
  for (int t = 0; t < NQ; t += 4) {
    float4 v = *reinterpret_cast<const float4*>(qrow - A + t);
    qv[t] = v.x; qv[t + 1] = v.y; qv[t + 2] = v.z; qv[t + 3] = v.w;
  }
#pragma unroll
  for (int t = 0; t < 2 * A + 1; t += 4) {
    float4 v = *reinterpret_cast<const float4*>(kc - A + t);
    kv[t] = v.x; kv[t + 1] = v.y; kv[t + 2] = v.z; kv[t + 3] = v.w;
  }
#pragma unroll
  for (int dz = -W; dz <= W; dz++) {
    const float k = kv[dz + A];
#pragma unroll
    for (int o = 0; o < BZ; o++) acc[o] = fmaf(k, qv[o - dz + A], acc[o]);
  }
}

// The stencil is even in x and in y (its samples depend on |dx|, |dy|, |dz|),
// so the 2 or 4 input rows that share a column (x0 -+ dx, y -+ dy) are summed
// before the FMAs: nr = 1, 2 or 4 rows r[0..nr).
template <int W>
__device__ __forceinline__ void ball_column_sym(float (&acc)[BZ], const float* r0, const float* r1, const float* r2,
                                                const float* r3, int nr, const float* __restrict__ kc) {
  const float* r[4] = {r0, r1, r2, r3};
  constexpr int A = (W + 3) & ~3;
  constexpr int NQ = BZ + 2 * A;
  constexpr int NK = 2 * A + 4;
  float qv[NQ], kv[NK];
#pragma unroll
  for (int t = 0; t < NQ; t += 4) {
    float4 v = *reinterpret_cast<const float4*>(r[0] - A + t);
    qv[t] = v.x; qv[t + 1] = v.y; qv[t + 2] = v.z; qv[t + 3] = v.w;
  }
#pragma unroll
  for (int k = 1; k < 4; k++) {
    if (k < nr) {
#pragma unroll
      for (int t = 0; t < NQ; t += 4) {
        float4 v = *reinterpret_cast<const float4*>(r[k] - A + t);
        qv[t] += v.x; qv[t + 1] += v.y; qv[t + 2] += v.z; qv[t + 3] += v.w;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 2 * A + 1; t += 4) {
    float4 v = *reinterpret_cast<const float4*>(kc - A + t);
    kv[t] = v.x; kv[t + 1] = v.y; kv[t + 2] = v.z; kv[t + 3] = v.w;
  }
#pragma unroll
  for (int dz = -W; dz <= W; dz++) {
    const float k = kv[dz + A];
#pragma unroll
    for (int o = 0; o < BZ; o++) acc[o] = fmaf(k, qv[o - dz + A], acc[o]);
  }
}

template <int W>
__device__ __forceinline__ void virial_column(float (&w6)[6], const float (&qown)[BZ],
                                              const float* __restrict__ qrow, const float* __restrict__ kd,
                                              int kstride) {
  constexpr int A = (W + 3) & ~3;
  constexpr int NQ = BZ + 2 * A;
  float qv[NQ];
#pragma unroll
  for (int t = 0; t < NQ; t += 4) {
    float4 v = *reinterpret_cast<const float4*>(qrow - A + t);
    qv[t] = v.x; qv[t + 1] = v.y; qv[t + 2] = v.z; qv[t + 3] = v.w;
  }
  float c[2 * W + 1];
#pragma unroll
  for (int dz = -W; dz <= W; dz++) {
    float s = 0.f;
#pragma unroll
    for (int o = 0; o < BZ; o++) s = fmaf(qown[o], qv[o - dz + A], s);
    c[dz + W] = s;
  }
#pragma unroll
  for (int k = 0; k < 6; k++) {
    float kv[2 * A + 4];
#pragma unroll
    for (int t = 0; t < 2 * A + 1; t += 4) {
      float4 v = *reinterpret_cast<const float4*>(kd + k * kstride - A + t);
      kv[t] = v.x; kv[t + 1] = v.y; kv[t + 2] = v.z; kv[t + 3] = v.w;
    }
#pragma unroll
    for (int dz = -W; dz <= W; dz++) w6[k] = fmaf(kv[dz + A], c[dz + W], w6[k]);
  }
}

// p = 4 (raw samples): ds_ab(n) = g(n) (h_1 o n)_a (h_1 o n)_b, so one weight
// column g replaces the six and the contraction needs only the moments
// sum g C', sum g C' dz, sum g C' dz^2 of the column. cx = h_x dx, cy = h_y dy;
// w6[2], w6[4], w6[5] collect the dz moments without their h_z factors.
template <int W>
__device__ __forceinline__ void virial_column_fact(float (&w6)[6], const float (&qown)[BZ],
                                                   const float* __restrict__ qrow, const float* __restrict__ gd,
                                                   float cx, float cy) {
  constexpr int A = (W + 3) & ~3;
  constexpr int NQ = BZ + 2 * A;
  float qv[NQ], gv[2 * A + 4];
#pragma unroll
  for (int t = 0; t < NQ; t += 4) {
    float4 v = *reinterpret_cast<const float4*>(qrow - A + t);
    qv[t] = v.x; qv[t + 1] = v.y; qv[t + 2] = v.z; qv[t + 3] = v.w;
  }
#pragma unroll
  for (int t = 0; t < 2 * A + 1; t += 4) {
    float4 v = *reinterpret_cast<const float4*>(gd - A + t);
    gv[t] = v.x; gv[t + 1] = v.y; gv[t + 2] = v.z; gv[t + 3] = v.w;
  }
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int dz = -W; dz <= W; dz++) {
    float c = 0.f;
#pragma unroll
    for (int o = 0; o < BZ; o++) c = fmaf(qown[o], qv[o - dz + A], c);
    const float t = gv[dz + A] * c;
    s0 += t;
    s1 = fmaf(t, (float)dz, s1);
    s2 = fmaf(t, (float)(dz * dz), s2);
  }
  w6[0] = fmaf(cx * cx, s0, w6[0]);
  w6[1] = fmaf(cy * cy, s0, w6[1]);
  w6[2] += s2;
  w6[3] = fmaf(cx * cy, s0, w6[3]);
  w6[4] = fmaf(cx, s1, w6[4]);
  w6[5] = fmaf(cy, s1, w6[5]);
}

// dispatch on the (even) column half-width w
template <int W, int WMAX>
struct Col {
  static __device__ __forceinline__ void stencil(int w, float (&acc)[BZ], const float* q, const float* k) {
    if (w == W)
      ball_column<W>(acc, q, k);
    else
      Col<W + 2, WMAX>::stencil(w, acc, q, k);
  }
  static __device__ __forceinline__ void stencil_sym(int w, float (&acc)[BZ], const float* r0, const float* r1,
                                                     const float* r2, const float* r3, int nr, const float* k) {
    if (w == W)
      ball_column_sym<W>(acc, r0, r1, r2, r3, nr, k);
    else
      Col<W + 2, WMAX>::stencil_sym(w, acc, r0, r1, r2, r3, nr, k);
  }
  static __device__ __forceinline__ void virial(int w, float (&w6)[6], const float (&qown)[BZ], const float* q,
                                                const float* k, int ks) {
    if (w == W)
      virial_column<W>(w6, qown, q, k, ks);
    else
      Col<W + 2, WMAX>::virial(w, w6, qown, q, k, ks);
  }
  static __device__ __forceinline__ void virial_fact(int w, float (&w6)[6], const float (&qown)[BZ], const float* q,
                                                     const float* g, float cx, float cy) {
    if (w == W)
      virial_column_fact<W>(w6, qown, q, g, cx, cy);
    else
      Col<W + 2, WMAX>::virial_fact(w, w6, qown, q, g, cx, cy);
  }
};
template <int WMAX>
struct Col<WMAX, WMAX> {
  static __device__ __forceinline__ void stencil(int, float (&acc)[BZ], const float* q, const float* k) {
    ball_column<WMAX>(acc, q, k);
  }
  static __device__ __forceinline__ void stencil_sym(int, float (&acc)[BZ], const float* r0, const float* r1,
                                                     const float* r2, const float* r3, int nr, const float* k) {
    ball_column_sym<WMAX>(acc, r0, r1, r2, r3, nr, k);
  }
  static __device__ __forceinline__ void virial(int, float (&w6)[6], const float (&qown)[BZ], const float* q,
                                                const float* k, int ks) {
    virial_column<WMAX>(w6, qown, q, k, ks);
  }
  static __device__ __forceinline__ void virial_fact(int, float (&w6)[6], const float (&qown)[BZ], const float* q,
                                                     const float* g, float cx, float cy) {
    virial_column_fact<WMAX>(w6, qown, q, g, cx, cy);
  }
};

// ------------------------------------------------------------------ staging
// Copies of input plane x = x0 - dx of the padded grid (rows y0-Ry .. y0+TY-1+Ry,
// columns z0-hz .. z0+TZ-1+hz), of the nk stencil slabs of this dx and of its
// column table, into stage buffer b.
__device__ __forceinline__ void stage_ball(const LevDev& L, const TileItem& it, int step,
                                           const float* __restrict__ grid, const float* __restrict__ kpool,
                                           long long koff, int nk, const int* __restrict__ wpool, long long woff,
                                           float* plane, float* kslab, int* wsl, int stride) {
  const int Rx = L.R[0], Ry = L.R[1], hz = L.hz;
  const int rows = TY + 2 * Ry, cpr = (TZ + 2 * hz) / 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int px = it.x0 + 2 * Rx - step;  // padded index of x0 - dx, dx = step - Rx
  const float* src = grid + L.p_off + ((long long)px * L.pn[1] + it.y0) * L.pn[2] + it.z0;
  for (int r = warp; r < rows; r += NT / 32)
    if (lane < cpr) cp_async16(plane + r * stride + 4 * lane, src + (long long)r * L.pn[2] + 4 * lane);
  const int kchunks = nk * (2 * Ry + 1) * kSK(hz) / 4;
  const float* ks = kpool + koff + (long long)step * nk * (2 * Ry + 1) * kSK(hz);
  for (int e = threadIdx.x; e < kchunks; e += NT) cp_async16(kslab + 4 * e, ks + 4 * e);
  for (int e = threadIdx.x; e < 2 * Ry + 1; e += NT) wsl[e] = wpool[woff + (long long)step * (2 * Ry + 1) + e];
  cp_async_commit();
}

// Copies of input planes x0 - dx and x0 + dx (one plane for dx = 0) of the
// padded grid, of the stencil slab of +dx and of its column table, into one
// stage buffer.
__device__ __forceinline__ void stage_pair(const LevDev& L, const TileItem& it, int dx,
                                           const float* __restrict__ grid, const float* __restrict__ kpool,
                                           const int* __restrict__ wpool, float* planeA, float* planeB,
                                           float* kslab, int* wsl, int stride) {
  const int Rx = L.R[0], Ry = L.R[1], hz = L.hz;
  const int rows = TY + 2 * Ry, cpr = (TZ + 2 * hz) / 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int pl = 0; pl < (dx > 0 ? 2 : 1); pl++) {
    const int px = it.x0 + Rx + (pl == 0 ? -dx : dx);  // padded index of x0 -+ dx
    float* dst = pl == 0 ? planeA : planeB;
    const float* src = grid + L.p_off + ((long long)px * L.pn[1] + it.y0) * L.pn[2] + it.z0;
    for (int r = warp; r < rows; r += NT / 32)
      if (lane < cpr) cp_async16(dst + r * stride + 4 * lane, src + (long long)r * L.pn[2] + 4 * lane);
  }
  const int step = Rx + dx;
  const int kchunks = (2 * Ry + 1) * kSK(hz) / 4;
  const float* ks = kpool + L.k_off + (long long)step * (2 * Ry + 1) * kSK(hz);
  for (int e = threadIdx.x; e < kchunks; e += NT) cp_async16(kslab + 4 * e, ks + 4 * e);
  for (int e = threadIdx.x; e < 2 * Ry + 1; e += NT) wsl[e] = wpool[L.w_off + (long long)step * (2 * Ry + 1) + e];
  cp_async_commit();
}

template <int WMAX>
__global__ void __launch_bounds__(NT) k_stencil_ball(const LevDev* __restrict__ levs,
                                                     const TileItem* __restrict__ items,
                                                     const float* __restrict__ kpool, const int* __restrict__ wpool,
                                                     float* __restrict__ grid, int stride, int plane_sz, int kslab_sz) {
  extern __shared__ __align__(16) float smem[];
  float* planes = smem;                    // one stage buffer of 2 planes
  float* kslabs = smem + 2 * plane_sz;
  int* wsl = reinterpret_cast<int*>(kslabs + kslab_sz);
  const TileItem it = items[blockIdx.x];
  const LevDev& L = levs[it.lev];
  const int Rx = L.R[0], Ry = L.R[1], hz = L.hz, SK = kSK(hz);
  const int ty = threadIdx.x % TY, zb = threadIdx.x / TY;
  float acc[BZ];
#pragma unroll
  for (int o = 0; o < BZ; o++) acc[o] = 0.f;
  for (int dx = 0; dx <= Rx; dx++) {
    __syncthreads();
    stage_pair(L, it, dx, grid, kpool, wpool, planes, planes + plane_sz, kslabs, wsl, stride);
    cp_async_wait_all();
    __syncthreads();
    const float* pa = planes;
    const float* pb = pa + plane_sz;
    const float* kslab = kslabs;
    const int* wc = wsl;
    for (int dy = 0; dy <= Ry; dy++) {
      const int w = wc[dy + Ry];
      if (w < 0) continue;
      const int o1 = (ty - dy + Ry) * stride + zb * BZ + hz, o2 = (ty + dy + Ry) * stride + zb * BZ + hz;
      // rows sharing the column: (x0-dx, y-dy), (x0-dx, y+dy), (x0+dx, y-dy), (x0+dx, y+dy)
      const int nr = (dx > 0 ? 2 : 1) * (dy > 0 ? 2 : 1);
      const float* r1 = dy > 0 ? pa + o2 : pb + o1;
      Col<0, WMAX>::stencil_sym(w, acc, pa + o1, r1, pb + o1, pb + o2, nr, kslab + (dy + Ry) * SK + hz);
    }
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

// General ball (tilted cells, where the samples have only the point symmetry
// s(n) = s(-n)): every x-plane x0 - dx, dx = -R .. R, is staged in turn with
// the stencil x-slab of that dx, and every column (dx, dy) applies its
// samples on dz in [c - w, c + w] about the column's centre c (a multiple of
// 4, so the shifted 16-byte row loads stay aligned; the halo hz covers
// |c| + w). Same per-thread register blocking as the symmetric kernel, with
// no mirrored rows to fold: 16 (2w + 1) FMA per column and output tile row.
template <int WMAX>
__global__ void __launch_bounds__(NT) k_stencil_gen(const LevDev* __restrict__ levs, const TileItem* __restrict__ items,
                                                    const float* __restrict__ kpool, const int* __restrict__ wpool,
                                                    float* __restrict__ grid, int stride, int plane_sz, int kslab_sz) {
  extern __shared__ __align__(16) float smem[];
  float* plane = smem;
  float* kslab = smem + plane_sz;
  int* wsl = reinterpret_cast<int*>(kslab + kslab_sz);
  const TileItem it = items[blockIdx.x];
  const LevDev& L = levs[it.lev];
  const int Rx = L.R[0], Ry = L.R[1], hz = L.hz, SK = kSK(hz);
  const int ty = threadIdx.x % TY, zb = threadIdx.x / TY;
  float acc[BZ];
#pragma unroll
  for (int o = 0; o < BZ; o++) acc[o] = 0.f;
  for (int step = 0; step <= 2 * Rx; step++) {
    __syncthreads();
    stage_ball(L, it, step, grid, kpool, L.k_off, 1, wpool, L.w_off, plane, kslab, wsl, stride);
    cp_async_wait_all();
    __syncthreads();
    const int* cen = wpool + L.c_off + (long long)step * (2 * Ry + 1);
    for (int dy = -Ry; dy <= Ry; dy++) {
      const int w = wsl[dy + Ry];
      if (w < 0) continue;
      const int c = __ldg(cen + dy + Ry);
      const float* qrow = plane + (ty - dy + Ry) * stride + zb * BZ + hz - c;
      Col<0, WMAX>::stencil(w, acc, qrow, kslab + (dy + Ry) * SK + hz);
    }
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

template <int WMAX, bool FACT, bool GEN = false>
__global__ void __launch_bounds__(NT) k_virial_ball(const SysDev* __restrict__ sys, const LevDev* __restrict__ levs,
                                                    const TileItem* __restrict__ items,
                                                    const float* __restrict__ kpool, const int* __restrict__ wpool,
                                                    const float* __restrict__ grid, double* __restrict__ part,
                                                    int stride, int plane_sz, int kslab_sz) {
  extern __shared__ __align__(16) float smem[];
  __shared__ double red[NT / 32][6];
  float* planes = smem;
  float* kslabs = smem + plane_sz;
  int* wsl = reinterpret_cast<int*>(kslabs + kslab_sz);
  const TileItem it = items[blockIdx.x];
  const LevDev& L = levs[it.lev];
  const int Rx = L.R[0], Ry = L.R[1], hz = L.hz, SK = kSK(hz);
  const int ty = threadIdx.x % TY, zb = threadIdx.x / TY;
  const int kstride = (2 * Ry + 1) * SK;
  constexpr int NK = FACT ? 1 : 6;
  float hx = 0.f, hy = 0.f, hzs = 0.f;
  if (FACT) {
    const SysDev& S = sys[L.sys];
    hx = S.h1f[0];
    hy = S.h1f[1];
    hzs = S.h1f[2];
  }
  float qown[BZ];  // raw q~ at this thread's points (the window below reads the prefiltered q')
  {
    const int y = it.y0 + ty, z0 = it.z0 + zb * BZ;
    const float* row = grid + L.q_off + ((long long)it.x0 * L.n[1] + y) * L.n[2];
#pragma unroll
    for (int o = 0; o < BZ; o++) qown[o] = (y < L.n[1] && z0 + o < L.n[2]) ? row[z0 + o] : 0.f;
  }
  float w6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  // the half-space weights vanish for dx < 0: walk the planes dx = 0 .. Rx only
  const int nsteps = 2 * Rx + 1;
  for (int step = Rx; step < nsteps; step++) {
    __syncthreads();
    stage_ball(L, it, step, grid, kpool, L.dk_off, NK, wpool, L.wh_off, planes, kslabs, wsl, stride);
    cp_async_wait_all();
    __syncthreads();
    const float* plane = planes;
    const float* kslab = kslabs;
    const int* wc = wsl;
    const float cx = hx * (float)(step - Rx);
    const int* cen = GEN ? wpool + L.c_off + (long long)step * (2 * Ry + 1) : nullptr;
    for (int dy = -Ry; dy <= Ry; dy++) {
      const int w = wc[dy + Ry];
      if (w < 0) continue;
      const int c = GEN ? __ldg(cen + dy + Ry) : 0;  // column centre (tilted cells)
      const float* qrow = plane + (ty - dy + Ry) * stride + zb * BZ + hz - c;
      const float* kd = kslab + (dy + Ry) * SK + hz;
      if (FACT)
        Col<0, WMAX>::virial_fact(w, w6, qown, qrow, kd, cx, hy * (float)dy);
      else
        Col<0, WMAX>::virial(w, w6, qown, qrow, kd, kstride);
    }
  }
  if (FACT) {
    w6[2] *= hzs * hzs;
    w6[4] *= hzs;
    w6[5] *= hzs;
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
// Batch plans, levels of at most kBoxStage points (the folded small levels and
// the open top levels): one block stages the whole level in shared memory and
// each thread sums the box for one output point. Single-system plans and larger
// levels: one warp per output point; the lanes split the box entries t
// (coalesced stencil loads), then a shuffle reduction.

struct BoxIter {
  int a, b, c;
  __device__ __forceinline__ void init(int t, const LevDev& L) {
    c = t % L.bsz[2];
    b = (t / L.bsz[2]) % L.bsz[1];
    a = t / (L.bsz[2] * L.bsz[1]);
  }
  __device__ __forceinline__ void advance32(const LevDev& L) {
    c += 32;
    while (c >= L.bsz[2]) {
      c -= L.bsz[2];
      if (++b >= L.bsz[1]) {
        b = 0;
        ++a;
      }
    }
  }
};

// storage index of q_(m - d) or -1 (open axis, outside)
__device__ __forceinline__ int box_src(const LevDev& L, const int m[3], const BoxIter& t) {
  int s[3] = {m[0] - (t.a + L.blo[0]), m[1] - (t.b + L.blo[1]), m[2] - (t.c + L.blo[2])};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    if (L.per[d]) s[d] &= (L.n[d] - 1);  // periodic level sizes are powers of two
    else if (s[d] < 0 || s[d] >= L.n[d]) return -1;
  }
  return (s[0] * L.n[1] + s[1]) * L.n[2] + s[2];
}

// storage index of q_(m - d) along one axis of a box level, d = e + blo, or -1
// (open axis, outside); periodic level sizes are powers of two
__device__ __forceinline__ int box_axis(const LevDev& L, int d, int m, int e) {
  const int s = m - (e + L.blo[d]);
  if (L.per[d]) return s & (L.n[d] - 1);
  return (s >= 0 && s < L.n[d]) ? s : -1;
}

__global__ void __launch_bounds__(kBoxThreads) k_stencil_box(const LevDev* __restrict__ levs,
                                                             const RangeItem* __restrict__ items,
                                                             const float* __restrict__ kpool,
                                                             float* __restrict__ grid) {
  __shared__ float qs[kBoxStage];
  const RangeItem it = items[blockIdx.x];
  const LevDev& L = levs[it.lev];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nt = L.bsz[0] * L.bsz[1] * L.bsz[2];
  const int npts = L.n[0] * L.n[1] * L.n[2];
  const float* q = grid + L.q_off;
  const float* K = kpool + L.k_off;
  if (L.box_tile) {
    // the whole level in shared memory, one output per thread; the lanes of a
    // warp read the same stencil entry (one broadcast load)
    for (int e = threadIdx.x; e < npts; e += kBoxThreads) qs[e] = q[e];
    __syncthreads();
    if ((int)threadIdx.x >= it.count) return;
    const int idx = it.start + threadIdx.x;
    const int m[3] = {idx / (L.n[1] * L.n[2]), (idx / L.n[2]) % L.n[1], idx % L.n[2]};
    // nested sums (row, plane, box) keep the rounding of each at a few dozen terms
    float acc = 0.f;
    for (int a = 0; a < L.bsz[0]; a++) {
      const int sx = box_axis(L, 0, m[0], a);
      if (sx < 0) continue;
      float pl = 0.f;
      for (int b = 0; b < L.bsz[1]; b++) {
        const int sy = box_axis(L, 1, m[1], b);
        if (sy < 0) continue;
        const float* qr = qs + (sx * L.n[1] + sy) * L.n[2];
        const float* kr = K + (a * L.bsz[1] + b) * L.bsz[2];
        float row = 0.f;
        for (int c = 0; c < L.bsz[2]; c++) {
          const int sz = box_axis(L, 2, m[2], c);
          if (sz >= 0) row = fmaf(__ldg(kr + c), qr[sz], row);
        }
        pl += row;
      }
      acc += pl;
    }
    grid[L.e_off + idx] = acc * L.scale;
    return;
  }
  for (int o = warp; o < it.count; o += kBoxThreads / 32) {
    const int idx = it.start + o;
    const int m[3] = {idx / (L.n[1] * L.n[2]), (idx / L.n[2]) % L.n[1], idx % L.n[2]};
    float acc = 0.f;
    BoxIter ti;
    ti.init(lane, L);
    for (int t = lane; t < nt; t += 32) {
      int s = box_src(L, m, ti);
      if (s >= 0) acc = fmaf(__ldg(K + t), q[s], acc);
      ti.advance32(L);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) grid[L.e_off + idx] = acc * L.scale;
  }
}

__global__ void __launch_bounds__(kBoxThreads) k_virial_box(const LevDev* __restrict__ levs,
                                                            const RangeItem* __restrict__ items,
                                                            const float* __restrict__ kpool,
                                                            const float* __restrict__ grid,
                                                            double* __restrict__ part) {
  __shared__ double red[kBoxThreads / 32][6];
  __shared__ float qs[kBoxStage];
  const RangeItem it = items[blockIdx.x];
  const LevDev& L = levs[it.lev];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nt = L.bsz[0] * L.bsz[1] * L.bsz[2];
  const int npts = L.n[0] * L.n[1] * L.n[2];
  const float* q = grid + L.q_off;
  const float* K = kpool + L.dk_off;
  float w6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (L.box_tile) {
    // the whole level in shared memory, one point m per thread:
    // w6 += q_m sum_d dK_d q_(m - d)
    for (int e = threadIdx.x; e < npts; e += kBoxThreads) qs[e] = q[e];
    __syncthreads();
    if ((int)threadIdx.x < it.count) {
      const int idx = it.start + threadIdx.x;
      const int m[3] = {idx / (L.n[1] * L.n[2]), (idx / L.n[2]) % L.n[1], idx % L.n[2]};
      const float qm = qs[idx];
      // nested sums (row, plane, box) as in the stencil
      for (int a = 0; a < L.bsz[0]; a++) {
        const int sx = box_axis(L, 0, m[0], a);
        if (sx < 0) continue;
        float pl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int b = 0; b < L.bsz[1]; b++) {
          const int sy = box_axis(L, 1, m[1], b);
          if (sy < 0) continue;
          const float* qr = qs + (sx * L.n[1] + sy) * L.n[2];
          const int t0 = (a * L.bsz[1] + b) * L.bsz[2];
          float row[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          for (int c = 0; c < L.bsz[2]; c++) {
            const int sz = box_axis(L, 2, m[2], c);
            if (sz < 0) continue;
            const float cq = qm * qr[sz];
            const float4 k0 = __ldg(reinterpret_cast<const float4*>(K + 8 * (long long)(t0 + c)));
            const float4 k1 = __ldg(reinterpret_cast<const float4*>(K + 8 * (long long)(t0 + c) + 4));
            row[0] = fmaf(k0.x, cq, row[0]);
            row[1] = fmaf(k0.y, cq, row[1]);
            row[2] = fmaf(k0.z, cq, row[2]);
            row[3] = fmaf(k0.w, cq, row[3]);
            row[4] = fmaf(k1.x, cq, row[4]);
            row[5] = fmaf(k1.y, cq, row[5]);
          }
#pragma unroll
          for (int k = 0; k < 6; k++) pl[k] += row[k];
        }
#pragma unroll
        for (int k = 0; k < 6; k++) w6[k] += pl[k];
      }
    }
  } else {
    for (int o = warp; o < it.count; o += kBoxThreads / 32) {
      const int idx = it.start + o;
      const int m[3] = {idx / (L.n[1] * L.n[2]), (idx / L.n[2]) % L.n[1], idx % L.n[2]};
      const float qm = q[idx];
      BoxIter ti;
      ti.init(lane, L);
      for (int t = lane; t < nt; t += 32) {
        int s = box_src(L, m, ti);
        if (s >= 0) {
          const float cq = qm * q[s];
#pragma unroll
          for (int k = 0; k < 6; k++) w6[k] = fmaf(__ldg(K + 8 * (long long)t + k), cq, w6[k]);
        }
        ti.advance32(L);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 6; c++) {
    double v = -0.5 * (double)L.scale * (double)w6[c];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int w = 0; w < kBoxThreads / 32; w++) v += red[w][threadIdx.x];
    part[6 * (long long)blockIdx.x + threadIdx.x] = v;
  }
}

// ------------------------------------------------------------------ launchers
// shared memory of one ball block: nplanes staged input planes, the stencil
// slabs of one dx (nk arrays) and its column table (one stage buffer)
static void ball_smem(const int ryz_max[2], int nk, int nplanes, int& stride, int& plane_sz, int& kslab_sz,
                      size_t& bytes) {
  const int Ry = ryz_max[0], hz = ryz_max[1];
  stride = TZ + 2 * hz;
  if ((stride / 4) % 2 == 0) stride += 4;  // 4 x odd floats: conflict-free 128-bit row loads
  plane_sz = (TY + 2 * Ry) * stride;
  kslab_sz = nk * (2 * Ry + 1) * kSK(hz);
  bytes = sizeof(float) * ((size_t)nplanes * plane_sz + (size_t)kslab_sz) + sizeof(int) * kWslMax;
}

template <int WMAX>
static void run_ball(const Work& w, const Tables& t, const TileItem* items, int nitems, int ryz_max[2],
                     cudaStream_t s) {
  int stride, plane_sz, kslab_sz;
  size_t bytes;
  ball_smem(ryz_max, 1, 2, stride, plane_sz, kslab_sz, bytes);  // planes x0 - dx, x0 + dx
  static size_t attr = 0;  // raise the dynamic shared-memory limit once per size
  if (bytes > attr && cudaFuncSetAttribute(k_stencil_ball<WMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)bytes) == cudaSuccess)
    attr = bytes;
  k_stencil_ball<WMAX><<<nitems, NT, bytes, s>>>(t.lev, items, t.kpool, t.wpool, w.grid, stride, plane_sz,
                                                 kslab_sz);
}

template <int WMAX, bool FACT, bool GEN>
static void run_virial_ball(const Work& w, const Tables& t, const TileItem* items, int nitems, int ryz_max[2],
                            int part_off, cudaStream_t s) {
  int stride, plane_sz, kslab_sz;
  size_t bytes;
  ball_smem(ryz_max, FACT ? 1 : 6, 1, stride, plane_sz, kslab_sz, bytes);
  static size_t attr = 0;
  if (bytes > attr && cudaFuncSetAttribute(k_virial_ball<WMAX, FACT, GEN>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
    attr = bytes;
  k_virial_ball<WMAX, FACT, GEN><<<nitems, NT, bytes, s>>>(t.sys, t.lev, items, t.kpool, t.wpool, w.grid,
                                                           w.part_wg + 6 * (long long)part_off, stride, plane_sz,
                                                           kslab_sz);
}

template <bool FACT, bool GEN>
static void dispatch_virial_ball(const Work& w, const Tables& t, const TileItem* items, int nitems, int rmax,
                                 int ryz_max[2], int part_off, cudaStream_t s) {
  if (rmax <= 8) run_virial_ball<8, FACT, GEN>(w, t, items, nitems, ryz_max, part_off, s);
  else if (rmax <= 12) run_virial_ball<12, FACT, GEN>(w, t, items, nitems, ryz_max, part_off, s);
  else if (rmax <= 16) run_virial_ball<16, FACT, GEN>(w, t, items, nitems, ryz_max, part_off, s);
  else run_virial_ball<24, FACT, GEN>(w, t, items, nitems, ryz_max, part_off, s);
}

template <int WMAX>
static void run_gen(const Work& w, const Tables& t, const TileItem* items, int nitems, int ryz_max[2],
                    cudaStream_t s) {
  int stride, plane_sz, kslab_sz;
  size_t bytes;
  ball_smem(ryz_max, 1, 1, stride, plane_sz, kslab_sz, bytes);
  static size_t attr = 0;
  if (bytes > attr && cudaFuncSetAttribute(k_stencil_gen<WMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)bytes) == cudaSuccess)
    attr = bytes;
  k_stencil_gen<WMAX><<<nitems, NT, bytes, s>>>(t.lev, items, t.kpool, t.wpool, w.grid, stride, plane_sz, kslab_sz);
}

void launch_pad(const Work& w, const Tables& t, const TileItem* items, int nitems, int pre_r, cudaStream_t s) {
  if (nitems <= 0) return;
  if (pre_r == 1) k_pad<1><<<nitems, kPadTY * kPadTZ, 0, s>>>(t.sys, t.lev, items, w.grid);
  else k_pad<0><<<nitems, kPadTY * kPadTZ, 0, s>>>(t.sys, t.lev, items, w.grid);
}

// ryz_max = {largest R_y, largest halo hz} over the ball levels; rmax = largest R_z
void launch_stencil_ball(const Work& w, const Tables& t, const TileItem* items, int nitems, int rmax,
                         int ryz_max[2], bool general, cudaStream_t s) {
  if (nitems <= 0) return;
  if (general) {  // tilted cells: shifted, non-symmetric columns
    if (rmax <= 8) run_gen<8>(w, t, items, nitems, ryz_max, s);
    else if (rmax <= 12) run_gen<12>(w, t, items, nitems, ryz_max, s);
    else if (rmax <= 16) run_gen<16>(w, t, items, nitems, ryz_max, s);
    else run_gen<24>(w, t, items, nitems, ryz_max, s);
    return;
  }
  if (rmax <= 8) run_ball<8>(w, t, items, nitems, ryz_max, s);
  else if (rmax <= 12) run_ball<12>(w, t, items, nitems, ryz_max, s);
  else if (rmax <= 16) run_ball<16>(w, t, items, nitems, ryz_max, s);
  else run_ball<24>(w, t, items, nitems, ryz_max, s);
}

// factorized: the ball tables hold raw samples (p = 4) with the one-column
// virial weights g
void launch_virial_ball(const Work& w, const Tables& t, const TileItem* items, int nitems, int rmax,
                        int ryz_max[2], int part_off, bool factorized, bool general, cudaStream_t s) {
  if (nitems <= 0) return;
  if (factorized) dispatch_virial_ball<true, false>(w, t, items, nitems, rmax, ryz_max, part_off, s);
  else if (general) dispatch_virial_ball<false, true>(w, t, items, nitems, rmax, ryz_max, part_off, s);
  else dispatch_virial_ball<false, false>(w, t, items, nitems, rmax, ryz_max, part_off, s);
}

void launch_stencil_box(const Work& w, const Tables& t, const RangeItem* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return;
  k_stencil_box<<<nitems, kBoxThreads, 0, s>>>(t.lev, items, t.kpool, w.grid);
}

void launch_virial_box(const Work& w, const Tables& t, const RangeItem* items, int nitems, int part_off,
                       cudaStream_t s) {
  if (nitems <= 0) return;
  k_virial_box<<<nitems, kBoxThreads, 0, s>>>(t.lev, items, t.kpool, w.grid, w.part_wg + 6 * (long long)part_off);
}

}  // namespace msm
