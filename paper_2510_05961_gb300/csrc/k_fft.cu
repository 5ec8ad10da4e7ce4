// k_fft.cu -- the level stencils of Eq. action_of_K_as_convolution applied in
// Fourier space on fully periodic levels ("spectral" level method).
//
// On a periodic level of n_x x n_y x n_z points (powers of two) the stencil
// sum e_m = sum_n K_(m-n) q~_n is a circular convolution with the folded
// stencil, so with the discrete Fourier transform Q(k) = sum_m q~_m
// exp(-2 pi i k.m / n),
//   e = IDFT(K^ Q),   K^(k) = sum_n K_n exp(-2 pi i k.n / n)  (the unfolded
//                     stencil's transform sampled at k / n: folding is exact),
// and the level's virial term -1/2 q~^T dK_ab q~ (reading of the virial as the
// strain derivative at fixed fractional coordinates) is, by Parseval,
//   -1/2 (1/N) sum_k dK^_ab(k) |Q(k)|^2,   N = n_x n_y n_z.
// For rectangular cells K and the diagonal dK_aa are even in every axis and
// dK_ab (a != b) is odd in a and b and even in the third, so every spectrum
// is real, equal to its value at (|k_x|, |k_y|, |k_z|) (folded to [0, n/2])
// times sgn(k_a) sgn(k_b) for the off-diagonal ones. The planner computes
// these octants in FP64 from K^1 and dK^1 (level l: scaled by 2^-(l-1)) and
// stores them pre-multiplied by 1/N (K^) and by -1/2 (1/N) (dK^).
//
// Three passes of one-dimensional FFTs over a complex work buffer per level
// (layout [x][y][z], z fastest), each over all spectral levels in one launch:
//   z: q~ (real) -> transform along z               (k_spec_z_fwd)
//   y: transform along y                            (k_spec_y, forward)
//   x: transform along x, virial sums over |Q|^2, multiply by K^, inverse
//      transform along x                            (k_spec_x)
//   y: inverse transform along y                    (k_spec_y, inverse)
//   z: inverse transform along z, real part -> e^l  (k_spec_z_inv)
// A block loads a tile of T lines into shared memory, lines interleaved (point j
// of line t at j (T + 1) + t: consecutive threads take consecutive lines, and
// the z pass's transposing copy meets at most two-way bank conflicts), and
// runs the radix-2 stages in rounds of up to three: each thread loads 8 (4, 2)
// points of one group into registers, applies the round's stages there with
// the radix-2 twiddles, and stores them back, one barrier per round. Forward
// transforms run by decimation in frequency (natural input, output in
// bit-reversed order) and inverse ones by decimation in time (bit-reversed
// input, natural output), so every pass reads and writes its lines in place
// and in order: between the forward and the inverse passes the work buffer
// holds the spectrum with each axis in bit-reversed order, which the x pass
// undoes only to look up the spectra.
// Twiddles exp(-2 pi i j / 256) come from a table in the stencil pool (FP64
// values rounded once); a level axis of n points uses every (256 / n)-th entry.
// The spectra are stored interleaved, eight floats per point (K^, dK^ xx yy zz
// xy xz yz, zero; two 16-byte loads) at [|k_x|][|k_y|][z position]: along z by
// the buffer's bit-reversed position, so the consecutive z of a tile read
// consecutive memory.
#include "msm_internal.h"

namespace msm {

namespace {
constexpr int kSpecThreads = 256;
constexpr int kPer = kSpecTile / kSpecThreads;  // tile elements per thread, at most
constexpr int kSpecBuf = kSpecTile + kSpecNmax; // interleaved tile with one padding point per line position

__device__ __forceinline__ int bitrev(int j, int lg) { return lg == 0 ? 0 : (int)(__brev((unsigned)j) >> (32 - lg)); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// One round of R radix-2 stages over the tile (T = 2^lgT lines of 2^lg points,
// point j of line t at buf[j * (T + 1) + t]). A group is the 2^R points j = base +
// m 2^lq (m < 2^R) that the round's stages combine; each thread takes whole
// groups in registers. DIF (forward, twiddles exp(-2 pi i ...)): stages with half
// spans 2^(lq+R-1) down to 2^lq; DIT (inverse, twiddles exp(+2 pi i ...)): half
// spans 2^lq up to 2^(lq+R-1). The stage of half span h pairs p, p + h (bit of h
// clear in p) with the twiddle of index (p mod h) 256 / (2 h) in the table.
template <bool DIT, int R>
__device__ __forceinline__ void fft_round(float2* buf, int lg, int lgT, int lq, const float2* tw) {
  constexpr int M = 1 << R;
  const int T = 1 << lgT, P = T + 1;
  const int ngroups = (1 << (lg - R)) << lgT;
  for (int g = threadIdx.x; g < ngroups; g += kSpecThreads) {
    const int t = g & (T - 1), rest = g >> lgT;
    const int lo = rest & ((1 << lq) - 1), hi = rest >> lq;
    const int base = (hi << (lq + R)) + lo;
    float2 x[M];
#pragma unroll
    for (int m = 0; m < M; m++) x[m] = buf[(base + (m << lq)) * P + t];
#pragma unroll
    for (int k = 0; k < R; k++) {
      const int sub = DIT ? k : R - 1 - k;
      const int h = 1 << sub, s2 = lq + sub;
#pragma unroll
      for (int m = 0; m < M; m++) {
        if (m & h) continue;
        float2 w = tw[((((m & (h - 1)) << lq) + lo) << (7 - s2))];
        const float2 a = x[m], c = x[m + h];
        if (DIT) {
          w.y = -w.y;
          const float2 v = cmul(c, w);
          x[m] = make_float2(a.x + v.x, a.y + v.y);
          x[m + h] = make_float2(a.x - v.x, a.y - v.y);
        } else {
          x[m] = make_float2(a.x + c.x, a.y + c.y);
          x[m + h] = cmul(make_float2(a.x - c.x, a.y - c.y), w);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < M; m++) buf[(base + (m << lq)) * P + t] = x[m];
  }
  __syncthreads();
}

// the whole transform of every line of the tile: rounds of three stages (the last one shorter)
template <bool DIT>
__device__ __forceinline__ void fft_tile(float2* buf, int lg, int lgT, const float2* tw) {
  if (DIT) {
    for (int k = 0; k < lg;) {
      const int R = min(3, lg - k);
      if (R == 3) fft_round<true, 3>(buf, lg, lgT, k, tw);
      else if (R == 2) fft_round<true, 2>(buf, lg, lgT, k, tw);
      else fft_round<true, 1>(buf, lg, lgT, k, tw);
      k += R;
    }
  } else {
    for (int k = lg; k > 0;) {
      const int R = min(3, k);
      if (R == 3) fft_round<false, 3>(buf, lg, lgT, k - 3, tw);
      else if (R == 2) fft_round<false, 2>(buf, lg, lgT, k - 2, tw);
      else fft_round<false, 1>(buf, lg, lgT, k - 1, tw);
      k -= R;
    }
  }
}

__device__ __forceinline__ void load_twiddles(float2* tw, const float* kpool, long long off) {
  for (int i = threadIdx.x; i < 256; i += kSpecThreads) tw[i] = make_float2(kpool[off + 2 * i], kpool[off + 2 * i + 1]);
}

__device__ __forceinline__ int fold_k(int k, int n) { return min(k, n - k); }
__device__ __forceinline__ float sgn_k(int k, int n) { return (k == 0 || 2 * k == n) ? 0.f : (2 * k < n ? 1.f : -1.f); }

__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }

// T lines' points j at g[j * stride + t] (t < T: consecutive z) into the tile
__device__ __forceinline__ void load_lines(float2* buf, const float2* __restrict__ g, long long stride, int lg, int lgT) {
  const int cnt = 1 << (lg + lgT), P = (1 << lgT) + 1;
  float2 r[kPer];
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    const int e = threadIdx.x + k * kSpecThreads;
    r[k] = e < cnt ? g[(long long)(e >> lgT) * stride + (e & ((1 << lgT) - 1))] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    const int e = threadIdx.x + k * kSpecThreads;
    if (e < cnt) buf[(e >> lgT) * P + (e & ((1 << lgT) - 1))] = r[k];
  }
  __syncthreads();
}

__device__ __forceinline__ void store_lines(const float2* buf, float2* __restrict__ g, long long stride, int lg, int lgT) {
  const int cnt = 1 << (lg + lgT), P = (1 << lgT) + 1;
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    const int e = threadIdx.x + k * kSpecThreads;
    if (e < cnt) g[(long long)(e >> lgT) * stride + (e & ((1 << lgT) - 1))] = buf[(e >> lgT) * P + (e & ((1 << lgT) - 1))];
  }
}
}  // namespace

// z pass, forward: item (lev, x, y0, rows): rows z-lines (y0 .. y0 + rows - 1) at x
__global__ void __launch_bounds__(kSpecThreads, 5) k_spec_z_fwd(const LevDev* __restrict__ lev, const TileItem* __restrict__ items,
                                                             const float* __restrict__ kpool, const float* __restrict__ grid,
                                                             float2* __restrict__ spec) {
  __shared__ float2 buf[kSpecBuf];
  __shared__ float2 tw[256];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = lev[it.lev];
  load_twiddles(tw, kpool, L.tw_off);
  const long long base = ((long long)it.x0 * L.n[1] + it.y0) * L.n[2];
  const float* q = grid + L.q_off + base;
  const int lg = L.lg[2], lgT = ilog2(it.z0), cnt = it.z0 << lg, P = it.z0 + 1;
  float r[kPer];
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    const int e = threadIdx.x + k * kSpecThreads;
    r[k] = e < cnt ? q[e] : 0.f;  // every load issued before the first shared-memory store
  }
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    const int e = threadIdx.x + k * kSpecThreads;  // line e >> lg, point e & (n - 1)
    if (e < cnt) buf[(e & ((1 << lg) - 1)) * P + (e >> lg)] = make_float2(r[k], 0.f);
  }
  __syncthreads();
  fft_tile<false>(buf, lg, lgT, tw);
  float2* out = spec + L.f_off + base;
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    const int e = threadIdx.x + k * kSpecThreads;
    if (e < cnt) out[e] = buf[(e & ((1 << lg) - 1)) * P + (e >> lg)];
  }
}

// z pass, inverse: e^l = Re(inverse transform along z)
__global__ void __launch_bounds__(kSpecThreads, 5) k_spec_z_inv(const LevDev* __restrict__ lev, const TileItem* __restrict__ items,
                                                             const float* __restrict__ kpool, float* __restrict__ grid,
                                                             const float2* __restrict__ spec) {
  __shared__ float2 buf[kSpecBuf];
  __shared__ float2 tw[256];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = lev[it.lev];
  load_twiddles(tw, kpool, L.tw_off);
  const long long base = ((long long)it.x0 * L.n[1] + it.y0) * L.n[2];
  const float2* in = spec + L.f_off + base;
  const int lg = L.lg[2], lgT = ilog2(it.z0), cnt = it.z0 << lg, P = it.z0 + 1;
  float2 r[kPer];
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    const int e = threadIdx.x + k * kSpecThreads;
    r[k] = e < cnt ? in[e] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    const int e = threadIdx.x + k * kSpecThreads;
    if (e < cnt) buf[(e & ((1 << lg) - 1)) * P + (e >> lg)] = r[k];
  }
  __syncthreads();
  fft_tile<true>(buf, lg, lgT, tw);
  float* e_out = grid + L.e_off + base;
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    const int e = threadIdx.x + k * kSpecThreads;
    if (e < cnt) e_out[e] = buf[(e & ((1 << lg) - 1)) * P + (e >> lg)].x;
  }
}

// y pass: item (lev, x, z0, cols): y-lines at x for z in [z0, z0 + cols); in place
template <bool INV>
__global__ void __launch_bounds__(kSpecThreads, 5) k_spec_y(const LevDev* __restrict__ lev, const TileItem* __restrict__ items,
                                                         const float* __restrict__ kpool, float2* __restrict__ spec) {
  __shared__ float2 buf[kSpecBuf];
  __shared__ float2 tw[256];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = lev[it.lev];
  load_twiddles(tw, kpool, L.tw_off);
  float2* g = spec + L.f_off + (long long)it.x0 * L.n[1] * L.n[2] + it.y0;
  const int lg = L.lg[1], lgT = ilog2(it.z0);
  load_lines(buf, g, L.n[2], lg, lgT);
  fft_tile<INV>(buf, lg, lgT, tw);
  store_lines(buf, g, L.n[2], lg, lgT);
}

// x pass: item (lev, y, z0, cols): forward transform along x (the spectrum
// is then complete, every axis in bit-reversed order), the virial sums, the
// product with K^ and the inverse transform along x; in place. part (when not
// null) receives the block's six virial sums at 6 * blockIdx.x.
template <bool MUL>
__global__ void __launch_bounds__(kSpecThreads, 5) k_spec_x(const LevDev* __restrict__ lev, const TileItem* __restrict__ items,
                                                         const float* __restrict__ kpool, float2* __restrict__ spec,
                                                         double* __restrict__ part) {
  __shared__ float2 buf[kSpecBuf];
  __shared__ float2 tw[256];
  __shared__ double red[kSpecThreads / 32][6];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = lev[it.lev];
  load_twiddles(tw, kpool, L.tw_off);
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  const int lg = L.lg[0], lgT = ilog2(it.z0), P = it.z0 + 1;
  float2* g = spec + L.f_off + (long long)it.x0 * nz + it.y0;  // x0 holds y, y0 holds z0
  const long long xs = (long long)ny * nz;
  load_lines(buf, g, xs, lg, lgT);
  fft_tile<false>(buf, lg, lgT, tw);
  // spectra, 8 floats per point (K^, dK^ xx yy zz xy xz yz, 0) at [|k_x|][|k_y|][z position]
  const int hy = ny / 2 + 1;
  const float4* sp = reinterpret_cast<const float4*>(kpool + L.sp_off);
  const int ky = bitrev(it.x0, L.lg[1]);
  const int fy = fold_k(ky, ny);
  const float sy = sgn_k(ky, ny);
  const int cnt = 1 << (lg + lgT);
  float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    const int e = threadIdx.x + k * kSpecThreads;
    if (e >= cnt) continue;
    const int t = e & ((1 << lgT) - 1), j = e >> lgT;
    const int kx = bitrev(j, lg), kz = bitrev(it.y0 + t, L.lg[2]);
    const long long o = ((long long)fold_k(kx, nx) * hy + fy) * nz + it.y0 + t;
    const float4 s0 = sp[2 * o];
    float2* bp = buf + j * P + t;
    const float2 z = *bp;
    if (part) {
      const float4 s1 = sp[2 * o + 1];
      const float p2 = fmaf(z.x, z.x, z.y * z.y);
      const float sx = sgn_k(kx, nx), sz = sgn_k(kz, nz);
      w[0] = fmaf(s0.y, p2, w[0]);
      w[1] = fmaf(s0.z, p2, w[1]);
      w[2] = fmaf(s0.w, p2, w[2]);
      w[3] = fmaf(sx * sy * s1.x, p2, w[3]);
      w[4] = fmaf(sx * sz * s1.y, p2, w[4]);
      w[5] = fmaf(sy * sz * s1.z, p2, w[5]);
    }
    if (MUL) *bp = make_float2(s0.x * z.x, s0.x * z.y);
  }
  if (part) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 6; c++) {
      double v = (double)w[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[wid][c] = v;
    }
  }
  __syncthreads();
  if (part && threadIdx.x < 6) {
    double v = 0.0;
    for (int k = 0; k < kSpecThreads / 32; k++) v += red[k][threadIdx.x];
    part[6 * (long long)blockIdx.x + threadIdx.x] = v;
  }
  if (!MUL) return;
  fft_tile<true>(buf, lg, lgT, tw);
  store_lines(buf, g, xs, lg, lgT);
}

// forward: e^l of every spectral level from q~^l (and, with part, the grid virial partials)
void launch_spectral(const Work& w, const Tables& t, const TileItem* zi, int nz, const TileItem* yi, int ny,
                     const TileItem* xi, int nx, double* part, cudaStream_t s) {
  if (nz <= 0) return;
  k_spec_z_fwd<<<nz, kSpecThreads, 0, s>>>(t.lev, zi, t.kpool, w.grid, w.spec);
  k_spec_y<false><<<ny, kSpecThreads, 0, s>>>(t.lev, yi, t.kpool, w.spec);
  k_spec_x<true><<<nx, kSpecThreads, 0, s>>>(t.lev, xi, t.kpool, w.spec, part);
  k_spec_y<true><<<ny, kSpecThreads, 0, s>>>(t.lev, yi, t.kpool, w.spec);
  k_spec_z_inv<<<nz, kSpecThreads, 0, s>>>(t.lev, zi, t.kpool, w.grid, w.spec);
}

// grid virial partials alone (a forward that did not compute them)
void launch_spectral_virial(const Work& w, const Tables& t, const TileItem* zi, int nz, const TileItem* yi, int ny,
                            const TileItem* xi, int nx, double* part, cudaStream_t s) {
  if (nz <= 0) return;
  k_spec_z_fwd<<<nz, kSpecThreads, 0, s>>>(t.lev, zi, t.kpool, w.grid, w.spec);
  k_spec_y<false><<<ny, kSpecThreads, 0, s>>>(t.lev, yi, t.kpool, w.spec);
  k_spec_x<false><<<nx, kSpecThreads, 0, s>>>(t.lev, xi, t.kpool, w.spec, part);
}

}  // namespace msm
