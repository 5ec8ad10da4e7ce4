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
// A block loads a tile of lines into shared memory and runs radix-2 stages
// with a barrier between them: decimation in time on bit-reversed input for
// forward transforms, decimation in frequency with bit-reversed output for
// inverse ones, so no separate permutation pass is needed. Twiddles
// exp(-2 pi i j / 256) come from a table in the stencil pool (FP64 values
// rounded once); a level axis of n points uses every (256 / n)-th entry.
#include "msm_internal.h"

namespace msm {

namespace {
constexpr int kSpecThreads = 256;

__device__ __forceinline__ int bitrev(int j, int lg) { return lg == 0 ? 0 : (int)(__brev((unsigned)j) >> (32 - lg)); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// radix-2 stages over T lines of n = 2^lg points held in shared memory, element
// j of line t at buf[t * ts + j * js]. DIT (forward, input bit-reversed) or DIF
// (inverse, output bit-reversed); conj selects exp(+2 pi i ...) twiddles.
template <bool DIT>
__device__ void fft_stages(float2* buf, int T, int lg, int ts, int js, const float2* tw, bool conj, bool tfast) {
  const int n = 1 << lg, nb = T * (n >> 1);
  for (int st = 0; st < lg; st++) {
    const int hl = DIT ? (1 << st) : (n >> (st + 1));  // half span of this stage
    const int sh = 8 - (DIT ? st + 1 : lg - st);        // twiddle step 256 / (2 hl) = 2^sh
    for (int b = threadIdx.x; b < nb; b += kSpecThreads) {
      int t, i;
      if (tfast) {
        t = b % T;
        i = b / T;
      } else {
        i = b & ((n >> 1) - 1);
        t = b >> (lg - 1);
      }
      const int g = i / hl, jj = i - g * hl;
      const int j0 = g * 2 * hl + jj, j1 = j0 + hl;
      float2 w = tw[jj << sh];
      if (conj) w.y = -w.y;
      float2* p0 = buf + t * ts + j0 * js;
      float2* p1 = buf + t * ts + j1 * js;
      const float2 a = *p0, c = *p1;
      if (DIT) {
        const float2 v = cmul(c, w);
        *p0 = make_float2(a.x + v.x, a.y + v.y);
        *p1 = make_float2(a.x - v.x, a.y - v.y);
      } else {
        *p0 = make_float2(a.x + c.x, a.y + c.y);
        *p1 = cmul(make_float2(a.x - c.x, a.y - c.y), w);
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void load_twiddles(float2* tw, const float* kpool, long long off) {
  for (int i = threadIdx.x; i < 256; i += kSpecThreads) tw[i] = make_float2(kpool[off + 2 * i], kpool[off + 2 * i + 1]);
}

__device__ __forceinline__ int fold_k(int k, int n) { return min(k, n - k); }
__device__ __forceinline__ float sgn_k(int k, int n) { return (k == 0 || 2 * k == n) ? 0.f : (2 * k < n ? 1.f : -1.f); }
}  // namespace

// z pass, forward: item (lev, x, y0, rows): rows z-lines (y0 .. y0 + rows - 1) at x
__global__ void __launch_bounds__(kSpecThreads) k_spec_z_fwd(const LevDev* __restrict__ lev, const TileItem* __restrict__ items,
                                                             const float* __restrict__ kpool, const float* __restrict__ grid,
                                                             float2* __restrict__ spec) {
  __shared__ float2 buf[kSpecTile];
  __shared__ float2 tw[256];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = lev[it.lev];
  load_twiddles(tw, kpool, L.tw_off);
  const int nz = L.n[2], lg = L.lg[2], T = it.z0;
  const long long base = ((long long)it.x0 * L.n[1] + it.y0) * nz;
  const float* q = grid + L.q_off + base;
  for (int e = threadIdx.x; e < T * nz; e += kSpecThreads) {
    const int t = e >> lg, j = e & (nz - 1);
    buf[t * nz + bitrev(j, lg)] = make_float2(q[e], 0.f);
  }
  __syncthreads();
  fft_stages<true>(buf, T, lg, nz, 1, tw, false, false);
  float2* out = spec + L.f_off + base;
  for (int e = threadIdx.x; e < T * nz; e += kSpecThreads) out[e] = buf[e];
}

// z pass, inverse: e^l = Re(inverse transform along z)
__global__ void __launch_bounds__(kSpecThreads) k_spec_z_inv(const LevDev* __restrict__ lev, const TileItem* __restrict__ items,
                                                             const float* __restrict__ kpool, float* __restrict__ grid,
                                                             const float2* __restrict__ spec) {
  __shared__ float2 buf[kSpecTile];
  __shared__ float2 tw[256];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = lev[it.lev];
  load_twiddles(tw, kpool, L.tw_off);
  const int nz = L.n[2], lg = L.lg[2], T = it.z0;
  const long long base = ((long long)it.x0 * L.n[1] + it.y0) * nz;
  const float2* in = spec + L.f_off + base;
  for (int e = threadIdx.x; e < T * nz; e += kSpecThreads) buf[e] = in[e];
  __syncthreads();
  fft_stages<false>(buf, T, lg, nz, 1, tw, true, false);
  float* e_out = grid + L.e_off + base;
  for (int e = threadIdx.x; e < T * nz; e += kSpecThreads) {
    const int t = e >> lg, j = e & (nz - 1);
    e_out[e] = buf[t * nz + bitrev(j, lg)].x;
  }
}

// y pass: item (lev, x, z0, cols): y-lines at x for z in [z0, z0 + cols); in place
template <bool INV>
__global__ void __launch_bounds__(kSpecThreads) k_spec_y(const LevDev* __restrict__ lev, const TileItem* __restrict__ items,
                                                         const float* __restrict__ kpool, float2* __restrict__ spec) {
  __shared__ float2 buf[kSpecTile];
  __shared__ float2 tw[256];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = lev[it.lev];
  load_twiddles(tw, kpool, L.tw_off);
  const int ny = L.n[1], nz = L.n[2], lg = L.lg[1], T = it.z0;
  float2* g = spec + L.f_off + (long long)it.x0 * ny * nz + it.y0;
  // shared layout [j][t]: t (z) fastest, matching the global order
  for (int e = threadIdx.x; e < T * ny; e += kSpecThreads) {
    const int t = e % T, j = e / T;
    buf[(INV ? j : bitrev(j, lg)) * T + t] = g[(long long)j * nz + t];
  }
  __syncthreads();
  if (INV) fft_stages<false>(buf, T, lg, 1, T, tw, true, true);
  else fft_stages<true>(buf, T, lg, 1, T, tw, false, true);
  for (int e = threadIdx.x; e < T * ny; e += kSpecThreads) {
    const int t = e % T, j = e / T;
    g[(long long)j * nz + t] = buf[(INV ? bitrev(j, lg) : j) * T + t];
  }
}

// x pass: item (lev, y, z0, cols): forward transform along x (the spectrum
// Q(k_x, k_y = y, k_z = z) is then complete), the virial sums, the product
// with K^ and the inverse transform along x; in place. part (when not null)
// receives the block's six virial sums at 6 * blockIdx.x.
template <bool MUL>
__global__ void __launch_bounds__(kSpecThreads) k_spec_x(const LevDev* __restrict__ lev, const TileItem* __restrict__ items,
                                                         const float* __restrict__ kpool, float2* __restrict__ spec,
                                                         double* __restrict__ part) {
  __shared__ float2 buf[kSpecTile];
  __shared__ float2 tw[256];
  __shared__ double red[kSpecThreads / 32][6];
  const TileItem it = items[blockIdx.x];
  const LevDev& L = lev[it.lev];
  load_twiddles(tw, kpool, L.tw_off);
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2], lg = L.lg[0], T = it.z0;
  float2* g = spec + L.f_off + (long long)it.x0 * nz + it.y0;  // x0 holds y, y0 holds z0
  const long long xs = (long long)ny * nz;
  for (int e = threadIdx.x; e < T * nx; e += kSpecThreads) {
    const int t = e % T, j = e / T;
    buf[bitrev(j, lg) * T + t] = g[(long long)j * xs + t];
  }
  __syncthreads();
  fft_stages<true>(buf, T, lg, 1, T, tw, false, true);
  // spectra octants: 7 arrays of (nx/2+1)(ny/2+1)(nz/2+1) floats: K^, then dK^ xx yy zz xy xz yz
  const int hy = ny / 2 + 1, hz = nz / 2 + 1;
  const long long oct = (long long)(nx / 2 + 1) * hy * hz;
  const float* sp = kpool + L.sp_off;
  const int ky = it.x0;
  const int fy = fold_k(ky, ny);
  const float sy = sgn_k(ky, ny);
  float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int e = threadIdx.x; e < T * nx; e += kSpecThreads) {
    const int t = e % T, kx = e / T, kz = it.y0 + t;
    const long long o = ((long long)fold_k(kx, nx) * hy + fy) * hz + fold_k(kz, nz);
    const float2 z = buf[e];
    if (part) {
      const float p2 = fmaf(z.x, z.x, z.y * z.y);
      const float sx = sgn_k(kx, nx), sz = sgn_k(kz, nz);
      w[0] = fmaf(sp[oct + o], p2, w[0]);
      w[1] = fmaf(sp[2 * oct + o], p2, w[1]);
      w[2] = fmaf(sp[3 * oct + o], p2, w[2]);
      w[3] = fmaf(sx * sy * sp[4 * oct + o], p2, w[3]);
      w[4] = fmaf(sx * sz * sp[5 * oct + o], p2, w[4]);
      w[5] = fmaf(sy * sz * sp[6 * oct + o], p2, w[5]);
    }
    if (MUL) {
      const float kk = sp[o];
      buf[e] = make_float2(kk * z.x, kk * z.y);
    }
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
  fft_stages<false>(buf, T, lg, 1, T, tw, true, true);
  for (int e = threadIdx.x; e < T * nx; e += kSpecThreads) {
    const int t = e % T, j = e / T;
    g[(long long)j * xs + t] = buf[bitrev(j, lg) * T + t];
  }
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
