// k_cell.cu -- a new cell for an existing plan, on the device (dynamic cells,
// Sec. 3.2.2: the stencils K^l sample the level kernels on grids that scale
// with the cell, so a cell change needs new stencils; the grid counts M, the
// level ranges and the stencil array sizes stay fixed, as in the paper's
// static-shape design, whose limits Sec. 4.1 lists: a compressed cell needs
// more stencil points than a fixed array holds).
//
// For the ball levels of a periodic system with raw samples (p = 4, minimal
// quasi-interpolation) everything cell-dependent is a pointwise function of
// the new level-1 spacings h_1: the samples s^1(n) = k_1(|h_1 o n|) of the
// level-1 kernel k_1 = gamma(r/a)/a - gamma(r/2a)/(2a) (Sec. 3.4), the
// factorized half-space virial weights g(n) = f(n) k_1'(|v|)/|v| (v = h_1 o n,
// f = 2 on the half space, 1 at n = 0, 0 elsewhere), and the column
// half-widths the ball kernels read. One block per stencil column (dx, dy)
// evaluates its dz entries in FP64 and stores them in FP32 at the layout the
// planner uses; a block reduction gives the column's half-widths. The system
// descriptor is passed by value and copied by one thread, so the host keeps
// no buffer alive after the call.
#include "msm_internal.h"

namespace msm {

// gamma(rho): 1/rho for rho >= 1, else sum_k c_k (1 - rho^2)^k with c_0 = 1,
// c_k = c_(k-1) (2k - 1) / (2k) (the Taylor polynomial of s^-1/2 about s = 1)
__device__ double cell_soft(int p, double rho) {
  if (rho >= 1.0) return 1.0 / rho;
  double c[8];
  c[0] = 1.0;
  for (int k = 1; k < p; k++) c[k] = c[k - 1] * (2.0 * k - 1.0) / (2.0 * k);
  const double t = 1.0 - rho * rho;
  double v = c[p - 1];
  for (int k = p - 2; k >= 0; k--) v = v * t + c[k];
  return v;
}

// d gamma / d rho
__device__ double cell_soft_d(int p, double rho) {
  if (rho >= 1.0) return -1.0 / (rho * rho);
  double c[8];
  c[0] = 1.0;
  for (int k = 1; k < p; k++) c[k] = c[k - 1] * (2.0 * k - 1.0) / (2.0 * k);
  const double t = 1.0 - rho * rho;
  double v = (p - 1) * c[p - 1];
  for (int k = p - 2; k >= 1; k--) v = v * t + k * c[k];
  return -2.0 * rho * v;
}

// level-1 kernel of an intermediate level (the top level of a periodic
// system is not evaluated) and its r-derivative
__device__ double cell_k1(int p, double a, double r, bool deriv) {
  const double s2 = 2.0 * a;
  if (r >= s2) return 0.0;
  if (deriv) return cell_soft_d(p, r / a) / (a * a) - cell_soft_d(p, r / s2) / (s2 * s2);
  return cell_soft(p, r / a) / a - cell_soft(p, r / s2) / s2;
}

struct CellStencilArgs {
  double h1[3];
  double a;
  int p;
  int B[3];      // ball radius (capacity of the plan)
  int hz;        // z halo of a stored column row
  long long kball_off, dkh_off, wb_off, wh_off;
};

constexpr int kCellThreads = 64;

__global__ void __launch_bounds__(kCellThreads) k_cell_stencils(CellStencilArgs A, float* __restrict__ kpool,
                                                                int* __restrict__ wpool) {
  __shared__ int red[2][kCellThreads / 32];
  const int ny = 2 * A.B[1] + 1, SK = kSK(A.hz);
  const int col = blockIdx.x, xi = col / ny, yi = col % ny;
  const int x = xi - A.B[0], y = yi - A.B[1];
  float* krow = kpool + A.kball_off + (long long)col * SK;
  float* grow = kpool + A.dkh_off + (long long)col * SK;
  int wb = -1, wh = -1;
  for (int e = threadIdx.x; e < SK; e += blockDim.x) {
    const int z = e - A.hz;
    float s = 0.f, g = 0.f;
    if (z >= -A.B[2] && z <= A.B[2]) {
      const double vx = A.h1[0] * x, vy = A.h1[1] * y, vz = A.h1[2] * z;
      const double rr = sqrt(vx * vx + vy * vy + vz * vz);
      s = (float)cell_k1(A.p, A.a, rr, false);
      const bool half = x > 0 || (x == 0 && y > 0) || (x == 0 && y == 0 && z > 0);
      const bool zero = x == 0 && y == 0 && z == 0;
      const double f = half ? 2.0 : (zero ? 1.0 : 0.0);
      g = rr > 0.0 ? (float)(f * cell_k1(A.p, A.a, rr, true) / rr) : 0.0f;
      const int wz = abs(z) + (abs(z) & 1);  // half-widths rounded up to even values
      if (s != 0.0f) wb = max(wb, wz);
      if (g != 0.0f) wh = max(wh, wz);
    }
    krow[e] = s;
    grow[e] = g;
  }
  for (int o = 16; o > 0; o >>= 1) {
    wb = max(wb, __shfl_down_sync(0xffffffffu, wb, o));
    wh = max(wh, __shfl_down_sync(0xffffffffu, wh, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = wb;
    red[1][threadIdx.x >> 5] = wh;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kCellThreads / 32; w++) {
      wb = max(wb, red[0][w]);
      wh = max(wh, red[1][w]);
    }
    wpool[A.wb_off + col] = wb;
    wpool[A.wh_off + col] = wh;
  }
}

// Spectra of the spectral level method for the new cell (plans of the same
// kind: periodic, p = 4, raw samples): K^ = w(kx) w(ky) w(kz) s^ and dK^_ab =
// w w w ds^_ab, w the transform of omega' (omega'_0 + 2 sum_m omega'_m
// cos(2 pi k m / n)), s^ and ds^ the DFTs of the raw samples s(n) = k_1(|v|)
// and ds_ab(n) = k_1'(|v|) v_a v_b / |v| over the sample box (v = h_1 o n;
// samples beyond 2a vanish), evaluated as separable sums (z, then y, then x)
// with cosines along even axes and sines along odd ones (K, dK_aa even in
// every axis; dK_ab odd in a and b, its transform minus the sine-sine-cosine
// sum). Level l stores them times 2^-(l-1) / N and -1/2 2^-(l-1) / N at its
// octant, interleaved as the planner does. Samples in FP64, sums in FP32.
struct SpecCellArgs {
  double h1[3];
  double a;
  int p;
  int B[3];
  float om[8];
  int hw;
  int nlev;               // levels, one grid dimension of the launches each
  int n[kMaxLev];         // points per axis
  long long sp[kMaxLev];  // spectrum offsets in the stencil pool
  long long oa[kMaxLev];  // scratch offsets of the z sums and of the y sums
  long long ob[kMaxLev];
};

namespace {
constexpr int kSpecCellThreads = 256;
constexpr int kSpecCellBox = 2 * kBallRmax + 1;  // longest sample-box axis
constexpr int kSpecCellH = kSpecNmax / 2 + 1;    // longest octant axis
// trigonometric parity (0 cos, 1 sin) per component and axis: K, xx, yy, zz, xy, xz, yz
__constant__ int c_spec_par[7][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};

// cs[j], sn[j] = cos, sin of 2 pi j / n for j < n (n a power of two: the angle of k m is
// that of (k m) & (n - 1), exactly, for negative m too)
__device__ void trig_table(float* cs, float* sn, int n) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) sincospif(2.0f * (float)j / (float)n, &sn[j], &cs[j]);
}
}  // namespace

// raw samples of the seven components on the box [-B, B]^3, once for all levels:
// smp[(c * ncol + col) * nzb + zi] (FP64 evaluation, stored as float)
__global__ void __launch_bounds__(kSpecCellThreads) k_spec_cell_smp(SpecCellArgs A, float* __restrict__ smp) {
  const int nyb = 2 * A.B[1] + 1, nzb = 2 * A.B[2] + 1, ncol = (2 * A.B[0] + 1) * nyb;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ncol * nzb) return;
  const int col = e / nzb, zi = e - col * nzb;
  const int x = col / nyb - A.B[0], y = col % nyb - A.B[1], z = zi - A.B[2];
  const double v[3] = {A.h1[0] * x, A.h1[1] * y, A.h1[2] * z};
  const double rr = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const double g = rr > 0.0 ? cell_k1(A.p, A.a, rr, true) / rr : 0.0;
  const float val[7] = {(float)cell_k1(A.p, A.a, rr, false), (float)(g * v[0] * v[0]), (float)(g * v[1] * v[1]),
                        (float)(g * v[2] * v[2]),           (float)(g * v[0] * v[1]), (float)(g * v[0] * v[2]),
                        (float)(g * v[1] * v[2])};
#pragma unroll
  for (int c = 0; c < 7; c++) smp[((long long)c * ncol + col) * nzb + zi] = val[c];
}

// z sums: one block per sample column (x, y) and level; out[(c * ncol + col) * hz + kz]
__global__ void __launch_bounds__(kSpecCellThreads) k_spec_cell_z(SpecCellArgs A, const float* __restrict__ smp_g,
                                                                  float* __restrict__ scratch) {
  __shared__ float cs[kSpecNmax], sn[kSpecNmax];
  __shared__ float smp[7][kSpecCellBox];
  const int n = A.n[blockIdx.y], msk = n - 1;
  float* out = scratch + A.oa[blockIdx.y];
  const int nyb = 2 * A.B[1] + 1, nzb = 2 * A.B[2] + 1, ncol = (2 * A.B[0] + 1) * nyb;
  const int col = blockIdx.x;
  const int hz = n / 2 + 1;
  for (int e = threadIdx.x; e < 7 * nzb; e += blockDim.x) {
    const int c = e / nzb, zi = e - c * nzb;
    smp[c][zi] = smp_g[((long long)c * ncol + col) * nzb + zi];
  }
  trig_table(cs, sn, n);
  __syncthreads();
  for (int e = threadIdx.x; e < 7 * hz; e += blockDim.x) {
    const int c = e / hz, kz = e - c * hz;
    const float* t = c_spec_par[c][2] ? sn : cs;
    float acc = 0.f;
    for (int zi = 0; zi < nzb; zi++) acc = fmaf(smp[c][zi], t[(kz * (zi - A.B[2])) & msk], acc);
    out[((long long)c * ncol + col) * hz + kz] = acc;
  }
}

// y sums: one block per (component, x) and level, the column slice staged in shared
// memory; out[((c * nxb + xi) * hy + ky) * hz + kz]
__global__ void __launch_bounds__(kSpecCellThreads) k_spec_cell_y(SpecCellArgs A, const float* __restrict__ scr_a,
                                                                  float* __restrict__ scr_b) {
  __shared__ float cs[kSpecNmax], sn[kSpecNmax];
  __shared__ float slice[kSpecCellBox * kSpecCellH];
  const int n = A.n[blockIdx.y], msk = n - 1;
  const float* in = scr_a + A.oa[blockIdx.y];
  float* out = scr_b + A.ob[blockIdx.y];
  const int nxb = 2 * A.B[0] + 1, nyb = 2 * A.B[1] + 1, ncol = nxb * nyb;
  const int c = blockIdx.x / nxb, xi = blockIdx.x - c * nxb;
  const int hy = n / 2 + 1, hz = n / 2 + 1;
  const float* src = in + ((long long)c * ncol + (long long)xi * nyb) * hz;
  for (int e = threadIdx.x; e < nyb * hz; e += blockDim.x) slice[e] = src[e];
  trig_table(cs, sn, n);
  __syncthreads();
  const float* t = c_spec_par[c][1] ? sn : cs;
  for (int e = threadIdx.x; e < hy * hz; e += blockDim.x) {
    const int ky = e / hz, kz = e - ky * hz;
    float acc = 0.f;
    for (int yi = 0; yi < nyb; yi++) acc = fmaf(slice[yi * hz + kz], t[(ky * (yi - A.B[1])) & msk], acc);
    out[(((long long)c * nxb + xi) * hy + ky) * hz + kz] = acc;
  }
}

// x sums, the omega' transforms and the scale: one block per (component, k_y) and level, the
// slice [x][k_z] staged in shared memory
__global__ void __launch_bounds__(kSpecCellThreads) k_spec_cell_x(SpecCellArgs A, const float* __restrict__ scr_b,
                                                                  float* __restrict__ kpool) {
  __shared__ float cs[kSpecNmax], sn[kSpecNmax];
  __shared__ float wt[kSpecCellH];
  __shared__ float slice[kSpecCellBox * kSpecCellH];
  const int level = blockIdx.y + 1, n = A.n[blockIdx.y], msk = n - 1;
  const float* in = scr_b + A.ob[blockIdx.y];
  const long long sp_off = A.sp[blockIdx.y];
  const int nxb = 2 * A.B[0] + 1, h = n / 2 + 1;
  if ((int)blockIdx.x >= 7 * h) return;  // the grid is sized for level 1
  const int c = blockIdx.x / h, ky = blockIdx.x - c * h;
  for (int e = threadIdx.x; e < nxb * h; e += blockDim.x) {
    const int xi = e / h, kz = e - xi * h;
    slice[e] = in[(((long long)c * nxb + xi) * h + ky) * h + kz];
  }
  trig_table(cs, sn, n);
  __syncthreads();
  for (int k = threadIdx.x; k < h; k += blockDim.x) {  // transform of omega' at index k
    float w = A.om[0];
    for (int m = 1; m <= A.hw; m++) w = fmaf(2.0f * A.om[m], cs[(k * m) & msk], w);
    wt[k] = w;
  }
  __syncthreads();
  const double N = (double)n * n * n;
  const float scale = (float)((c == 0 ? 1.0 : -0.5) * (c >= 4 ? -1.0 : 1.0) * ldexp(1.0, -(level - 1)) / N);
  const float wy = wt[ky] * scale;
  const float* t = c_spec_par[c][0] ? sn : cs;
  for (int e = threadIdx.x; e < h * h; e += blockDim.x) {
    const int kx = e / h, kz = e - kx * h;
    float acc = 0.f;
    for (int xi = 0; xi < nxb; xi++) acc = fmaf(slice[xi * h + kz], t[(kx * (xi - A.B[0])) & msk], acc);
    // at [|k_x|][|k_y|][z position]: the positions whose bit reversal is k_z or n - k_z
    const float val = acc * wy * wt[kx] * wt[kz];
    int lgn = 0;
    while ((1 << lgn) < n) lgn++;
    const int z0 = (int)(__brev((unsigned)kz) >> (32 - lgn)), z1 = (int)(__brev((unsigned)((n - kz) & msk)) >> (32 - lgn));
    const long long row = ((long long)kx * h + ky) * n;
    kpool[sp_off + 8 * (row + z0) + c] = val;
    kpool[sp_off + 8 * (row + z1) + c] = val;
  }
}

void launch_spec_cell(const double h1[3], double a, int p, const int B[3], const double* om, int hw, int nlev,
                      const int* n, const long long* sp_off, float* scratch_a, float* scratch_b, float* kpool,
                      cudaStream_t s) {
  SpecCellArgs A;
  for (int d = 0; d < 3; d++) {
    A.h1[d] = h1[d];
    A.B[d] = B[d];
  }
  A.a = a;
  A.p = p;
  A.hw = hw;
  for (int m = 0; m < 8; m++) A.om[m] = m <= hw ? (float)om[m] : 0.f;
  const int nxb = 2 * B[0] + 1, ncol = nxb * (2 * B[1] + 1);
  A.nlev = nlev < kMaxLev ? nlev : kMaxLev;
  long long oa = 0, ob = 0;
  for (int l = 0; l < A.nlev; l++) {
    const long long h = n[l] / 2 + 1;
    A.n[l] = n[l];
    A.sp[l] = sp_off[l];
    A.oa[l] = oa;
    A.ob[l] = ob;
    oa += 7 * ncol * h;
    ob += 7 * nxb * h * h;
  }
  if (A.nlev <= 0) return;
  const int h1max = n[0] / 2 + 1;  // level 1 has the most points
  // the samples go after the regions of the y sums in scratch_b
  float* smp = scratch_b + ob;
  const int nzb = 2 * B[2] + 1;
  k_spec_cell_smp<<<(ncol * nzb + kSpecCellThreads - 1) / kSpecCellThreads, kSpecCellThreads, 0, s>>>(A, smp);
  k_spec_cell_z<<<dim3(ncol, A.nlev), kSpecCellThreads, 0, s>>>(A, smp, scratch_a);
  k_spec_cell_y<<<dim3(7 * nxb, A.nlev), kSpecCellThreads, 0, s>>>(A, scratch_a, scratch_b);
  k_spec_cell_x<<<dim3(7 * h1max, A.nlev), kSpecCellThreads, 0, s>>>(A, scratch_b, kpool);  // blocks (c, k_y)
}

__global__ void k_set_sys(SysDev* __restrict__ dst, SysDev val) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = val;
}

void launch_set_sys(SysDev* d_sys, const SysDev& val, cudaStream_t s) { k_set_sys<<<1, 32, 0, s>>>(d_sys, val); }

void launch_cell_update(SysDev* d_sys, const SysDev& val, const double h1[3], double a, int p, const int B[3], int hz,
                        long long kball_off, long long dkh_off, long long wb_off, long long wh_off, float* kpool,
                        int* wpool, cudaStream_t s) {
  k_set_sys<<<1, 32, 0, s>>>(d_sys, val);
  CellStencilArgs A;
  for (int d = 0; d < 3; d++) {
    A.h1[d] = h1[d];
    A.B[d] = B[d];
  }
  A.a = a;
  A.p = p;
  A.hz = hz;
  A.kball_off = kball_off;
  A.dkh_off = dkh_off;
  A.wb_off = wb_off;
  A.wh_off = wh_off;
  const int ncol = (2 * B[0] + 1) * (2 * B[1] + 1);
  k_cell_stencils<<<ncol, kCellThreads, 0, s>>>(A, kpool, wpool);
}

}  // namespace msm
