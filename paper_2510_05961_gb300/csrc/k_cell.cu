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
