// k_short.cu -- short-range part U^0 of the MSM (Eq. U_zero) over the cell
// list: for every sorted atom i, every atom j and every periodic image with
// 0 < |d| < a,
//   phi0_i += q_j k_0(|d|),  k_0(r) = 1/r - gamma(r/a)/a   (Sec. 3.4),
//   F0_i   += q_i q_j k_0'(r) d / r,
//   W0     += -1/2 q_i q_j k_0'(r) d d^T / r,
// and phi0_i -= q_i gamma(0)/a (the self term, sum_(l>=1) k_l(0)).
//
// Virial. With g_ij = q_i q_j k_0'(r)/r and F_i = sum_(j,n) g_ij d_ij, write
// d = xi_j + t - xi_i with xi the atom's offset from a reference point of its
// own and t the offset between the two reference points (periodic image
// included). Pairing every ordered pair (i, j, n) with (j, i, -n) turns the
// sum over xi_j into one over xi_i, which gives the exact identity
//   -1/2 sum g d d^T = sum_i xi_i F_i^T - 1/2 sum_i sum_runs t (sum_run g d)^T.
// Rectangular cells (k_short) use it for the x and y components with xi the
// offset from the cell corner (at most one cell edge) and t the column offset
// (ox e_x, oy e_y), constant over a neighbour column, so the x, y parts cost
// one outer product per column; the z components (where the sorted z is
// measured from the column base, up to L_z) are summed pair by pair. Every term
// is then bounded by a few cell edges times |g d|, so the rounding does not
// grow with the atoms' distance from the origin. The tilted-cell kernel uses
// the identity with xi = r_i (the whole position) and t = A n, i.e.
//   -1/2 sum g d d^T = sum_i r_i F_i^T - 1/2 sum_(i,j,n) (A n) (g d)^T,
// whose last sum only has terms for periodic images n != 0; its rounding
// grows with |r_i| |F_i|.
//
// Rectangular cells (k_short): one thread per sorted atom i. Candidates: for
// each (dx, dy) column of cells around i's cell whose xy distance to i is
// below a, the cells of that column along z within sqrt(a^2 - dxy^2) of i.
// Cells of one column are consecutive in the sorted order, so each column
// contributes one contiguous range of atoms per periodic image along z.
// Sorted positions keep x, y relative to the cell corner and z relative to
// the column base, so the displacement to a candidate is (ox * edge_x + x_j -
// x_i, oy * edge_y + y_j - y_i, z_j + kz * L_z - z_i) with no wrap arithmetic
// per pair. The self pair gives exactly d = 0 and every other image of i lies
// a period away, so the pair test 0 < r^2 < a^2 excludes exactly (j, image) =
// (i, 0) (distinct atoms at one point have infinite Coulomb energy and are
// outside the method's domain). Small periodic cells visit the same cells at
// several offsets: every image within the cutoff counts. One thread per
// sorted atom; each thread sums its own pairs, so the result does not depend
// on scheduling. Whether forces and the virial are wanted are template
// parameters, so the pair loop carries no runtime flags.
#include "msm_internal.h"

namespace msm {

__device__ __forceinline__ int floordiv_s(int a, int b) {
  int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// k L - z, rounded once (FP64 only for the z-runs across a periodic face)
__device__ __forceinline__ float image_shift(int k, double L, float z) {
  if (k == 0) return -z;
  return (float)(k * L - (double)z);
}

// NB threads per block: NB = kChunk (one block per atom item) or kChunk / 2
// (two blocks per item), chosen by the autotuner
template <int P, bool WF, bool WW, int NB>
__global__ void __launch_bounds__(NB, 1024 / NB) k_short(const SysDev* __restrict__ sys, const AtomItem* __restrict__ items,
                                              const int* __restrict__ cell_start, const int* __restrict__ scell,
                                              const float4* __restrict__ xq, float* __restrict__ phi_sr,
                                              float4* __restrict__ f_sr, double* __restrict__ part_w0) {
  constexpr int NSPLIT = kChunk / NB;
  const int item = blockIdx.x / NSPLIT, part = blockIdx.x % NSPLIT;
  AtomItem it = items[item];
  const SysDev& S = sys[it.sys];
  const int slot = part * NB + (int)threadIdx.x;  // atom of the item
  int local = it.start + slot;
  bool active = slot < it.count && local < S.n;
  float w6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (active) {
    const int k = S.atom_off + local;
    const float4 xi = xq[k];
    const int cell = scell[k];
    const int Cx = S.C[0], Cy = S.C[1], Cz = S.C[2];
    const int ci[3] = {cell / (Cy * Cz), (cell / Cz) % Cy, cell % Cz};
    float gc[P], gdc[P - 1];
#pragma unroll
    for (int t = 0; t < P; t++) gc[t] = S.gca[t];
#pragma unroll
    for (int t = 0; t < P - 1; t++) gdc[t] = S.gdca[t];
    const float a2 = S.a2, inv_a2 = S.inv_a2;
    const float ex = S.edge[0], ey = S.edge[1], inv_ez = 1.0f / S.edge[2];
    // the binning contract may place an atom a rounding step outside its cell's
    // faces; culling keeps a margin of 2e-4 cell edges (enough for C <= 512)
    constexpr float mg = 2e-4f;
    float ph = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
    // virial sums (xx yy zz xy xz yz): xx, yy, xy the column terms t (sum g d)^T of
    // the identity above, zz, xz, yz sum q_j k_0'(r)/r d_z d pair by pair
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int ox = -S.nnbr[0]; ox <= S.nnbr[0]; ox++) {
      const float tx = (float)ox * ex;  // offset between the cell corners of i and of this column
      const int ux = ci[0] + ox;
      if (!S.pbc[0] && (ux < 0 || ux >= Cx)) continue;
      // image shift along x, in cells: C is a power of two on a periodic axis,
      // and an open axis only visits u in [0, C)
      const int wx = ux - ((ux >> S.cshift[0]) << S.cshift[0]);
      const float bx = (float)ox * ex - xi.x;  // d_x = bx + x_j
      const float mx = fmaxf((ox > 0 ? bx : (ox < 0 ? -(bx + ex) : 0.f)) - mg * ex, 0.f);
      for (int oy = -S.nnbr[1]; oy <= S.nnbr[1]; oy++) {
        const int uy = ci[1] + oy;
        if (!S.pbc[1] && (uy < 0 || uy >= Cy)) continue;
        const float by = (float)oy * ey - xi.y;
        const float my = fmaxf((oy > 0 ? by : (oy < 0 ? -(by + ey) : 0.f)) - mg * ey, 0.f);
        const float rxy2 = mx * mx + my * my;
        if (rxy2 >= a2) continue;
        const int wy = uy - ((uy >> S.cshift[1]) << S.cshift[1]);
        const float zr2 = a2 - rxy2;  // > 0
        const float zr = zr2 * rsqrt_nrm(zr2) + mg * S.edge[2];
        int zlo = (int)floorf((xi.z - zr) * inv_ez), zhi = (int)floorf((xi.z + zr) * inv_ez);
        if (!S.pbc[2]) {
          zlo = max(zlo, 0);
          zhi = min(zhi, Cz - 1);
        }
        const int colbase = S.cell_off + (wx * Cy + wy) * Cz;
        float sx = 0.f, sy = 0.f;  // sum of q_j k_0'(r)/r d_x, d_y over the column
        int uz = zlo;
        while (uz <= zhi) {
          const int kz = uz >> S.cshift[2];
          const int wz = uz - (kz << S.cshift[2]);
          const int wend = min(Cz - 1, wz + (zhi - uz));
          int jb = cell_start[colbase + wz], je = cell_start[colbase + wend + 1];
          if (!MSM_CHECK(S, jb >= S.atom_off && je <= S.atom_off + S.n)) je = jb;
          const float bz = image_shift(kz, S.Ld[2], xi.z);  // d_z = bz + z_j
          for (int j = jb; j < je; j++) {
            const float4 xj = xq[j];
            const float dx = bx + xj.x, dy = by + xj.y, dz = bz + xj.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < a2 && r2 > 0.f) {
              const float rinv = rsqrt_nrm(r2);
              const float s = 1.0f - r2 * inv_a2;
              float g = gc[P - 1];
#pragma unroll
              for (int t = P - 2; t >= 0; t--) g = fmaf(g, s, gc[t]);
              ph = fmaf(xj.w, rinv - g, ph);  // k_0 = 1/r - gamma(r/a)/a
              if (WF || WW) {
                float dg = gdc[P - 2];
#pragma unroll
                for (int t = P - 3; t >= 0; t--) dg = fmaf(dg, s, gdc[t]);
                // k_0'(r)/r = -1/r^3 + (2/a^3) d gamma/d s
                const float fr = xj.w * fmaf(-rinv * rinv, rinv, dg);
                if (WW) {
                  sx = fmaf(fr, dx, sx);
                  sy = fmaf(fr, dy, sy);
                  const float gz = fr * dz;
                  fz += gz;
                  v[2] = fmaf(gz, dz, v[2]);
                  v[4] = fmaf(gz, dx, v[4]);
                  v[5] = fmaf(gz, dy, v[5]);
                } else {
                  fx = fmaf(fr, dx, fx);
                  fy = fmaf(fr, dy, fy);
                  fz = fmaf(fr, dz, fz);
                }
              }
            }
          }
          uz += wend - wz + 1;
        }
        if (WW) {
          fx += sx;
          fy += sy;
          const float ty = (float)oy * ey;
          v[0] = fmaf(tx, sx, v[0]);
          v[1] = fmaf(ty, sy, v[1]);
          v[3] = fmaf(tx, sy, fmaf(ty, sx, v[3]));
        }
      }
    }
    phi_sr[k] = ph - xi.w * S.self_coef;
    if (WF) f_sr[k] = make_float4(fx, fy, fz, 0.f);  // field of the other charges; the force is q_i times it
    if (WW) {
      // xx, yy, xy: q_i (xi_i f_i^T) - 1/2 q_i sum_columns t (s_col)^T with xi_i the atom's
      // offset from its cell corner and t the offset between the cell corners; zz, xz, yz:
      // -1/2 q_i sum q_j k_0'(r)/r d d^T pair by pair
      const float hq = -0.5f * xi.w;
      w6[0] = xi.w * (xi.x * fx) + hq * v[0];
      w6[1] = xi.w * (xi.y * fy) + hq * v[1];
      w6[2] = hq * v[2];
      w6[3] = xi.w * (0.5f * (xi.x * fy + xi.y * fx)) + 0.5f * hq * v[3];
      w6[4] = hq * v[4];
      w6[5] = hq * v[5];
    }
  }
  if (!WW) return;
  // per-warp partials of the six virial components: FP32 across the warp's 32
  // atoms, FP64 from there on (fixed order, no block barrier)
  const int lane = threadIdx.x & 31, wid = slot >> 5;
#pragma unroll
  for (int c = 0; c < 6; c++) {
    float v = w6[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) part_w0[6 * ((long long)item * kChunkWarps + wid) + c] = (double)v;
  }
}

// Short-range part of the vector-Jacobian product of the forces (L =
// sum_k u_k . F_k for an upstream u, Sec. 3.2.2's derivatives taken once
// more): with p_b = q_b u_b, f1 = k_0'(r)/r and the pair Hessian
// H0(d) = f2 d d^T + f1 I, f2 = (k_0'' - k_0'/r)/r^2,
//   psi0_i = sum_(b,n) f1 p_b . d           (potential at r_i of the dipoles p_b),
//   h0_i   = sum_(b,n) q_b H0(d) (u_i - u_b) (the short-range rows of H u, / q_i),
// d = r_b + A n - r_i, over the same candidates as k_short. In s = 1 - r^2/a^2,
// f1 = -1/r^3 + sum_k gdca[k] s^k and f2 = 3/r^5 - (2/a^2) sum_k k gdca[k] s^(k-1).
// us holds (u, q) in the sorted order; out gets (h0, psi0).
template <int P>
__global__ void __launch_bounds__(kChunk) k_short_fvjp(const SysDev* __restrict__ sys,
                                                       const AtomItem* __restrict__ items,
                                                       const int* __restrict__ cell_start,
                                                       const int* __restrict__ scell, const float4* __restrict__ xq,
                                                       const float4* __restrict__ us, float4* __restrict__ out) {
  const AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  const int local = it.start + (int)threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  const int k = S.atom_off + local;
  const float4 xi = xq[k];
  const float4 ui = us[k];
  const int cell = scell[k];
  const int Cx = S.C[0], Cy = S.C[1], Cz = S.C[2];
  const int ci[3] = {cell / (Cy * Cz), (cell / Cz) % Cy, cell % Cz};
  float gdc[P - 1];
#pragma unroll
  for (int t = 0; t < P - 1; t++) gdc[t] = S.gdca[t];
  const float a2 = S.a2, inv_a2 = S.inv_a2;
  const float ex = S.edge[0], ey = S.edge[1], inv_ez = 1.0f / S.edge[2];
  constexpr float mg = 2e-4f;
  float psi = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
  for (int ox = -S.nnbr[0]; ox <= S.nnbr[0]; ox++) {
    const int ux = ci[0] + ox;
    if (!S.pbc[0] && (ux < 0 || ux >= Cx)) continue;
    const int wx = ux - floordiv_s(ux, Cx) * Cx;
    const float bx = (float)ox * ex - xi.x;
    const float mx = fmaxf((ox > 0 ? bx : (ox < 0 ? -(bx + ex) : 0.f)) - mg * ex, 0.f);
    for (int oy = -S.nnbr[1]; oy <= S.nnbr[1]; oy++) {
      const int uy = ci[1] + oy;
      if (!S.pbc[1] && (uy < 0 || uy >= Cy)) continue;
      const float by = (float)oy * ey - xi.y;
      const float my = fmaxf((oy > 0 ? by : (oy < 0 ? -(by + ey) : 0.f)) - mg * ey, 0.f);
      const float rxy2 = mx * mx + my * my;
      if (rxy2 >= a2) continue;
      const int wy = uy - floordiv_s(uy, Cy) * Cy;
      const float zr2 = a2 - rxy2;  // > 0
      const float zr = zr2 * rsqrt_nrm(zr2) + mg * S.edge[2];
      int zlo = (int)floorf((xi.z - zr) * inv_ez), zhi = (int)floorf((xi.z + zr) * inv_ez);
      if (!S.pbc[2]) {
        zlo = max(zlo, 0);
        zhi = min(zhi, Cz - 1);
      }
      const int colbase = S.cell_off + (wx * Cy + wy) * Cz;
      int uz = zlo;
      while (uz <= zhi) {
        const int kz = floordiv_s(uz, Cz);
        const int wz = uz - kz * Cz;
        const int wend = min(Cz - 1, wz + (zhi - uz));
        int jb = cell_start[colbase + wz], je = cell_start[colbase + wend + 1];
        if (!MSM_CHECK(S, jb >= S.atom_off && je <= S.atom_off + S.n)) je = jb;
        const float bz = image_shift(kz, S.Ld[2], xi.z);
        for (int j = jb; j < je; j++) {
          const float4 xj = xq[j];
          const float dx = bx + xj.x, dy = by + xj.y, dz = bz + xj.z;
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < a2 && r2 > 0.f) {
            const float4 uj = us[j];
            const float rinv = rsqrt_nrm(r2);
            const float rinv2 = rinv * rinv;
            const float s = 1.0f - r2 * inv_a2;
            float p1 = gdc[P - 2], dp1 = (float)(P - 2) * gdc[P - 2];
#pragma unroll
            for (int c = P - 3; c >= 0; c--) {
              p1 = fmaf(p1, s, gdc[c]);
              if (c >= 1) dp1 = fmaf(dp1, s, (float)c * gdc[c]);
            }
            if (P - 2 < 1) dp1 = 0.f;
            const float f1 = fmaf(-rinv2, rinv, p1);
            const float f2 = fmaf(3.0f * rinv2 * rinv2, rinv, -2.0f * inv_a2 * dp1);
            // dipole potential p_b . d f1
            psi = fmaf(f1 * uj.w, uj.x * dx + uj.y * dy + uj.z * dz, psi);
            // q_b H0(d) (u_i - u_b)
            const float wxv = ui.x - uj.x, wyv = ui.y - uj.y, wzv = ui.z - uj.z;
            const float dw = f2 * (dx * wxv + dy * wyv + dz * wzv);
            hx = fmaf(uj.w, fmaf(dw, dx, f1 * wxv), hx);
            hy = fmaf(uj.w, fmaf(dw, dy, f1 * wyv), hy);
            hz = fmaf(uj.w, fmaf(dw, dz, f1 * wzv), hz);
          }
        }
        uz += wend - wz + 1;
      }
    }
  }
  out[k] = make_float4(hx, hy, hz, psi);
}

// k_short_fvjp over the candidates of k_short_tri (tilted cells)
template <int P>
__global__ void __launch_bounds__(kChunk) k_short_fvjp_tri(const SysDev* __restrict__ sys,
                                                           const AtomItem* __restrict__ items,
                                                           const int* __restrict__ cell_start,
                                                           const int* __restrict__ scell,
                                                           const float4* __restrict__ xq, const float4* __restrict__ uq,
                                                           const float4* __restrict__ us, float4* __restrict__ out) {
  const AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  const int local = it.start + (int)threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  const int k = S.atom_off + local;
  const float4 xi = xq[k];
  const float4 ui = us[k];
  const float siz = uq[k].z / S.Mf[2];
  const int cell = scell[k];
  const int Cx = S.C[0], Cy = S.C[1], Cz = S.C[2];
  const int ci[3] = {cell / (Cy * Cz), (cell / Cz) % Cy, cell % Cz};
  float gdc[P - 1];
#pragma unroll
  for (int t = 0; t < P - 1; t++) gdc[t] = S.gdca[t];
  const float a2 = S.a2, inv_a2 = S.inv_a2;
  const double ta[3] = {S.Ad[0] / Cx, S.Ad[1] / Cx, S.Ad[2] / Cx}, tb[3] = {S.Ad[3] / Cy, S.Ad[4] / Cy, S.Ad[5] / Cy};
  const float rz = S.reach[2] + 2e-4f / Cz;
  const int zlo = (int)floorf((siz - rz) * Cz), zhi = (int)floorf((siz + rz) * Cz);
  float psi = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
  for (int ox = -S.nnbr[0]; ox <= S.nnbr[0]; ox++) {
    const int ux = ci[0] + ox;
    const int wx = ux - floordiv_s(ux, Cx) * Cx;
    for (int oy = -S.nnbr[1]; oy <= S.nnbr[1]; oy++) {
      const int uy = ci[1] + oy;
      const int wy = uy - floordiv_s(uy, Cy) * Cy;
      const int colbase = S.cell_off + (wx * Cy + wy) * Cz;
      double bxy[3];
      for (int e = 0; e < 3; e++) bxy[e] = ox * ta[e] + oy * tb[e];
      int uz = zlo;
      while (uz <= zhi) {
        const int kz = floordiv_s(uz, Cz);
        const int wz = uz - kz * Cz;
        const int wend = min(Cz - 1, wz + (zhi - uz));
        int jb = cell_start[colbase + wz], je = cell_start[colbase + wend + 1];
        if (!MSM_CHECK(S, jb >= S.atom_off && je <= S.atom_off + S.n)) je = jb;
        const float bx = (float)(bxy[0] + kz * S.Ad[6] - (double)xi.x);
        const float by = (float)(bxy[1] + kz * S.Ad[7] - (double)xi.y);
        const float bz = (float)(bxy[2] + kz * S.Ad[8] - (double)xi.z);
        for (int j = jb; j < je; j++) {
          const float4 xj = xq[j];
          const float dx = bx + xj.x, dy = by + xj.y, dz = bz + xj.z;
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < a2 && r2 > 0.f) {
            const float4 uj = us[j];
            const float rinv = rsqrt_nrm(r2);
            const float rinv2 = rinv * rinv;
            const float sg = 1.0f - r2 * inv_a2;
            float p1 = gdc[P - 2], dp1 = (float)(P - 2) * gdc[P - 2];
#pragma unroll
            for (int c = P - 3; c >= 0; c--) {
              p1 = fmaf(p1, sg, gdc[c]);
              if (c >= 1) dp1 = fmaf(dp1, sg, (float)c * gdc[c]);
            }
            const float f1 = fmaf(-rinv2, rinv, p1);
            const float f2 = fmaf(3.0f * rinv2 * rinv2, rinv, -2.0f * inv_a2 * dp1);
            psi = fmaf(f1 * uj.w, uj.x * dx + uj.y * dy + uj.z * dz, psi);
            const float wxv = ui.x - uj.x, wyv = ui.y - uj.y, wzv = ui.z - uj.z;
            const float dw = f2 * (dx * wxv + dy * wyv + dz * wzv);
            hx = fmaf(uj.w, fmaf(dw, dx, f1 * wxv), hx);
            hy = fmaf(uj.w, fmaf(dw, dy, f1 * wyv), hy);
            hz = fmaf(uj.w, fmaf(dw, dz, f1 * wzv), hz);
          }
        }
        uz += wend - wz + 1;
      }
    }
  }
  out[k] = make_float4(hx, hy, hz, psi);
}

void launch_short_fvjp(const Work& w, const Tables& t, const AtomItem* items, int nitems, const float4* us,
                       float4* out, cudaStream_t s, int p, bool tilted) {
  if (tilted) {
    switch (p) {
      case 4: k_short_fvjp_tri<4><<<nitems, kChunk, 0, s>>>(t.sys, items, w.cell_start, w.scell, w.xq, w.uq, us, out); break;
      case 6: k_short_fvjp_tri<6><<<nitems, kChunk, 0, s>>>(t.sys, items, w.cell_start, w.scell, w.xq, w.uq, us, out); break;
      default: k_short_fvjp_tri<8><<<nitems, kChunk, 0, s>>>(t.sys, items, w.cell_start, w.scell, w.xq, w.uq, us, out); break;
    }
    return;
  }
  switch (p) {
    case 4: k_short_fvjp<4><<<nitems, kChunk, 0, s>>>(t.sys, items, w.cell_start, w.scell, w.xq, us, out); break;
    case 6: k_short_fvjp<6><<<nitems, kChunk, 0, s>>>(t.sys, items, w.cell_start, w.scell, w.xq, us, out); break;
    default: k_short_fvjp<8><<<nitems, kChunk, 0, s>>>(t.sys, items, w.cell_start, w.scell, w.xq, us, out); break;
  }
}

// General-cell variant (tilted periodic cells; correct for rectangular cells
// too): positions are Cartesian offsets from the base c_x/C_x a + c_y/C_y b of
// the atom's cell column, so the displacement to a candidate of column
// (c_x + ox, c_y + oy) at z image kz is ox a/C_x + oy b/C_y + kz c + x_j - x_i,
// the shift formed in FP64 once per run. A point within a of atom i has
// |s_d - s_i,d| <= a / w_d (w_d the distance between the cell faces across d),
// so every column within nnbr cells and, in each, the z cells within that
// reach are visited; the pair test selects. The virial uses the same identity
// as k_short, the image term (A n) s^T with A n = n_x a + n_y b + kz c.
template <int P, bool WF, bool WW>
__global__ void __launch_bounds__(kChunk) k_short_tri(const SysDev* __restrict__ sys,
                                                      const AtomItem* __restrict__ items,
                                                      const int* __restrict__ cell_start,
                                                      const int* __restrict__ scell, const float4* __restrict__ xq,
                                                      const float4* __restrict__ uq, float* __restrict__ phi_sr,
                                                      float4* __restrict__ f_sr, double* __restrict__ part_w0) {
  const int item = blockIdx.x;
  AtomItem it = items[item];
  const SysDev& S = sys[it.sys];
  const int slot = (int)threadIdx.x;
  const int local = it.start + slot;
  const bool active = slot < it.count && local < S.n;
  float w6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (active) {
    const int k = S.atom_off + local;
    const float4 xi = xq[k];
    const float siz = uq[k].z / S.Mf[2];
    const int cell = scell[k];
    const int Cx = S.C[0], Cy = S.C[1], Cz = S.C[2];
    const int ci[3] = {cell / (Cy * Cz), (cell / Cz) % Cy, cell % Cz};
    float gc[P], gdc[P - 1];
#pragma unroll
    for (int t = 0; t < P; t++) gc[t] = S.gca[t];
#pragma unroll
    for (int t = 0; t < P - 1; t++) gdc[t] = S.gdca[t];
    const float a2 = S.a2, inv_a2 = S.inv_a2;
    const double ta[3] = {S.Ad[0] / Cx, S.Ad[1] / Cx, S.Ad[2] / Cx}, tb[3] = {S.Ad[3] / Cy, S.Ad[4] / Cy, S.Ad[5] / Cy};
    const float rz = S.reach[2] + 2e-4f / Cz;  // fractional reach along c, with a rounding margin
    int zlo = (int)floorf((siz - rz) * Cz), zhi = (int)floorf((siz + rz) * Cz);
    float ph = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
    float img[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int ox = -S.nnbr[0]; ox <= S.nnbr[0]; ox++) {
      const int ux = ci[0] + ox;
      const int nxw = floordiv_s(ux, Cx), wx = ux - nxw * Cx;
      for (int oy = -S.nnbr[1]; oy <= S.nnbr[1]; oy++) {
        const int uy = ci[1] + oy;
        const int nyw = floordiv_s(uy, Cy), wy = uy - nyw * Cy;
        const int colbase = S.cell_off + (wx * Cy + wy) * Cz;
        double bxy[3];
        for (int e = 0; e < 3; e++) bxy[e] = ox * ta[e] + oy * tb[e];
        int uz = zlo;
        while (uz <= zhi) {
          const int kz = floordiv_s(uz, Cz);
          const int wz = uz - kz * Cz;
          const int wend = min(Cz - 1, wz + (zhi - uz));
          int jb = cell_start[colbase + wz], je = cell_start[colbase + wend + 1];
          if (!MSM_CHECK(S, jb >= S.atom_off && je <= S.atom_off + S.n)) je = jb;
          const float bx = (float)(bxy[0] + kz * S.Ad[6] - (double)xi.x);
          const float by = (float)(bxy[1] + kz * S.Ad[7] - (double)xi.y);
          const float bz = (float)(bxy[2] + kz * S.Ad[8] - (double)xi.z);
          float sx = 0.f, sy = 0.f, sz = 0.f;
          for (int j = jb; j < je; j++) {
            const float4 xj = xq[j];
            const float dx = bx + xj.x, dy = by + xj.y, dz = bz + xj.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < a2 && r2 > 0.f) {
              const float rinv = rsqrt_nrm(r2);
              const float sg = 1.0f - r2 * inv_a2;
              float g = gc[P - 1];
#pragma unroll
              for (int t = P - 2; t >= 0; t--) g = fmaf(g, sg, gc[t]);
              ph = fmaf(xj.w, rinv - g, ph);
              if (WF || WW) {
                float dg = gdc[P - 2];
#pragma unroll
                for (int t = P - 3; t >= 0; t--) dg = fmaf(dg, sg, gdc[t]);
                const float fr = xj.w * fmaf(-rinv * rinv, rinv, dg);
                sx = fmaf(fr, dx, sx);
                sy = fmaf(fr, dy, sy);
                sz = fmaf(fr, dz, sz);
              }
            }
          }
          fx += sx;
          fy += sy;
          fz += sz;
          if (WW && (nxw | nyw | kz) != 0) {
            float tv[3];
            for (int e = 0; e < 3; e++) tv[e] = (float)(nxw * S.Ad[e] + nyw * S.Ad[3 + e] + kz * S.Ad[6 + e]);
            img[0] = fmaf(tv[0], sx, img[0]);
            img[1] = fmaf(tv[1], sy, img[1]);
            img[2] = fmaf(tv[2], sz, img[2]);
            img[3] = fmaf(0.5f * tv[0], sy, fmaf(0.5f * tv[1], sx, img[3]));
            img[4] = fmaf(0.5f * tv[0], sz, fmaf(0.5f * tv[2], sx, img[4]));
            img[5] = fmaf(0.5f * tv[1], sz, fmaf(0.5f * tv[2], sy, img[5]));
          }
          uz += wend - wz + 1;
        }
      }
    }
    phi_sr[k] = ph - xi.w * S.self_coef;
    if (WF) f_sr[k] = make_float4(fx, fy, fz, 0.f);
    if (WW) {
      // r_i in the frame of the displacements: the column base plus the offset
      float r[3];
      for (int e = 0; e < 3; e++)
        r[e] = (float)(ci[0] * ta[e] + ci[1] * tb[e] + (double)(e == 0 ? xi.x : (e == 1 ? xi.y : xi.z)));
      const float hq = -0.5f * xi.w;
      w6[0] = xi.w * (r[0] * fx) + hq * img[0];
      w6[1] = xi.w * (r[1] * fy) + hq * img[1];
      w6[2] = xi.w * (r[2] * fz) + hq * img[2];
      w6[3] = xi.w * (0.5f * (r[0] * fy + r[1] * fx)) + hq * img[3];
      w6[4] = xi.w * (0.5f * (r[0] * fz + r[2] * fx)) + hq * img[4];
      w6[5] = xi.w * (0.5f * (r[1] * fz + r[2] * fy)) + hq * img[5];
    }
  }
  if (!WW) return;
  const int lane = threadIdx.x & 31, wid = slot >> 5;
#pragma unroll
  for (int c = 0; c < 6; c++) {
    double v = (double)w6[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) part_w0[6 * ((long long)item * kChunkWarps + wid) + c] = v;
  }
}

template <int P>
static void run_short_tri(const Work& w, const Tables& t, const AtomItem* items, int nitems, bool forces, bool virial,
                          cudaStream_t s) {
  auto kern = virial ? (forces ? k_short_tri<P, true, true> : k_short_tri<P, false, true>)
                     : (forces ? k_short_tri<P, true, false> : k_short_tri<P, false, false>);
  kern<<<nitems, kChunk, 0, s>>>(t.sys, items, w.cell_start, w.scell, w.xq, w.uq, w.phi_sr, w.f_sr, w.part_w0);
}

template <int P, int NB>
static void run_short_nb(const Work& w, const Tables& t, const AtomItem* items, int nitems, bool forces, bool virial,
                         cudaStream_t s) {
  auto kern = virial ? (forces ? k_short<P, true, true, NB> : k_short<P, false, true, NB>)
                     : (forces ? k_short<P, true, false, NB> : k_short<P, false, false, NB>);
  kern<<<nitems * (kChunk / NB), NB, 0, s>>>(t.sys, items, w.cell_start, w.scell, w.xq, w.phi_sr, w.f_sr,
                                             w.part_w0);
}

template <int P>
static void run_short(const Work& w, const Tables& t, const AtomItem* items, int nitems, bool forces, bool virial,
                      cudaStream_t s, int block) {
  if (block == kShortTilted) run_short_tri<P>(w, t, items, nitems, forces, virial, s);
  else if (block == kShortCluster) launch_short_cluster(w, t, items, nitems, forces, virial, s, P);
  else if (block == kChunk / 2) run_short_nb<P, kChunk / 2>(w, t, items, nitems, forces, virial, s);
  else run_short_nb<P, kChunk>(w, t, items, nitems, forces, virial, s);
}

// block: threads per block of the rectangular-cell kernel (kChunk or kChunk / 2), kShortCluster
// (cluster-pair tiles, k_short_cl.cu) or kShortTilted
void launch_short(const Work& w, const Tables& t, const AtomItem* items, int nitems, bool forces, bool virial,
                  cudaStream_t s, int p, int block) {
  switch (p) {
    case 4: run_short<4>(w, t, items, nitems, forces, virial, s, block); break;
    case 6: run_short<6>(w, t, items, nitems, forces, virial, s, block); break;
    default: run_short<8>(w, t, items, nitems, forces, virial, s, block); break;
  }
}

}  // namespace msm
