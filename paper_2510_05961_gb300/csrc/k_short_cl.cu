// k_short_cl.cu -- the short-range sums of Eq. U_zero (phi^0, the field
// -grad phi^0 and the virial W^0, the same quantities as k_short) organised as
// cluster-pair tiles, for rectangular cells.
//
// One warp takes i-clusters of 4 consecutive sorted atoms of one binning
// column (a cluster that straddles two columns is taken as one segment per
// column). For a cluster it
//  1. finds its candidate runs: every (ox, oy) column within the cutoff of the
//     cluster's bounding box and, in each, the z cells within reach of the box,
//     one run of consecutive sorted atoms per periodic z image; each lane
//     computes the runs of one column, and a warp scan lays them out one after
//     the other, so the candidates of all runs form one flat index range;
//  2. walks that range 32 candidates at a time, one per lane (the lane finds
//     its run from the run starts that fall in the chunk: an OR-reduction of
//     one bit per run start and a population count), shifts the candidate into
//     the cluster's frame (the column offset ox e_x, oy e_y; along z the image
//     kz L_z minus the z of one cluster atom, formed in FP64 and rounded once),
//     and keeps it when it lies within a of the bounding box; kept candidates go
//     to a per-warp queue in shared memory (ballot + prefix count);
//  3. evaluates the queue as 4 x 8 tiles: lane (il, jl) = (lane & 3, lane >> 2)
//     takes i-atom il and queue entry 8 t + jl, so every lane computes a pair
//     in every step; pairs outside the cutoff (about 43% of the tile at the
//     1M-atom density) and the self pair (d = 0 exactly) are weighted by zero;
//  4. reduces each i-atom's sums over its 8 lanes by shuffles.
// Each lane sums its own pairs in a fixed order, so results do not depend on
// scheduling. The virial is summed pair by pair (-1/2 q_i q_j k_0'(r)/r d d^T,
// every term bounded by a^2 |g|), FP32 per lane, FP32 across the warp, FP64 per
// warp partial, in the partial layout of k_short.
//
// The bounding-box test and the pair test compute the squared distance with
// the same operations in the same order on the same FP32 values, and the box
// distance is no larger than any atom's distance along each axis, so rounding
// is monotone between them: no pair that passes the pair test is culled.
//
// Plans may use this kernel when every system is rectangular, reaches at most
// 4 binning columns along x and y (nnbr <= 4) and, along a periodic z axis,
// has L_z >= a + 2 e_z, so one column needs at most 3 z images (kz = -1, 0, 1).
#include "msm_internal.h"

namespace msm {

namespace {
constexpr int kClI = 4;                   // i-atoms per cluster
constexpr int kClJ = 8;                   // queue entries per tile step
constexpr int kClFlush = 128;             // queue length that triggers tile steps
constexpr int kClQ = kClFlush + 32;       // queue capacity (a chunk adds at most 32)
constexpr int kClRun = 3;                 // runs (z images) per column
constexpr int kClRunCap = 32 * kClRun;    // run table of one pass over 32 columns
constexpr float kFar = 1e18f;             // coordinate of padding entries: every pair fails the cutoff test
}  // namespace

// pair sums of lane (il, jl) over queue entries [0, n), n a multiple of kClJ
template <int P, bool WF, bool WW>
__device__ __forceinline__ void cl_tiles(const float4* __restrict__ Q, int n, int jl, float4 xi, const float (&gc)[P],
                                         const float (&gdc)[P - 1], float a2, float inv_a2, float& ph, float& fx,
                                         float& fy, float& fz, float (&v)[6]) {
#pragma unroll 1
  for (int e = jl; e < n; e += kClJ) {
    const float4 xj = Q[e];
    const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool in = r2 < a2 && r2 > 0.f;
    const float rs = in ? r2 : a2;
    const float qj = in ? xj.w : 0.f;
    const float rinv = rsqrt_nrm(rs);
    const float sg = fmaf(-rs, inv_a2, 1.0f);
    float g = gc[P - 1];
#pragma unroll
    for (int t = P - 2; t >= 0; t--) g = fmaf(g, sg, gc[t]);
    ph = fmaf(qj, rinv - g, ph);  // k_0 = 1/r - gamma(r/a)/a
    if (WF || WW) {
      float dg = gdc[P - 2];
#pragma unroll
      for (int t = P - 3; t >= 0; t--) dg = fmaf(dg, sg, gdc[t]);
      // q_j k_0'(r)/r = q_j (-1/r^3 + (2/a^3) d gamma / d s)
      const float fr = qj * fmaf(-rinv * rinv, rinv, dg);
      const float gx = fr * dx, gy = fr * dy, gz = fr * dz;
      fx += gx;
      fy += gy;
      fz += gz;
      if (WW) {
        v[0] = fmaf(gx, dx, v[0]);
        v[1] = fmaf(gy, dy, v[1]);
        v[2] = fmaf(gz, dz, v[2]);
        v[3] = fmaf(gx, dy, v[3]);
        v[4] = fmaf(gz, dx, v[4]);
        v[5] = fmaf(gz, dy, v[5]);
      }
    }
  }
}

// one block per atom item (kChunk atoms, kChunkWarps warps); warp w takes the
// item's atoms [32 w, 32 w + 32) as 8 clusters
template <int P, bool WF, bool WW>
__global__ void __launch_bounds__(kChunk, 3) k_short_cl(const SysDev* __restrict__ sys, const AtomItem* __restrict__ items,
                                                        const int* __restrict__ cell_start, const int* __restrict__ scell,
                                                        const float4* __restrict__ xq, float* __restrict__ phi_sr,
                                                        float4* __restrict__ f_sr, double* __restrict__ part_w0) {
  __shared__ float4 s_q[kChunkWarps][kClQ];         // queued candidates: (position in the cluster's frame, q)
  __shared__ float4 s_rt[kChunkWarps][kClRunCap];   // runs: (tx, ty, tz, first sorted atom - first flat index)
  __shared__ int s_ro[kChunkWarps][kClRunCap];      // runs: first flat index
  __shared__ float s_w6[kChunkWarps][6][32];         // per-lane virial sums (kept out of registers)
  const int item = blockIdx.x;
  const AtomItem it = items[item];
  const SysDev& S = sys[it.sys];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int il = lane & (kClI - 1), jl = lane >> 2;
  float4* Q = s_q[wid];
  float4* RT = s_rt[wid];
  int* RO = s_ro[wid];
  const unsigned kAll = 0xffffffffu;
  const unsigned lt_mask = (1u << lane) - 1u, le_mask = (2u << lane) - 1u;

  float gc[P], gdc[P - 1];
#pragma unroll
  for (int t = 0; t < P; t++) gc[t] = S.gca[t];
#pragma unroll
  for (int t = 0; t < P - 1; t++) gdc[t] = S.gdca[t];
  const float a2 = S.a2, inv_a2 = S.inv_a2;
  const float ex = S.edge[0], ey = S.edge[1], ez = S.edge[2], inv_ez = 1.0f / ez;
  const int Cx = S.C[0], Cy = S.C[1], Cz = S.C[2];
  const int nx = S.nnbr[0], ny = S.nnbr[1], wy2 = 2 * ny + 1;
  const int ncol = (2 * nx + 1) * wy2;
  constexpr float mg = 2e-4f;  // culling margin in cell edges (binning rounding), as in k_short

  if (WW)
#pragma unroll
    for (int c = 0; c < 6; c++) s_w6[wid][c][lane] = 0.f;
  const int wbeg = 32 * wid;
  const int slot_end = min(min(it.count, S.n - it.start), wbeg + 32);
  for (int c0 = wbeg; c0 < slot_end; c0 += kClI) {
    const int cn = min(kClI, slot_end - c0);
    const bool iv = il < cn;
    const int ki = S.atom_off + it.start + c0 + min(il, cn - 1);
    const float4 xraw = xq[ki];
    const int col_i = scell[ki] / Cz;  // cx * Cy + cy
    int seg = 0;
    while (seg < cn) {
      // the atoms of this segment share a binning column (sorted order: contiguous)
      const int col = __shfl_sync(kAll, col_i, seg);
      const unsigned same = __ballot_sync(kAll, iv && il >= seg && col_i == col) & 0xFu;
      const bool act = ((same >> il) & 1u) != 0u;
      // the cluster's frame: x, y from the cell corner (as stored), z from zref,
      // the z of one of its atoms (differences of nearby z values stay exact)
      const float zref = __shfl_sync(kAll, xraw.z, seg);
      const float4 xi = act ? make_float4(xraw.x, xraw.y, xraw.z - zref, xraw.w) : make_float4(kFar, kFar, kFar, 0.f);
      float lo[3] = {act ? xi.x : INFINITY, act ? xi.y : INFINITY, act ? xi.z : INFINITY};
      float hi[3] = {act ? xi.x : -INFINITY, act ? xi.y : -INFINITY, act ? xi.z : -INFINITY};
#pragma unroll
      for (int o = 1; o < kClI; o <<= 1)
#pragma unroll
        for (int d = 0; d < 3; d++) {
          lo[d] = fminf(lo[d], __shfl_xor_sync(kAll, lo[d], o));
          hi[d] = fmaxf(hi[d], __shfl_xor_sync(kAll, hi[d], o));
        }
      const int cx = col / Cy, cy = col - (col / Cy) * Cy;
      float ph = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
      float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      // queue, run table and candidate walk, as one loop with one tile call site:
      // a pass builds the runs of 32 neighbour columns, a chunk queues the kept
      // candidates among 32 of them, and tile steps run whenever the queue holds
      // kClFlush entries and once at the end over the padded rest
      int qn = 0;  // queued entries (same in every lane)
      int pass = 0, cb = 0, T = 0, R = 0, r0 = -1;
      bool done = false;
      while (true) {
        if (cb >= T) {
          if (pass * 32 >= ncol) {
            done = true;
          } else {
            // 1. runs of this lane's neighbour column
            int rjb[kClRun], rn[kClRun];
            float rtz[kClRun];
#pragma unroll
            for (int r = 0; r < kClRun; r++) {
              rjb[r] = 0;
              rn[r] = 0;
              rtz[r] = 0.f;
            }
            float tx = 0.f, ty = 0.f;
            const int cidx = pass * 32 + lane;
            if (cidx < ncol) {
              const int ox = cidx / wy2 - nx, oy = cidx - (cidx / wy2) * wy2 - ny;
              const int ux = cx + ox, uy = cy + oy;
              const bool exists = (S.pbc[0] || (ux >= 0 && ux < Cx)) && (S.pbc[1] || (uy >= 0 && uy < Cy));
              tx = (float)ox * ex;
              ty = (float)oy * ey;
              // distance in x and y from the bounding box to the column [tx, tx + ex] x [ty, ty + ey]
              const float mx = fmaxf((ox > 0 ? tx - hi[0] : (ox < 0 ? lo[0] - (tx + ex) : 0.f)) - mg * ex, 0.f);
              const float my = fmaxf((oy > 0 ? ty - hi[1] : (oy < 0 ? lo[1] - (ty + ey) : 0.f)) - mg * ey, 0.f);
              const float rxy2 = mx * mx + my * my;
              if (exists && rxy2 < a2) {
                const int wx = ux - ((ux >> S.cshift[0]) << S.cshift[0]);
                const int wy = uy - ((uy >> S.cshift[1]) << S.cshift[1]);
                const float zr2 = a2 - rxy2;
                const float zr = zr2 * rsqrt_nrm(zr2) + mg * ez;
                int zlo = (int)floorf((lo[2] + zref - zr) * inv_ez), zhi = (int)floorf((hi[2] + zref + zr) * inv_ez);
                if (!S.pbc[2]) {
                  zlo = max(zlo, 0);
                  zhi = min(zhi, Cz - 1);
                }
                const int colbase = S.cell_off + (wx * Cy + wy) * Cz;
                const int czs = S.cshift[2];
                int uz = zlo;
#pragma unroll
                for (int r = 0; r < kClRun; r++) {
                  if (uz <= zhi) {
                    const int kz = uz >> czs;
                    const int wz = uz - (kz << czs);
                    const int wend = min(Cz - 1, wz + (zhi - uz));
                    int jb = cell_start[colbase + wz], je = cell_start[colbase + wend + 1];
                    if (!MSM_CHECK(S, jb >= S.atom_off && je <= S.atom_off + S.n && je >= jb)) je = jb;
                    rjb[r] = jb;
                    rn[r] = je - jb;
                    rtz[r] = (float)(kz * S.Ld[2] - (double)zref);  // image shift into the cluster's frame, rounded once
                    uz += wend - wz + 1;
                  }
                }
                if (!MSM_CHECK(S, uz > zhi)) rn[0] = rn[1] = rn[2] = 0;  // more z images than the plan allows
              }
            }
            // 2. lay the non-empty runs out one after the other (packed scan: runs << 24 | candidates)
            int nr = 0, nc = 0;
#pragma unroll
            for (int r = 0; r < kClRun; r++) {
              nr += rn[r] > 0 ? 1 : 0;
              nc += rn[r];
            }
            int incl = (nr << 24) | nc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int y = __shfl_up_sync(kAll, incl, o);
              if (lane >= o) incl += y;
            }
            const int tot = __shfl_sync(kAll, incl, 31);
            R = tot >> 24;
            T = tot & 0xffffff;
            int rbase = (incl >> 24) - nr, cbase = (incl & 0xffffff) - nc;
            __syncwarp();  // the previous pass's chunks have read the run table
#pragma unroll
            for (int r = 0; r < kClRun; r++) {
              if (rn[r] > 0) {
                RT[rbase] = make_float4(tx, ty, rtz[r], __int_as_float(rjb[r] - cbase));
                RO[rbase] = cbase;
                rbase++;
                cbase += rn[r];
              }
            }
            __syncwarp();
            pass++;
            cb = 0;
            r0 = -1;
            continue;
          }
        }
        if (!done) {
          // 3. candidates cb .. cb + 31, one per lane; kept ones are queued in the cluster's frame
          const int rr = r0 + 1 + lane;
          unsigned bit = 0u;
          if (rr < R) {
            const int o = RO[rr];
            if (o < cb + 32) bit = 1u << (o - cb);
          }
          const unsigned starts = __reduce_or_sync(kAll, bit);
          const int myr = r0 + __popc(starts & le_mask);
          r0 += __popc(starts);
          const int c = cb + lane;
          bool keep = false;
          float4 xj = make_float4(0.f, 0.f, 0.f, 0.f);
          if (c < T) {
            const float4 rt = RT[myr];
            xj = xq[__float_as_int(rt.w) + c];
            xj.x += rt.x;
            xj.y += rt.y;
            xj.z += rt.z;
            const float ux = fmaxf(fmaxf(lo[0] - xj.x, xj.x - hi[0]), 0.f);
            const float uy = fmaxf(fmaxf(lo[1] - xj.y, xj.y - hi[1]), 0.f);
            const float uzv = fmaxf(fmaxf(lo[2] - xj.z, xj.z - hi[2]), 0.f);
            keep = fmaf(ux, ux, fmaf(uy, uy, uzv * uzv)) < a2;
          }
          const unsigned km = __ballot_sync(kAll, keep);
          if (keep) Q[qn + __popc(km & lt_mask)] = xj;
          qn += __popc(km);
          cb += 32;
          if (qn < kClFlush) continue;
        }
        // 4. tile steps over the queue: whole steps, or at the end the rest padded
        int n8 = qn & ~(kClJ - 1);
        if (done) {
          n8 = (qn + kClJ - 1) & ~(kClJ - 1);
          if (lane < n8 - qn) Q[qn + lane] = make_float4(kFar, kFar, kFar, 0.f);
        }
        __syncwarp();
        cl_tiles<P, WF, WW>(Q, n8, jl, xi, gc, gdc, a2, inv_a2, ph, fx, fy, fz, v);
        __syncwarp();
        if (done) break;
        const int rem = qn - n8;
        float4 tmp = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane < rem) tmp = Q[n8 + lane];
        __syncwarp();
        if (lane < rem) Q[lane] = tmp;
        __syncwarp();
        qn = rem;
      }
      // 5. each i-atom's sums over its 8 lanes
#pragma unroll
      for (int o = kClI; o < 32; o <<= 1) {
        ph += __shfl_xor_sync(kAll, ph, o);
        fx += __shfl_xor_sync(kAll, fx, o);
        fy += __shfl_xor_sync(kAll, fy, o);
        fz += __shfl_xor_sync(kAll, fz, o);
      }
      if (act && jl == 0) {
        phi_sr[ki] = ph - xraw.w * S.self_coef;
        if (WF) f_sr[ki] = make_float4(fx, fy, fz, 0.f);  // field of the other charges; the force is q_i times it
      }
      if (WW && act) {
        const float hq = -0.5f * xraw.w;
#pragma unroll
        for (int c = 0; c < 6; c++) s_w6[wid][c][lane] = fmaf(hq, v[c], s_w6[wid][c][lane]);
      }
      seg += __popc(same);
    }
  }
  if (!WW) return;
  // per-warp partials of the six virial components (xx yy zz xy xz yz)
#pragma unroll
  for (int c = 0; c < 6; c++) {
    float x = s_w6[wid][c][lane];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kAll, x, o);
    if (lane == 0) part_w0[6 * ((long long)item * kChunkWarps + wid) + c] = (double)x;
  }
}

void launch_short_cluster(const Work& w, const Tables& t, const AtomItem* items, int nitems, bool forces,
                          bool virial, cudaStream_t s, int p) {
#define MSM_CL(PP)                                                                                         \
  {                                                                                                        \
    auto kern = virial ? (forces ? k_short_cl<PP, true, true> : k_short_cl<PP, false, true>)               \
                       : (forces ? k_short_cl<PP, true, false> : k_short_cl<PP, false, false>);            \
    kern<<<nitems, kChunk, 0, s>>>(t.sys, items, w.cell_start, w.scell, w.xq, w.phi_sr, w.f_sr, w.part_w0); \
  }
  switch (p) {
    case 4: MSM_CL(4) break;
    case 6: MSM_CL(6) break;
    default: MSM_CL(8) break;
  }
#undef MSM_CL
}

}  // namespace msm
