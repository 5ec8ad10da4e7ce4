// k_bin.cu -- cell-list binning by a stable counting sort (all systems of a
// batch in one set of launches).
//
// Cell-index contract (bit-exact, FP32, round-to-nearest, no contraction):
//   s = x * (float)(1/L) (tilted cells: s_d = ((T_d0 x + T_d1 y) + T_d2 z),
//   T = (float) A^-T); periodic: s -= floorf(s), s >= 1 -> 0;
//   open: s outside [0,1] -> MSM_DEV_OUT_OF_CELL (axis cell 0);
//   c = min((int)(s * (float)C), C-1); cell = (cx*Cy + cy)*Cz + cz.
// Within a cell the sorted order is ascending atom index (stable), so the
// sorted arrays are identical from run to run.
//
// Pipeline: count (atomic slot per atom) -> exclusive scan of the packed cell
// counts of all systems -> scatter atom ids into buckets -> rank each atom in
// its bucket by original index and write the sorted arrays. The rank scan
// costs n_c^2 comparisons per cell of n_c atoms; the short-range kernel
// already tests every ordered pair of a cell's atoms (a cell is in its own
// neighbourhood), so binning never costs more than a fraction of it, whatever
// the clustering.
#include "msm_internal.h"

namespace msm {

__global__ void k_prologue(int* __restrict__ cell_count, int total_cells, int* __restrict__ status,
                           SysDev* __restrict__ sys, int nsys, int n_single) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int c = t; c < total_cells; c += gridDim.x * blockDim.x) cell_count[c] = 0;
  for (int s = t; s < nsys; s += gridDim.x * blockDim.x) sys[s].status = status;
  if (t == 0) {
    *status = 0;
    if (n_single >= 0) sys[0].n = n_single;
  }
}

// FP32 reduced coordinate s of one axis (the contract above); returns the
// status bits it raises.
__device__ __forceinline__ int reduced_coord(const SysDev& S, int d, float x, float& s) {
  s = 0.0f;
  if (!isfinite(x)) return kDevNonFinite;
  float v = __fmul_rn(x, S.invL[d]);
  if (S.pbc[d]) {
    v = __fsub_rn(v, floorf(v));
    if (v >= 1.0f) v = 0.0f;
  } else if (!(v >= 0.0f && v <= 1.0f)) {
    return kDevOutOfCell;
  }
  s = v;
  return 0;
}

// Tilted (periodic) cells: s_d = ((T_d0 x + T_d1 y) + T_d2 z) in FP32 with
// every product and sum rounded once (T = (float) A^-T), then wrapped as a
// periodic axis; for a rectangular cell this is the single product above.
__device__ __forceinline__ int tilted_coords(const SysDev& S, const float* x, float (&s)[3]) {
  s[0] = s[1] = s[2] = 0.0f;
  if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2])) return kDevNonFinite;
  for (int d = 0; d < 3; d++) {
    const float* T = S.Tf + 3 * d;
    float v = __fadd_rn(__fadd_rn(__fmul_rn(T[0], x[0]), __fmul_rn(T[1], x[1])), __fmul_rn(T[2], x[2]));
    v = __fsub_rn(v, floorf(v));
    if (v >= 1.0f) v = 0.0f;
    s[d] = v;
  }
  return 0;
}

__device__ __forceinline__ int axis_cell(const SysDev& S, int d, float s, float& t) {
  t = __fmul_rn(s, (float)S.C[d]);
  int c = (int)t;
  return c > S.C[d] - 1 ? S.C[d] - 1 : c;
}

__global__ void k_bin_count(const SysDev* __restrict__ sys, const AtomItem* __restrict__ items,
                            const float* __restrict__ pos, const float* __restrict__ q, int* __restrict__ cell_id,
                            int* __restrict__ slot, int* __restrict__ cell_count, int* __restrict__ status) {
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  int local = it.start + threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  int g = S.atom_off + local;
  int bad = isfinite(q[g]) ? 0 : kDevNonFinite;
  int c[3];
  if (S.tri) {
    float s[3];
    bad |= tilted_coords(S, pos + 3 * (long long)g, s);
    for (int d = 0; d < 3; d++) {
      float t;
      c[d] = bad ? 0 : axis_cell(S, d, s[d], t);
    }
  } else {
    for (int d = 0; d < 3; d++) {
      float s, t;
      int b = reduced_coord(S, d, pos[3 * g + d], s);
      bad |= b;
      c[d] = b ? 0 : axis_cell(S, d, s, t);
    }
  }
  int cell = (c[0] * S.C[1] + c[1]) * S.C[2] + c[2];
  cell_id[g] = cell;
  slot[g] = atomicAdd(&cell_count[S.cell_off + cell], 1);
  if (bad) atomicOr(status, bad);
}

// exclusive scan of cell_count over tiles of 4096 cells
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int& total) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  int pre = (wid > 0 ? sh[wid - 1] : 0) + x - v;
  total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return pre;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int* __restrict__ cnt, int total_cells,
                                                              int* __restrict__ start, int* __restrict__ tiles) {
  __shared__ int sh[32];
  int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  int v[kScanPer], sum = 0;
  for (int k = 0; k < kScanPer; k++) {
    v[k] = (base + k < total_cells) ? cnt[base + k] : 0;
    sum += v[k];
  }
  int total;
  int pre = block_exclusive_scan(sum, sh, total);
  for (int k = 0; k < kScanPer; k++) {
    if (base + k < total_cells) start[base + k] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0) tiles[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_fix(int* __restrict__ start, int total_cells,
                                                            const int* __restrict__ tiles, int ntiles) {
  __shared__ int sh[32];
  __shared__ int s_off;
  // offset of this tile = sum of the totals of the tiles before it
  int acc = 0;
  for (int t = threadIdx.x; t < (int)blockIdx.x; t += blockDim.x) acc += tiles[t];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w];
    s_off = s;
  }
  __syncthreads();
  int off = s_off;
  int base = blockIdx.x * kScanTile;
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x)
    if (base + k < total_cells) start[base + k] += off;
  if (blockIdx.x == (unsigned)(ntiles - 1) && threadIdx.x == 0) start[total_cells] = off + tiles[ntiles - 1];
}

// each atom's (index, cell) at its slot of its cell's range; the rank kernel
// then walks the sorted positions and finds each entry's stable place in the
// same cell range
__global__ void k_bin_scatter(const SysDev* __restrict__ sys, const AtomItem* __restrict__ items,
                              const int* __restrict__ cell_id, const int* __restrict__ slot,
                              const int* __restrict__ cell_start, int2* __restrict__ bucket) {
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  int local = it.start + threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  int g = S.atom_off + local;
  const int cell = cell_id[g];
  const int b = cell_start[S.cell_off + cell] + slot[g];
  if (MSM_CHECK(S, b >= S.atom_off && b < S.atom_off + S.n)) bucket[b] = make_int2(g, cell);
}

// One thread per sorted position k of the bucket: the entry (g, cell) there
// goes to its stable place dst in the cell's range (the number of the range's
// entries with a smaller atom index), so the stores of a warp stay within the
// few cells its positions cover; the atom's position and charge are gathered.
__global__ void __launch_bounds__(kChunk, 6) k_bin_rank(const SysDev* __restrict__ sys, const AtomItem* __restrict__ items,
                           const float* __restrict__ pos, const float* __restrict__ q,
                           const int* __restrict__ cell_start, const int2* __restrict__ bucket,
                           int* __restrict__ perm, int* __restrict__ iperm, int* __restrict__ scell,
                           float4* __restrict__ xq, float4* __restrict__ uq) {
  AtomItem it = items[blockIdx.x];
  const SysDev& S = sys[it.sys];
  // low part of the binning cell edges, edged - (float)edged (once per block:
  // the per-atom corner below then needs no FP64 arithmetic)
  __shared__ float s_elo[2];
  if (threadIdx.x < 2) s_elo[threadIdx.x] = (float)(S.edged[threadIdx.x] - (double)S.edge[threadIdx.x]);
  __syncthreads();
  int local = it.start + threadIdx.x;
  if ((int)threadIdx.x >= it.count || local >= S.n) return;
  const int2 bg = bucket[S.atom_off + local];
  const int g = bg.x, cell = bg.y;
  if (!MSM_CHECK(S, g >= S.atom_off && g < S.atom_off + S.n && cell >= 0 && cell < S.C[0] * S.C[1] * S.C[2])) return;
  const float qq = q[g];
  const float px[3] = {pos[3 * (long long)g], pos[3 * (long long)g + 1], pos[3 * (long long)g + 2]};
  const int b = cell_start[S.cell_off + cell], e = cell_start[S.cell_off + cell + 1];
  if (!MSM_CHECK(S, b >= S.atom_off && e <= S.atom_off + S.n && b <= e)) return;
  int rank = 0;
  for (int t = b; t < e; t++) rank += (bucket[t].x < g);
  int dst = b + rank;
  perm[dst] = g;
  iperm[g] = dst;
  scell[dst] = cell;
  // x, y relative to the cell's lower faces, z relative to the column base
  // (the Cartesian z of the image next to the cell), formed in FP64 from the
  // FP32 input so that displacements between nearby atoms are exact to FP32
  float loc[3], u[3];
  if (S.tri) {
    const int c[3] = {cell / (S.C[1] * S.C[2]), (cell / S.C[2]) % S.C[1], cell % S.C[2]};
    // Cartesian position relative to the base of the cell's column, c_x / C_x a +
    // c_y / C_y b, formed in FP64 from the FP32 input and wrapped the way the
    // FP32 contract placed the atom (a fractional coordinate that rounds across
    // a face follows its cell)
    float sf[3];
    tilted_coords(S, pos + 3 * (long long)g, sf);
    const double x[3] = {pos[3 * g], pos[3 * g + 1], pos[3 * g + 2]};
    double sd[3];
    for (int d = 0; d < 3; d++) {
      double v = S.Td[3 * d] * x[0] + S.Td[3 * d + 1] * x[1] + S.Td[3 * d + 2] * x[2];
      v -= floor(v);
      if (c[d] == 0 && v > 0.5) v -= 1.0;
      if (c[d] == S.C[d] - 1 && v < 0.5) v += 1.0;
      sd[d] = v - (d < 2 ? (double)c[d] / S.C[d] : 0.0);
      u[d] = sf[d] * S.Mf[d];
    }
    for (int e = 0; e < 3; e++) loc[e] = (float)(sd[0] * S.Ad[e] + sd[1] * S.Ad[3 + e] + sd[2] * S.Ad[6 + e]);
    xq[dst] = make_float4(loc[0], loc[1], loc[2], qq);
    uq[dst] = make_float4(u[0], u[1], u[2], qq);
    return;
  }
  for (int d = 0; d < 3; d++) {
    float s, t;
    const float x = px[d];
    if (reduced_coord(S, d, x, s)) {
      loc[d] = 0.0f;
      u[d] = 0.0f;
      continue;
    }
    const int cd = axis_cell(S, d, s, t);  // the cell coordinate k_bin_count packed into cell_id
    u[d] = s * S.Mf[d];
    // A periodic coordinate outside [0, L), or one in cell 0 near the far face
    // (s rounded up to 1 wraps to cell 0), is wrapped in FP64. x < (float)L
    // implies x < L whichever way L rounded; for C <= 2 the cell-0 test also
    // sends some inner atoms here, which only costs time.
    if (S.pbc[d] && !(x >= 0.0f && x < S.Lf[d] && !(cd == 0 && x >= 0.25f * S.Lf[d]))) {
      double xd = x;
      if (!(xd >= 0.0 && xd < S.Ld[d])) xd -= S.Ld[d] * floor(xd / S.Ld[d]);
      if (cd == 0 && xd > 0.5 * S.Ld[d]) xd -= S.Ld[d];
      loc[d] = d < 2 ? (float)(xd - cd * S.edged[d]) : (float)xd;
      continue;
    }
    if (d == 2) {
      loc[d] = x;
      continue;
    }
    // x - c e rounded once, with c e = ph + pe + c elo exactly up to the last
    // term's rounding: ph = fl(c eh), pe = c eh - ph (exact by FMA), and
    // x - ph is exact (x lies in cell c, so ph / 2 <= x <= 2 ph, Sterbenz)
    const float cf = (float)cd, eh = S.edge[d];
    const float ph = cf * eh;
    const float pe = fmaf(cf, eh, -ph);
    loc[d] = (x - ph) - fmaf(cf, s_elo[d], pe);
  }
  xq[dst] = make_float4(loc[0], loc[1], loc[2], qq);
  uq[dst] = make_float4(u[0], u[1], u[2], qq);
}

void launch_prologue(const Work& w, int total_cells, SysDev* sys, int nsys, int n_single, cudaStream_t s) {
  int blocks = (total_cells + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 1024) blocks = 1024;
  k_prologue<<<blocks, 256, 0, s>>>(w.cell_count, total_cells, w.status, sys, nsys, n_single);
}

void launch_bin(const Work& w, const Tables& t, const AtomItem* items, int nitems, int total_cells,
                int total_atoms, const float* pos, const float* q, cudaStream_t s) {
  (void)total_atoms;
  k_bin_count<<<nitems, kChunk, 0, s>>>(t.sys, items, pos, q, w.cell_id, w.slot, w.cell_count, w.status);
  int ntiles = (total_cells + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<ntiles, kScanThreads, 0, s>>>(w.cell_count, total_cells, w.cell_start, w.scan_tiles);
  k_scan_fix<<<ntiles, kScanThreads, 0, s>>>(w.cell_start, total_cells, w.scan_tiles, ntiles);
  k_bin_scatter<<<nitems, kChunk, 0, s>>>(t.sys, items, w.cell_id, w.slot, w.cell_start, w.bucket);
  k_bin_rank<<<nitems, kChunk, 0, s>>>(t.sys, items, pos, q, w.cell_start, w.bucket, w.perm, w.iperm, w.scell,
                                       w.xq, w.uq);
}

}  // namespace msm
