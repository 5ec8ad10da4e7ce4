// msm_internal.h -- device-side descriptors and kernel launchers of the
// GB300 MSM library. Everything here is private to the library; the public
// boundary is include/msm_gb300.h.
//
// Every kernel is batch-native: it reads per-system descriptors (SysDev),
// per-level descriptors (LevDev) and a list of work items built on the host at
// plan time, so one launch serves one system or hundreds of systems alike.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace msm {

constexpr int kMaxLev = 20;
constexpr int kChunk = 256;        // atoms per per-atom work item
constexpr int kChunkWarps = kChunk / 32;
constexpr int kShortTilted = -1;  // short-range launch code of plans with tilted cells (k_short_tri)
constexpr int kShortCluster = 4;  // short-range launch code of the cluster-pair kernel (k_short_cl: i-clusters of 4 atoms)
constexpr int kAnterpTX = 16, kAnterpTY = 8;  // dipole anterpolation tile columns (x, y); its z-extent is tuned
constexpr int kAntWarps = 4;       // anterpolation: binning-column items (one per warp) per block
constexpr int kAntFootMax = 16;    // largest footprint of a binning column per axis (grid columns)
constexpr int kAntSumZ = 128;      // anterpolation sums: level-1 points along z per grid column and block
constexpr int kAntSumY = 1;        // anterpolation sums: grid columns (consecutive y) per block (4 measured slower)
constexpr int kBallTY = 32;        // stencil tile rows (y)
constexpr int kBallBZ = 16;        // outputs per thread along z
constexpr int kBallTZ = 32;        // stencil tile depth (z)
constexpr int kBallThreads = kBallTY * (kBallTZ / kBallBZ);
constexpr int kBallRmax = 24;      // largest ball-stencil radius with a compiled kernel
constexpr int kBoxChunk = 16;      // outputs per box-stencil work item (one block) of a level above kBoxStage points
constexpr int kBoxStage = 8192;    // box levels of at most this many points: staged in shared memory, one output per thread
constexpr int kBoxThreads = 256;   // threads per box-stencil block
constexpr int kResTX = 4, kResTY = 4, kResTZ = 16;  // restriction tiles (coarse points)
constexpr int kResNT = kResTX * kResTY * kResTZ;    // threads per restriction block
constexpr int kVirialSlices = 64;  // most virial reduction slices per system
constexpr int kProTX = 4, kProTY = 4, kProTZ = 32;  // prolongation tiles (fine points)
constexpr int kFoldPts = 512;      // batch plans fold levels this small into dense boxes
constexpr int kPadTX = 16, kPadTY = 8, kPadTZ = 32;  // halo-padding tiles (x planes, y rows, z columns)
constexpr int kSpecTile = 2048;    // spectral level method: complex values per FFT tile (lines x points)
constexpr int kSpecNmax = 256;     // spectral level method: most points per axis (twiddle table of 256)

// device status bits (mirrors MSM_DEV_* of the public header)
constexpr int kDevOutOfCell = 1;
constexpr int kDevNonFinite = 2;
constexpr int kDevNonNeutral = 4;
constexpr int kDevCheck = 8;  // MSM_CHECKS builds: an index outside its array was caught and the access skipped
constexpr float kNeutralTol = 1e-5f;  // |sum q| > kNeutralTol * sum |q| counts as non-neutral

struct SysDev {
  int* status;      // the call's device status word (written by the prologue; used by MSM_CHECKS builds)
  double Ld[3];     // cell lengths (FP64: periodic image shifts of the pair displacements)
  double edged[3];  // binning cell edges (FP64)
  int n;            // atoms of this system
  int atom_off;     // first packed (user-order and sorted) atom index
  int C[3];         // binning cells per axis
  int cell_off;     // first packed cell index
  int nnbr[3];      // neighbour-cell reach ceil(a / edge)
  int cshift[3];    // log2 of C rounded up (C is a power of two on periodic axes)
  int pbc[3];
  int M[3];         // level-1 interval counts (u = s * M)
  int p;            // B-spline order
  int ncomp;        // evaluated grid levels
  int lev0;         // index of level 1 in the LevDev table
  int item0, nitem; // per-atom work items of this system
  float edge[3];    // binning cell edges
  float invL[3];    // (float)(1/L): binning contract
  float Mf[3];      // M as float
  float inv_h1[3];  // 1/h_1 per axis
  float Lf[3];      // cell lengths
  float h1f[3];     // level-1 spacings
  float a2, inv_a, inv_a2, inv_a3;
  float self_coef;  // gamma(0)/a (self term of Eq. U_zero)
  float gca[8];     // softening polynomial over a, in s = 1 - (r/a)^2: gamma(r/a)/a = sum_k gca[k] s^k
  float gdca[8];    // (2/a^3) d gamma / d s = sum_k gdca[k] s^k, so k_0'(r)/r = -1/r^3 + sum_k gdca[k] s^k
  float jc[9];      // restriction coefficients J_k, k = -p/2 .. p/2 (index k + p/2)
  float bsp[4][8];  // centred B-spline Phi_p on |t| in [i, i+1): sum_k bsp[i][k] (|t| - i)^k
  float om[4];      // prefilter of the ball levels: omega'_0 .. omega'_(pre_r) (symmetric), or identity
  int pre_r;        // prefilter half-width (p/2 - 1 when the ball kernels apply raw samples, else 0)
  // general (tilted, periodic) cells; tri = 0 for rectangular cells
  int tri;
  float Tf[9];      // (float) A^-T: binning contract s_d = ((T_d0 x + T_d1 y) + T_d2 z)
  double Ad[9];     // cell rows a, b, c (FP64: positions and image shifts)
  double Td[9];     // A^-T (FP64)
  float Jg[9];      // A^-1 diag(M): Cartesian gradient from level-1 grid derivatives
  float reach[3];   // a / (distance between cell faces): fractional reach of the cutoff per axis
  // anterpolation by binning columns: level-1 grid columns (x, y) that the atoms of one
  // binning column reach, and the float offset of this system's column partials
  int afoot[2];
  long long apart;
  int ashift[3];    // log2 of the level-1 intervals per binning cell where the cells are aligned with the grid, else -1
  float aratio[3];  // M / C (axes whose cells are not aligned with the grid)
  float ainv[3];    // C / M
};

// Debug builds (-DMSM_CHECKS=1, build.build(checks=True)): kernels test their
// data-dependent indices before the access; a failed test sets kDevCheck in
// the status word (through S.status) and skips the access, so the call ends
// with the bit set instead of touching memory outside an array. Normal builds
// compile the tests away.
#ifndef MSM_CHECKS
#define MSM_CHECKS 0
#endif
#if MSM_CHECKS
#define MSM_CHECK(S, cond) ((cond) ? true : (atomicOr((S).status, kDevCheck), false))
#else
#define MSM_CHECK(S, cond) true
#endif

struct LevDev {
  int sys, level;           // owning system, level number (1-based)
  int n[3], lo[3], per[3];  // grid points, first grid index, periodic flags
  long long q_off, e_off;   // float offsets of q~^l and e^l in the grid pool
  int kind;                 // 0 = ball stencil (radius R, wrap/zero), 1 = dense box (folded)
  int box_tile;             // box: 1 = staged in shared memory, one output per thread (batch plans,
                            // levels of at most kBoxStage points); 0 = one warp per output
  int R[3];                 // ball radius per axis
  int blo[3], bsz[3];       // box: offsets d in [blo, blo + bsz)
  float scale;              // stencil scale 2^-(l-1) relative to the stored values
  long long k_off;          // stencil values. box: dense bsz product; ball: per (dx, dy)
                            // column, dz = -hz .. hz at [0, 2hz] of a row of kSK(hz) floats
  long long dk_off;         // virial weights. box: per entry the 6 values padded to 8 (16-byte aligned); ball: [dx][6][dy][row]
  long long w_off;          // ball: column half-widths of K (int pool, (2Rx+1)(2Ry+1), -1 = empty)
  long long wh_off;         // ball: column half-widths of the virial weights
  int hz;                   // ball: z halo of the padded grid (>= R[2], multiple of 4)
  int pn[3];                // ball: padded grid dims
  long long c_off;          // ball: column centres (int pool; all zero for rectangular cells)
  long long p_off;          // ball: float offset of the halo-padded, omega'-prefiltered copy of q~^l
                            // (ball levels apply raw kernel samples; R is the sample radius)
  // spectral level method (fully periodic single-system plans, k_fft.cu): float2 offset of the
  // level's complex work buffer, float offsets of its spectra (eight floats per point: K^, dK^
  // xx yy zz xy xz yz, 0; at [|k_x|][|k_y|][z position], k_z the bit reversal of the position)
  // and of the twiddle table in the stencil pool (-1 where the level has none), log2 of n per axis
  long long f_off, sp_off, tw_off;
  int lg[3];
};

// row length (floats) of one stored ball-stencil column with halo hz
__host__ __device__ constexpr int kSK(int hz) { return 2 * hz + 4; }

#ifdef __CUDACC__
// 1/sqrt(x) for a normal x > 0: the hardware approximation (relative error
// below 2^-22), flush-to-zero form, so no rescaling of subnormal inputs
__device__ __forceinline__ float rsqrt_nrm(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
#endif

struct AtomItem { int sys, start, count; };
struct TileItem { int lev, x0, y0, z0; };
struct RangeItem { int lev, start, count; };

// workspace arrays of one call (device pointers resolved by the host)
struct Work {
  int* status;
  int* cell_count;
  int* cell_start;
  int* scan_tiles;
  int* cell_id;
  int* slot;
  int2* bucket;    // binning: (atom, cell) at the atom's slot of its cell, before the stable rank
  int* perm;
  int* iperm;      // binning: sorted position of each atom, atom order
  int* scell;
  float4* xq;      // Cartesian position (the periodic image next to its cell) and charge, sorted
  float4* uq;      // level-1 grid coordinates and charge, sorted order
  float* phi_sr;   // short-range potential incl. self term, sorted
  float4* f_sr;    // short-range field -grad phi0 (force / q), sorted
  float* phi_lr;   // long-range potential, sorted
  float4* f_lr;    // long-range field -grad phi^(1+) (force / q), sorted
  float4* res;     // outputs of the last forward, sorted: phi and F = q field
  float2* part_e;  // per atom item: sum q phi as hi + lo
  float2* part_q;  // per atom item: sum q and sum |q|
  double* part_w0; // per warp of each atom item: 6 short-range virial components
  double* part_wg; // per virial item: 6 grid virial components
  double* part_vs; // per system and reduction slice: 6 virial components
  float* grid;     // grid pool
  float* apart;    // anterpolation: level-1 partial sums of each binning column (per system at SysDev::apart)
  float2* spec;    // spectral level method: complex work buffers of the levels (LevDev::f_off)
  float4* vjp_u;   // force vector-Jacobian product: upstream (u, q), sorted
  float4* vjp_h;   // force vector-Jacobian product: short-range rows of H u and psi, sorted
  // staging of msm_evaluate_host (caller's atom order)
  float* io_pos;   // n x 3 positions
  float* io_q;     // n charges
  float* io_dpos;  // n x 3 dE/dpos
  float* io_dq;    // n dE/dq
  double* io_e;    // energy per system, then dL/dE = 1 per system, then 9 virial components per system
};

struct Tables {
  const SysDev* sys;
  const LevDev* lev;
  const float* kpool;
  const int* wpool;
};

// ---------------------------------------------------------------- launchers
// binning (k_bin.cu)
void launch_prologue(const Work& w, int total_cells, SysDev* sys, int nsys, int n_single, cudaStream_t s);
void launch_bin(const Work& w, const Tables& t, const AtomItem* items, int nitems, int total_cells,
                int total_atoms, const float* pos, const float* q, cudaStream_t s);
// short range (k_short.cu)
void launch_short(const Work& w, const Tables& t, const AtomItem* items, int nitems, bool forces, bool virial,
                  cudaStream_t s, int p, int block);
// short range as cluster-pair tiles (k_short_cl.cu), rectangular cells
void launch_short_cluster(const Work& w, const Tables& t, const AtomItem* items, int nitems, bool forces,
                          bool virial, cudaStream_t s, int p);
// anterpolation / interpolation (k_interp.cu)
void launch_anterp(const Work& w, const Tables& t, const TileItem* items, int nitems, cudaStream_t s, int p, int tz);
// anterpolation by binning columns (k_interp.cu): per-column partial sums, then their sum per point
int anterp_cols_wstride(int fx_max, int fy_max, int tz, int p);
void launch_anterp_cols(const Work& w, const Tables& t, const TileItem* cols, int ncol, const TileItem* sums,
                        int nsum, int tz, int wstride, cudaStream_t s, int p);
void launch_interp(const Work& w, const Tables& t, const AtomItem* items, int nitems, bool forces,
                   cudaStream_t s, int p);
// restriction / prolongation (k_grid.cu)
void launch_restrict(const Work& w, const Tables& t, const TileItem* items, int nitems, cudaStream_t s, int p);
void launch_prolong(const Work& w, const Tables& t, const TileItem* items, int nitems, cudaStream_t s, int p);
// stencils and grid virial (k_stencil.cu)
void launch_pad(const Work& w, const Tables& t, const TileItem* items, int nitems, int pre_r, cudaStream_t s);
void launch_stencil_ball(const Work& w, const Tables& t, const TileItem* items, int nitems, int rmax,
                         int ryz_max[2], bool general, cudaStream_t s);
void launch_stencil_box(const Work& w, const Tables& t, const RangeItem* items, int nitems, cudaStream_t s);
void launch_virial_ball(const Work& w, const Tables& t, const TileItem* items, int nitems, int rmax,
                        int ryz_max[2], int part_off, bool factorized, bool general, cudaStream_t s);
void launch_virial_box(const Work& w, const Tables& t, const RangeItem* items, int nitems, int part_off,
                       cudaStream_t s);
// outputs (k_final.cu)
// phi and F (forces: the fields were computed) per sorted atom into w.res, the energy partials
void launch_finalize(const Work& w, const Tables& t, const AtomItem* items, int nitems, bool forces, cudaStream_t s);
// w.res to the caller's atom order (either pointer may be null); forces times fsign (-1: dE/dr for dL/dE = 1)
void launch_outputs(const Work& w, const Tables& t, const AtomItem* items, int nitems, float* phi, float* forces,
                    float fsign, cudaStream_t s);
void launch_energy(const Work& w, const Tables& t, int nsys, double* energy, cudaStream_t s);  // also flags non-neutral periodic systems
// spectral level method (k_fft.cu): e^l of every spectral level (part: grid virial partials, one
// per x item, or null), or the virial partials alone
void launch_spectral(const Work& w, const Tables& t, const TileItem* zi, int nz, const TileItem* yi, int ny,
                     const TileItem* xi, int nx, double* part, cudaStream_t s);
void launch_spectral_virial(const Work& w, const Tables& t, const TileItem* zi, int nz, const TileItem* yi, int ny,
                            const TileItem* xi, int nx, double* part, cudaStream_t s);
void launch_virial_out(const Work& w, const Tables& t, int nsys, int nslice, const int* vitem_off,
                       const double* grad, double* virial, cudaStream_t s);
// from_res: from the forward's w.res (its forces included when dE_dpos is wanted); else from the
// sorted potentials and fields
void launch_backward_scale(const Work& w, const Tables& t, const AtomItem* items, int nitems,
                           const double* grad, float* dE_dpos, float* dE_dq, bool from_res, cudaStream_t s);
void launch_field(const Work& w, const Tables& t, const AtomItem* items, int nitems, float* field, cudaStream_t s);
void launch_fill(double* p, int n, double v, cudaStream_t s);
// vector-Jacobian product of the forces (k_final.cu, k_short.cu, k_interp.cu)
void launch_sort_u(const Work& w, const Tables& t, const AtomItem* items, int nitems, const float* u, float4* us,
                   cudaStream_t s);
void launch_short_fvjp(const Work& w, const Tables& t, const AtomItem* items, int nitems, const float4* us,
                       float4* out, cudaStream_t s, int p, bool tilted);
void launch_interp_hess(const Work& w, const Tables& t, const AtomItem* items, int nitems, const float4* us,
                        cudaStream_t s, int p);
void launch_anterp_dipole(const Work& w, const Tables& t, const TileItem* items, int nitems, cudaStream_t s, int p,
                          int tz, const float4* us);
// vector-Jacobian product of the potentials (k_final.cu)
void launch_pvjp_prep(const Work& w, const Tables& t, const AtomItem* items, int nitems, const float* g,
                      cudaStream_t s);
void launch_pvjp_final(const Work& w, const Tables& t, const AtomItem* items, int nitems, float* dq, float* dpos,
                       cudaStream_t s);
void launch_fvjp_final(const Work& w, const Tables& t, const AtomItem* items, int nitems, const float4* hs, float* dq,
                       float* dpos, cudaStream_t s);
// dynamic cell (k_cell.cu): new system descriptor (alone, or with the ball stencils of a periodic p = 4 plan)
void launch_set_sys(SysDev* d_sys, const SysDev& val, cudaStream_t s);
// spectral level method, dynamic cell (k_cell.cu): the spectra of levels 1 .. nlev (cubic grids of n[l-1]
// points per axis, n[0] the largest) of a periodic p = 4 plan from its raw samples, into the stencil pool
// at sp_off[l-1], three launches for all levels; scratch_a: sum over levels of 7 (2B_x+1)(2B_y+1)(n/2+1)
// floats, scratch_b: sum of 7 (2B_x+1)(n/2+1)^2 floats, then 7 (2B_x+1)(2B_y+1)(2B_z+1) for the samples
void launch_spec_cell(const double h1[3], double a, int p, const int B[3], const double* om, int hw, int nlev,
                      const int* n, const long long* sp_off, float* scratch_a, float* scratch_b, float* kpool,
                      cudaStream_t s);
void launch_cell_update(SysDev* d_sys, const SysDev& val, const double h1[3], double a, int p, const int B[3], int hz,
                        long long kball_off, long long dkh_off, long long wb_off, long long wh_off, float* kpool,
                        int* wpool, cudaStream_t s);

}  // namespace msm
