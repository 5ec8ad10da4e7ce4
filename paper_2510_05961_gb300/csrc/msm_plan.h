// msm_plan.h -- host-side plan and engine of the GB300 MSM library (private).
#pragma once

#include <string>
#include <vector>

#include "../../include/msm_gb300.h"
#include "msm_internal.h"

namespace msm {

struct LevelHost {
  int n[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, per[3] = {0, 0, 0};
  int kind = 0;                      // 0 ball, 1 box
  int R[3] = {0, 0, 0};
  int blo[3] = {0, 0, 0}, bsz[3] = {0, 0, 0};
  float scale = 1.0f;
  std::vector<float> kbox, dkbox;    // box kind: folded stencil and 6 derivative arrays
};

struct SysHost {
  double L[3];                       // lengths of the cell vectors (edge lengths of a rectangular cell)
  // general (tilted, periodic) cells: rows a, b, c of A; fractional s = A^-T r
  bool tri = false;
  double A[9], Ainv[9], Tinv[9];
  double wplane[3];                  // distances between opposite cell faces
  int pbc[3];
  double a;
  int p;
  int M[3];
  double h1[3];
  int nlev = 0, ncomp = 0;
  int S[3], R[3];
  int qi_mode = 0;                   // 0 minimal quasi-interpolation, 1 exact interpolation
  int hw = 1;                        // half-width of omega' (p/2 - 1, or the exact-interpolation truncation)
  std::vector<double> omh;           // omega'_0 .. omega'_hw (symmetric)
  int B[3];                          // radius of the ball-kernel stencil: S (raw samples, p = 4) or R (K)
  bool prefilter = false;            // ball kernels apply raw samples to the omega'-prefiltered grid
  int C[3];
  double edge[3];
  int nnbr[3];
  double gc[8];
  double jc[9];
  std::vector<LevelHost> lev;
  bool has_ball = false;
  std::vector<double> kball, dk1;    // K^1 and its 6 strain derivatives, dense on [-R, R]^3 (host queries)
  std::vector<float> sball, dsh;     // ball-kernel stencil on [-B, B]^3 and half-space virial weights (6x)
  std::vector<float> fsh;            // p = 4: factorized half-space virial weights g = k_1'(|v|)/|v|
  std::vector<int> wball, whalf;     // column half-widths of sball / dsh about cball, -1 = empty column
  std::vector<int> cball;            // column centres (multiples of 4; zero for rectangular cells)
  int hzb = 0;                       // z halo of the ball levels' padded grids and stored rows
  int wmax = 0;                      // widest ball column (half-width about its centre)
  bool allow_ball = true;            // false: every level a dense box
  bool fold_small = false;           // batch plans: levels of <= kFoldPts points as folded dense boxes
  // offsets of this system's ball stencil, virial weights and column tables in the device pools
  long long kball_off = -1, dkh_off = -1, wb_off = -1, wh_off = -1, cb_off = -1;
};

int plan_system(const msm_params& P, SysHost& S, std::string* err);

// spectral level method: the seven spectrum octants of level l on a periodic grid of n points
// per axis (K^ times 1/N, then dK^ xx yy zz xy xz yz times -1/2 (1/N)), each (n_d/2+1) per axis
void level_spectra(const SysHost& S, int l, const int n[3], float* out);

// records the thread's last-error message of the C ABI and returns code
int api_error(int code, const std::string& msg);

struct Engine {
  int nsys = 0;
  bool single = true;
  int p = 4;
  int maxcomp = 0;
  int total_atoms = 0, total_cells = 0;
  long long grid_floats = 0;
  int rmax = 0, ryz[2] = {0, 0};
  std::vector<SysHost> sys;
  std::vector<SysDev> hsys;
  std::vector<LevDev> hlev;
  std::vector<AtomItem> atom_items;
  std::vector<TileItem> anterp_items, ball_items;
  // anterpolation by binning columns: one item per (binning column, z-segment), one sum
  // item per (kAntSumY level-1 grid columns, kAntSumZ points); used when every footprint fits
  // (ant_wstride > 0)
  std::vector<TileItem> acol_items;
  std::vector<TileItem> asum_items;
  long long apart_floats = 0;
  int ant_fmax[2] = {0, 0};
  int ant_wstride = 0;
  std::vector<RangeItem> box_items;
  std::vector<TileItem> pad_items;
  std::vector<std::vector<TileItem>> restrict_steps;
  std::vector<std::vector<TileItem>> prolong_steps;
  std::vector<int> restrict_off, prolong_off;
  std::vector<int> vb_off, vx_off;
  // spectral level method (k_fft.cu): single-system plans with a fully periodic rectangular cell
  // whose evaluated levels are ball levels of 2 .. kSpecNmax points per axis (powers of two).
  // The FFT items: z lines (lev, x, y0, rows), y lines (lev, x, z0, cols), x lines (lev, y, z0, cols).
  bool spec_ok = false;
  int level_method = 0;             // 0 = ball stencils, 1 = spectral (MSM_LEVELS_*)
  bool spec_virial_ready = false;   // the last forward left the spectral grid-virial partials in part_wg
  long long spec_complex = 0;       // float2 entries of the levels' complex work buffers
  std::vector<TileItem> spec_z_items, spec_y_items, spec_x_items;
  TileItem* d_spec_z = nullptr;
  TileItem* d_spec_y = nullptr;
  TileItem* d_spec_x = nullptr;
  std::vector<int> voff_spec;
  int* d_voff_spec = nullptr;       // virial partial ranges of the spectral method (x items, then boxes)
  // device path of msm_plan_set_cell for the spectra (periodic p = 4 plans): separable-sum scratch
  float* d_spec_scr_a = nullptr;
  float* d_spec_scr_b = nullptr;
  std::vector<int> spec_n;          // grid points per axis of each spectral level
  std::vector<long long> spec_sp;   // their spectrum offsets in the stencil pool
  // device tables (owned)
  SysDev* d_sys = nullptr;
  LevDev* d_lev = nullptr;
  float* d_kpool = nullptr;
  int* d_wpool = nullptr;
  AtomItem* d_atom_items = nullptr;
  TileItem* d_anterp_items = nullptr;
  TileItem* d_acol_items = nullptr;
  TileItem* d_asum_items = nullptr;
  TileItem* d_ball_items = nullptr;
  RangeItem* d_box_items = nullptr;
  TileItem* d_pad_items = nullptr;
  TileItem* d_res_items = nullptr;     // restriction tiles of all level steps
  TileItem* d_pro_items = nullptr;     // prolongation tiles of all level steps
  int* d_voff = nullptr;
  // workspace layout (byte offsets)
  size_t L_status, L_cell_count, L_cell_start, L_scan_tiles, L_cell_id, L_slot, L_bucket, L_perm, L_iperm, L_res, L_scell, L_xq,
      L_uq, L_phi_sr, L_phi_lr, L_f_sr, L_f_lr, L_part_e, L_part_q, L_part_w0, L_part_wg, L_part_vs, L_grid, L_vjp_u,
      L_vjp_h, L_io_pos, L_io_q, L_io_dpos, L_io_dq, L_io_e, L_apart, L_spec;
  size_t ws_bytes = 0;
  // state of the last forward pass
  bool have_fwd = false;
  int last_flags = 0;
  void* last_ws = nullptr;
  int last_n = 0;
  // phase timing (msm_profile) and launch counts
  bool profiling = false;
  bool serial = false;              // profiling mode 2: every phase on the caller's stream
  cudaEvent_t ev[2 * 10] = {};
  bool ev_used[10] = {};
  int launches_fwd = 0, launches_bwd = 0;
  // the short-range kernel runs on `side`, forked from and joined to the
  // caller's stream, so it overlaps the grid chain
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t copy = nullptr;      // msm_evaluate_host: device-to-host copies overlapping the grid virial
  cudaEvent_t ev_grad = nullptr;

  Engine() = default;
  Engine(const Engine&) = delete;
  Engine& operator=(const Engine&) = delete;
  ~Engine();
  int build(const msm_params* prm, const int* counts, int nsys, bool single, std::string* err);
  int upload(const std::vector<float>& kp, const std::vector<int>& wp, const std::vector<int>& voff,
             std::string* err);
  // tuned launch shapes (msm_autotune): anterpolation tile z-extent and
  // short-range threads per block
  int vslices = 1;                  // virial reduction slices per system (k_virial_slices)
  int anterp_tz = 32;
  int short_block = kChunk;
  bool any_tri = false;             // some system has a tilted cell: k_short_tri for all
  // the cluster-pair kernel's preconditions (k_short_cl.cu): rectangular cells,
  // nnbr <= 4 along x and y, at most three z images per column
  bool cluster_ok() const {
    for (const SysHost& S : sys)
      if (S.tri || S.nnbr[0] > 4 || S.nnbr[1] > 4 || (S.pbc[2] && S.L[2] < S.a + 2.0 * S.edge[2])) return false;
    return true;
  }
  int short_code() const {
    if (any_tri) return kShortTilted;
    if (short_block == kShortCluster && !cluster_ok()) return kChunk;
    return short_block;
  }
  double* d_energy_scratch = nullptr;  // the autotuner's forward writes its energies here
  double* d_virial_scratch = nullptr;  // the autotuner's grid-virial timing writes its virial here
  void build_anterp_items(int tz);
  void anterp(const Work& w, const Tables& t, cudaStream_t s) const;  // level-1 grid charges
  // e^l of every level by the plan's level method; virial: also the grid-virial partials
  // (spectral method; the ball method computes them in the backward)
  void stencils(const Work& w, const Tables& t, cudaStream_t s, bool virial);
  // grid-virial partials and their reduction to W^(1+) + W^0 times grad (backward)
  void grid_virial(const Work& w, const Tables& t, const double* grad, double* virial, cudaStream_t s);
  int set_level_method(int method, std::string* err);
  int set_anterp_tz(int tz, std::string* err);
  void assemble_pools(const std::vector<int>& lev0_of, std::vector<float>& kp, std::vector<int>& wp);
  // new cell for a single-system plan (msm_plan_set_cell), host path: stencils
  // rebuilt on the host and copied through pinned staging buffers
  int set_cell_host(const double L[3], cudaStream_t s, std::string* err, bool refill = true);
  int set_cell_tilted(const double* cell, cudaStream_t s, std::string* err);
  float* h_kstage = nullptr;
  int* h_wstage = nullptr;
  size_t kpool_n = 0, wpool_n = 0;
  cudaEvent_t ev_stage = nullptr;
  Work resolve(void* ws) const;
  Tables tables() const;
};

}  // namespace msm
