// msm_api.cu -- the C ABI (include/msm_gb300.h): plans, batches, forward and
// backward passes. Each call validates its arguments on the host, resolves
// the caller's workspace into arrays and enqueues the kernels on the caller's
// stream; nothing here waits for the GPU except msm_status.
#include <cstring>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "msm_plan.h"
#include <cmath>

using namespace msm;

struct msm_plan_s {
  Engine eng;
};
struct msm_batch_s {
  Engine eng;
};

static thread_local std::string g_err;

static int set_err(int code, const std::string& m) {
  g_err = m;
  return code;
}

int msm::api_error(int code, const std::string& msg) { return set_err(code, msg); }

static int check_launch(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(MSM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return MSM_OK;
}

// phase timing: an event pair around each phase when profiling is on, and an
// NVTX range named after the phase (host side: it brackets the launches, so
// a profiler's timeline groups each phase's kernels)
static const char* const kPhaseName[MSM_NPHASE] = {"msm:bin",    "msm:short",  "msm:anterp", "msm:restrict",
                                                   "msm:stencil", "msm:prolong", "msm:interp", "msm:final",
                                                   "msm:virial", "msm:bscale"};
struct Phase {
  Engine& E;
  int ph;
  cudaStream_t s;
  Phase(Engine& e, int p, cudaStream_t st) : E(e), ph(p), s(st) {
    nvtxRangePushA(kPhaseName[ph]);
    if (E.profiling) {
      cudaEventRecord(E.ev[2 * ph], s);
      E.ev_used[ph] = true;
    }
  }
  ~Phase() {
    if (E.profiling) cudaEventRecord(E.ev[2 * ph + 1], s);
    nvtxRangePop();
  }
};

// kernels each phase launches (for the launch count)
static int count_forward(const Engine& E, bool outputs) {
  int n = 1 + 5 + 1;                                   // prologue, binning, short range
  n += E.anterp_items.empty() ? 0 : (E.ant_wstride > 0 ? 2 : 1);  // anterpolation (columns: partials + sums)
  for (int l = 1; l < E.maxcomp; l++) n += 2;          // restriction + prolongation per level step
  if (E.level_method == 1) n += 5;                     // spectral: z, y, x (with the product), y, z passes
  else n += E.ball_items.empty() ? 0 : 2;              // halo padding + ball stencil
  n += E.box_items.empty() ? 0 : 1;
  n += 1 + 1 + 1 + (outputs ? 1 : 0);                  // interp, finalize, energy, outputs
  return n;
}

// forward pass of an engine; n_single >= 0 sets the atom count of a single-system plan
static int run_forward(Engine& E, void* ws, size_t ws_bytes, int n_single, const float* pos, const float* q,
                       double* energy, float* phi, float* forces, int flags, cudaStream_t s, float fsign = 1.0f) {
  if (!ws || !energy) return set_err(MSM_ERR_INVALID_ARG, "workspace and energy must not be NULL");
  if (ws_bytes < E.ws_bytes) return set_err(MSM_ERR_CAPACITY, "workspace smaller than msm_workspace_bytes");
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return set_err(MSM_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  int n_total = E.single ? n_single : E.total_atoms;
  if (n_total > 0 && (!pos || !q)) return set_err(MSM_ERR_INVALID_ARG, "positions and charges must not be NULL");
  if ((flags & MSM_WANT_FORCES) == 0 && forces) return set_err(MSM_ERR_INVALID_ARG, "forces requested without MSM_WANT_FORCES");
  const bool want_f = (flags & MSM_WANT_FORCES) != 0;
  const bool want_w = (flags & MSM_WANT_VIRIAL) != 0;
  Work w = E.resolve(ws);
  Tables t = E.tables();
  for (bool& u : E.ev_used) u = false;
  E.spec_virial_ready = false;
  const int nai = (int)E.atom_items.size();
  {
    Phase ph(E, MSM_PH_BIN, s);
    launch_prologue(w, E.total_cells, E.d_sys, E.nsys, E.single ? n_single : -1, s);
    launch_bin(w, t, E.d_atom_items, nai, E.total_cells, n_total, pos, q, s);
  }
  // anterpolation before the fork: its blocks then have the GPU to themselves
  // (measured faster than running it beside the short-range kernel)
  {
    Phase ph(E, MSM_PH_ANTERP, s);
    E.anterp(w, t, s);
  }
  // fork: the short-range pairs (side stream) overlap the rest of the grid
  // chain (caller's stream); serial profiling keeps them on the caller's stream
  cudaStream_t ss = E.serial ? s : E.side;
  if (!E.serial) {
    cudaEventRecord(E.ev_fork, s);
    cudaStreamWaitEvent(E.side, E.ev_fork, 0);
  }
  {
    Phase ph(E, MSM_PH_SHORT, ss);
    launch_short(w, t, E.d_atom_items, nai, want_f, want_w, ss, E.p,
                 E.short_code());
  }
  if (!E.serial) cudaEventRecord(E.ev_join, E.side);
  {
    Phase ph(E, MSM_PH_RESTRICT, s);
    for (int l = 1; l < E.maxcomp; l++) {
      int a = E.restrict_off[l - 1], b = E.restrict_off[l];
      launch_restrict(w, t, E.d_res_items + a, b - a, s, E.p);
    }
  }
  {
    Phase ph(E, MSM_PH_STENCIL, s);
    E.stencils(w, t, s, want_w);
  }
  {
    Phase ph(E, MSM_PH_PROLONG, s);
    for (int l = E.maxcomp - 1; l >= 1; l--) {
      int a = E.prolong_off[l - 1], b = E.prolong_off[l];
      launch_prolong(w, t, E.d_pro_items + a, b - a, s, E.p);
    }
  }
  {
    Phase ph(E, MSM_PH_INTERP, s);
    launch_interp(w, t, E.d_atom_items, nai, want_f, s, E.p);
  }
  if (!E.serial) cudaStreamWaitEvent(s, E.ev_join, 0);  // join
  {
    Phase ph(E, MSM_PH_FINAL, s);
    launch_finalize(w, t, E.d_atom_items, nai, want_f, s);
    launch_energy(w, t, E.nsys, energy, s);
    launch_outputs(w, t, E.d_atom_items, nai, phi, want_f ? forces : nullptr, fsign, s);
  }
  E.launches_fwd = count_forward(E, phi || (want_f && forces));
  E.launches_bwd = 0;
  int rc = check_launch("msm_forward");
  if (rc) return rc;
  E.have_fwd = true;
  E.last_flags = flags;
  E.last_ws = ws;
  E.last_n = n_total;
  return MSM_OK;
}

static int run_backward(Engine& E, void* ws, const double* grad, float* dE_dpos, float* dE_dq, double* virial,
                        cudaStream_t s) {
  if (!E.have_fwd || ws != E.last_ws) return set_err(MSM_ERR_NO_FORWARD, "msm_backward needs a prior msm_forward on this workspace");
  if (!grad) return set_err(MSM_ERR_INVALID_ARG, "grad_energy must not be NULL");
  Work w = E.resolve(ws);
  Tables t = E.tables();
  const int nai = (int)E.atom_items.size();
  const bool had_f = (E.last_flags & MSM_WANT_FORCES) != 0;
  const bool had_w = (E.last_flags & MSM_WANT_VIRIAL) != 0;
  const bool need_f = dE_dpos != nullptr;
  const bool need_w = virial != nullptr;
  // the forward's per-atom results serve unless the forces are wanted and it skipped them
  const bool from_res = !need_f || had_f;
  int nl = 0;
  if ((need_f && !had_f) || (need_w && !had_w)) {
    // the forward skipped these parts; the short-range kernel rewrites its
    // potential with identical values, so running it again is safe
    Phase ph(E, MSM_PH_SHORT, s);
    launch_short(w, t, E.d_atom_items, nai, need_f || had_f, need_w || had_w, s, E.p, E.short_code());
    nl++;
    if (need_f && !had_f) {
      launch_interp(w, t, E.d_atom_items, nai, true, s, E.p);
      nl++;
    }
    E.last_flags |= (need_f ? MSM_WANT_FORCES : 0) | (need_w ? MSM_WANT_VIRIAL : 0);
  }
  if (need_w) {
    Phase ph(E, MSM_PH_VIRIAL, s);
    if (E.level_method == 1) nl += E.spec_virial_ready ? 0 : 3;
    else nl += E.ball_items.empty() ? 0 : 1;
    E.grid_virial(w, t, grad, virial, s);
    nl += (E.box_items.empty() ? 0 : 1) + 2;
  }
  if (dE_dpos || dE_dq) {
    Phase ph(E, MSM_PH_BSCALE, s);
    launch_backward_scale(w, t, E.d_atom_items, nai, grad, dE_dpos, dE_dq, from_res, s);
    nl++;
  }
  E.launches_bwd = nl;
  return check_launch("msm_backward");
}

// End-to-end evaluation on host buffers (msm_evaluate_host): inputs copied into
// the workspace's staging arrays, then the forward (forces, virial) on the
// caller's stream writing, for dL/dE = 1, dE/dq = phi and dE/dr = -F straight
// into the staging outputs (the same values the backward's scaling would
// write); E and the per-atom gradients are copied back on a second stream
// while the backward forms the virial, then the virial; waits for both.
static int run_evaluate_host(Engine& E, void* ws, size_t ws_bytes, int n, const float* pos_h, const float* q_h,
                             double* e_h, float* dpos_h, float* dq_h, double* w_h, cudaStream_t s) {
  if (!ws || !e_h) return set_err(MSM_ERR_INVALID_ARG, "workspace and energy_host must not be NULL");
  if (n > 0 && (!pos_h || !q_h || !dpos_h || !dq_h))
    return set_err(MSM_ERR_INVALID_ARG, "host positions, charges and gradient buffers must not be NULL");
  if (ws_bytes < E.ws_bytes) return set_err(MSM_ERR_CAPACITY, "workspace smaller than msm_workspace_bytes");
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return set_err(MSM_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  if (!E.copy && (cudaStreamCreateWithFlags(&E.copy, cudaStreamNonBlocking) != cudaSuccess ||
                  cudaEventCreateWithFlags(&E.ev_grad, cudaEventDisableTiming) != cudaSuccess))
    return set_err(MSM_ERR_CUDA, "msm_evaluate_host: stream or event creation failed");
  Work w = E.resolve(ws);
  const int nsys = E.nsys;
  if (n > 0 && (cudaMemcpyAsync(w.io_pos, pos_h, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(w.io_q, q_h, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess))
    return set_err(MSM_ERR_CUDA, "msm_evaluate_host: input copy failed");
  launch_fill(w.io_e + nsys, nsys, 1.0, s);  // dL/dE = 1
  int rc = run_forward(E, ws, ws_bytes, n, w.io_pos, w.io_q, w.io_e, w.io_dq, w.io_dpos,
                       MSM_WANT_FORCES | (w_h ? MSM_WANT_VIRIAL : 0), s, -1.0f);
  if (rc) return rc;
  cudaEventRecord(E.ev_grad, s);
  cudaStreamWaitEvent(E.copy, E.ev_grad, 0);
  bool ok = cudaMemcpyAsync(e_h, w.io_e, sizeof(double), cudaMemcpyDeviceToHost, E.copy) == cudaSuccess;
  if (n > 0)
    ok = ok && cudaMemcpyAsync(dpos_h, w.io_dpos, sizeof(float) * 3 * (size_t)n, cudaMemcpyDeviceToHost, E.copy) ==
                   cudaSuccess &&
         cudaMemcpyAsync(dq_h, w.io_dq, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, E.copy) == cudaSuccess;
  if (ok && w_h) {
    if ((rc = run_backward(E, ws, w.io_e + nsys, nullptr, nullptr, w.io_e + 2 * nsys, s))) return rc;
    ok = cudaMemcpyAsync(w_h, w.io_e + 2 * nsys, sizeof(double) * 9, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  }
  if (!ok) return set_err(MSM_ERR_CUDA, "msm_evaluate_host: output copy failed");
  if (cudaStreamSynchronize(E.copy) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return set_err(MSM_ERR_CUDA, std::string("msm_evaluate_host: ") + cudaGetErrorString(cudaGetLastError()));
  return check_launch("msm_evaluate_host");
}

// field -grad phi at every atom from the last forward on ws (forces / q, no
// division); a forward without forces gets its field parts computed here
static int run_field(Engine& E, void* ws, float* field, cudaStream_t s) {
  if (!E.have_fwd || ws != E.last_ws) return set_err(MSM_ERR_NO_FORWARD, "msm_field needs a prior msm_forward on this workspace");
  if (!field && E.last_n > 0) return set_err(MSM_ERR_INVALID_ARG, "field must not be NULL");
  Work w = E.resolve(ws);
  Tables t = E.tables();
  const int nai = (int)E.atom_items.size();
  if ((E.last_flags & MSM_WANT_FORCES) == 0) {
    const bool had_w = (E.last_flags & MSM_WANT_VIRIAL) != 0;
    launch_short(w, t, E.d_atom_items, nai, true, had_w, s, E.p, E.short_code());
    launch_interp(w, t, E.d_atom_items, nai, true, s, E.p);
    E.last_flags |= MSM_WANT_FORCES;
  }
  if (E.last_n > 0) launch_field(w, t, E.d_atom_items, nai, field, s);
  return check_launch("msm_field");
}

// Autotuner: one forward fills the workspace (bins, sorted atoms, level-1
// grid), then each tunable launch shape is timed on those inputs (CUDA events,
// one warm-up and three timed launches per candidate) and the fastest is kept.
// Each shape belongs to one kernel, so the shapes are tuned independently.
static int run_autotune(Engine& E, void* ws, size_t ws_bytes, int n_single, const float* pos, const float* q,
                        cudaStream_t s) {
  if (!E.d_energy_scratch && cudaMalloc((void**)&E.d_energy_scratch, sizeof(double) * std::max(E.nsys, 1)) != cudaSuccess)
    return set_err(MSM_ERR_CUDA, "autotune: cudaMalloc failed");
  int rc = run_forward(E, ws, ws_bytes, n_single, pos, q, E.d_energy_scratch, nullptr, nullptr, 0, s);
  if (rc) return rc;
  Work w = E.resolve(ws);
  Tables t = E.tables();
  const int nai = (int)E.atom_items.size();
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
    return set_err(MSM_ERR_CUDA, "autotune: cudaEventCreate failed");
  auto timed = [&](auto&& launch) {
    launch();
    cudaEventRecord(a, s);
    for (int r = 0; r < 3; r++) launch();
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  };
  std::string err;
  int best_tz = E.anterp_tz;
  float best = 1e30f;
  for (int tz : {16, 32, 64}) {
    if ((rc = E.set_anterp_tz(tz, &err))) break;
    const float ms = timed([&] { E.anterp(w, t, s); });
    if (ms < best) {
      best = ms;
      best_tz = tz;
    }
  }
  if (!rc) rc = E.set_anterp_tz(best_tz, &err);
  int best_nb = E.short_block;
  best = 1e30f;
  if (!rc && !E.any_tri)
    for (int nb : {kChunk, kChunk / 2, kShortCluster}) {
      if (nb == kShortCluster && !E.cluster_ok()) continue;
      const float ms = timed([&] { launch_short(w, t, E.d_atom_items, nai, true, true, s, E.p, nb); });
      if (ms < best) {
        best = ms;
        best_nb = nb;
      }
    }
  E.short_block = best_nb;
  // level method (plans that allow the spectral one): the forward's stencils with the
  // backward's grid virial, per method
  if (!rc && E.spec_ok) {
    if (!E.d_virial_scratch && cudaMalloc((void**)&E.d_virial_scratch, sizeof(double) * 9) != cudaSuccess)
      rc = MSM_ERR_CUDA, err = "cudaMalloc failed";
    int best_m = E.level_method;
    best = 1e30f;
    for (int m : {0, 1}) {
      if (rc || (rc = E.set_level_method(m, &err))) break;
      const float ms = timed([&] {
        E.stencils(w, t, s, true);
        E.grid_virial(w, t, nullptr, E.d_virial_scratch, s);
      });
      if (ms < best) {
        best = ms;
        best_m = m;
      }
    }
    if (!rc) rc = E.set_level_method(best_m, &err);
  }
  E.have_fwd = false;  // the timed launches reused the workspace: a new forward is needed
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return set_err(rc, "autotune: " + err);
  return check_launch("msm_autotune");
}

static int read_status(Engine& E, void* ws, cudaStream_t s, int* out) {
  if (!ws || !out) return set_err(MSM_ERR_INVALID_ARG, "workspace and device_status must not be NULL");
  Work w = E.resolve(ws);
  int v = 0;
  if (cudaMemcpyAsync(&v, w.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return set_err(MSM_ERR_CUDA, std::string("msm_status: ") + cudaGetErrorString(cudaGetLastError()));
  *out = v;
  return MSM_OK;
}

static void fill_info(const SysHost& S, msm_plan_info* info) {
  std::memset(info, 0, sizeof(*info));
  info->nlev = S.nlev;
  info->ncomp = S.ncomp;
  for (int d = 0; d < 3; d++) {
    info->M[d] = S.M[d];
    info->h1[d] = S.h1[d];
    info->R[d] = S.R[d];
    info->C[d] = S.C[d];
    info->nnbr[d] = S.nnbr[d];
  }
  for (int l = 0; l < S.ncomp && l < 20; l++) {
    for (int d = 0; d < 3; d++) {
      info->lo[l][d] = S.lev[l].lo[d];
      info->n[l][d] = S.lev[l].n[d];
    }
    info->stencil_kind[l] = S.lev[l].kind;
  }
}

extern "C" {

const char* msm_last_error(void) { return g_err.c_str(); }

int msm_profile(msm_plan plan, int enable) {
  if (!plan) return set_err(MSM_ERR_INVALID_ARG, "plan must not be NULL");
  Engine& E = plan->eng;
  if (enable && !E.ev[0])
    for (auto& e : E.ev)
      if (cudaEventCreate(&e) != cudaSuccess) return set_err(MSM_ERR_CUDA, "cudaEventCreate failed");
  if (enable < 0 || enable > 2) return set_err(MSM_ERR_INVALID_ARG, "enable must be 0, 1 or 2");
  E.profiling = enable != 0;
  E.serial = enable == 2;
  return MSM_OK;
}

int msm_profile_read(msm_plan plan, double* ms, int* launches) {
  if (!plan || !ms) return set_err(MSM_ERR_INVALID_ARG, "NULL argument");
  Engine& E = plan->eng;
  for (int p = 0; p < MSM_NPHASE; p++) {
    ms[p] = 0.0;
    if (!E.profiling || !E.ev_used[p]) continue;
    float t = 0.f;
    if (cudaEventSynchronize(E.ev[2 * p + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, E.ev[2 * p], E.ev[2 * p + 1]) != cudaSuccess)
      return set_err(MSM_ERR_CUDA, "profile events not readable");
    ms[p] = t;
  }
  if (launches) *launches = E.launches_fwd + E.launches_bwd;
  return MSM_OK;
}

int msm_plan_create(const msm_params* params, msm_plan* out) {
  if (!params || !out) return set_err(MSM_ERR_INVALID_ARG, "params and out must not be NULL");
  if (params->max_atoms < 0) return set_err(MSM_ERR_INVALID_ARG, "max_atoms must be >= 0");
  msm_plan p = new (std::nothrow) msm_plan_s;
  if (!p) return set_err(MSM_ERR_CUDA, "out of host memory");
  std::string err;
  int rc = p->eng.build(params, &params->max_atoms, 1, true, &err);
  if (rc) {
    delete p;
    return set_err(rc, err);
  }
  *out = p;
  g_err.clear();
  return MSM_OK;
}

int msm_plan_destroy(msm_plan plan) {
  delete plan;
  return MSM_OK;
}

int msm_plan_get_info(msm_plan plan, msm_plan_info* info) {
  if (!plan || !info) return set_err(MSM_ERR_INVALID_ARG, "plan and info must not be NULL");
  fill_info(plan->eng.sys[0], info);
  info->anterp_tz = plan->eng.anterp_tz;
  info->short_block = plan->eng.short_block;
  info->anterp_kind = plan->eng.ant_wstride > 0 ? 1 : 0;
  info->level_method = plan->eng.level_method;
  info->spectral_ok = plan->eng.spec_ok ? 1 : 0;
  return MSM_OK;
}

int msm_set_level_method(msm_plan plan, int method) {
  if (!plan) return set_err(MSM_ERR_INVALID_ARG, "plan must not be NULL");
  std::string err;
  int rc = plan->eng.set_level_method(method, &err);
  if (rc) return set_err(rc, "msm_set_level_method: " + err);
  return MSM_OK;
}

int msm_plan_describe(const msm_params* params, msm_plan_info* info) {
  if (!params || !info) return set_err(MSM_ERR_INVALID_ARG, "params and info must not be NULL");
  SysHost S;
  std::string err;
  int rc = plan_system(*params, S, &err);
  if (rc) return set_err(rc, err);
  fill_info(S, info);
  info->anterp_kind = -1;
  return MSM_OK;
}

int msm_plan_stencil(const msm_params* params, int level, int which, float* out, size_t cap, int lo[3], int sz[3]) {
  if (!params || !lo || !sz) return set_err(MSM_ERR_INVALID_ARG, "NULL argument");
  if (which < 0 || which > 13) return set_err(MSM_ERR_INVALID_ARG, "which must be 0..13");
  SysHost S;
  std::string err;
  int rc = plan_system(*params, S, &err);
  if (rc) return set_err(rc, err);
  if (level < 1 || level > S.ncomp) return set_err(MSM_ERR_INVALID_ARG, "level out of range");
  const LevelHost& Lv = S.lev[level - 1];
  size_t count;
  const float* src;
  std::vector<float> tmp;
  if (which >= 7) {
    // the spectral level method's octant of this level's spectrum, as stored on the device
    bool ok = S.pbc[0] && S.pbc[1] && S.pbc[2] && !S.tri && Lv.kind == 0 && !S.kball.empty();
    for (int d = 0; d < 3 && ok; d++) ok = Lv.n[d] >= 2 && Lv.n[d] <= kSpecNmax && (Lv.n[d] & (Lv.n[d] - 1)) == 0;
    if (!ok) return set_err(MSM_ERR_UNSUPPORTED, "no spectral level method for this level");
    for (int d = 0; d < 3; d++) {
      lo[d] = 0;
      sz[d] = Lv.n[d] / 2 + 1;
    }
    count = (size_t)sz[0] * sz[1] * sz[2];
    tmp.resize(7 * count);
    level_spectra(S, level, Lv.n, tmp.data());
    src = tmp.data() + (size_t)(which - 7) * count;
  } else if (Lv.kind == 0) {
    for (int d = 0; d < 3; d++) {
      lo[d] = -S.R[d];
      sz[d] = 2 * S.R[d] + 1;
    }
    count = (size_t)sz[0] * sz[1] * sz[2];
    const double* v = which == 0 ? S.kball.data() : S.dk1.data() + (which - 1) * count;
    tmp.resize(count);
    for (size_t i = 0; i < count; i++) tmp[i] = (float)(v[i] * Lv.scale);
    src = tmp.data();
  } else {
    for (int d = 0; d < 3; d++) {
      lo[d] = Lv.blo[d];
      sz[d] = Lv.bsz[d];
    }
    count = (size_t)sz[0] * sz[1] * sz[2];
    src = which == 0 ? Lv.kbox.data() : Lv.dkbox.data() + (which - 1) * count;
  }
  if (!out) return MSM_OK;
  if (cap < count) return set_err(MSM_ERR_CAPACITY, "output buffer too small");
  std::memcpy(out, src, sizeof(float) * count);
  return MSM_OK;
}

int msm_workspace_bytes(msm_plan plan, size_t* bytes) {
  if (!plan || !bytes) return set_err(MSM_ERR_INVALID_ARG, "plan and bytes must not be NULL");
  *bytes = plan->eng.ws_bytes;
  return MSM_OK;
}

int msm_forward(msm_plan plan, void* workspace, size_t workspace_bytes, int n, const float* pos, const float* q,
                double* energy, float* phi, float* forces, int flags, void* stream) {
  if (!plan) return set_err(MSM_ERR_INVALID_ARG, "plan must not be NULL");
  if (n < 0 || n > plan->eng.total_atoms) return set_err(MSM_ERR_CAPACITY, "n outside [0, max_atoms]");
  return run_forward(plan->eng, workspace, workspace_bytes, n, pos, q, energy, phi, forces, flags,
                     (cudaStream_t)stream);
}

int msm_evaluate_host(msm_plan plan, void* workspace, size_t workspace_bytes, int n, const float* pos_host,
                      const float* q_host, double* energy_host, float* dE_dpos_host, float* dE_dq_host,
                      double* virial_host, void* stream) {
  if (!plan) return set_err(MSM_ERR_INVALID_ARG, "plan must not be NULL");
  if (n < 0 || n > plan->eng.total_atoms) return set_err(MSM_ERR_CAPACITY, "n outside [0, max_atoms]");
  return run_evaluate_host(plan->eng, workspace, workspace_bytes, n, pos_host, q_host, energy_host, dE_dpos_host,
                           dE_dq_host, virial_host, (cudaStream_t)stream);
}

int msm_backward(msm_plan plan, void* workspace, const double* grad_energy, float* dE_dpos, float* dE_dq,
                 double* virial, void* stream) {
  if (!plan) return set_err(MSM_ERR_INVALID_ARG, "plan must not be NULL");
  return run_backward(plan->eng, workspace, grad_energy, dE_dpos, dE_dq, virial, (cudaStream_t)stream);
}

// Vector-Jacobian product of the forces of the last forward on ws for an
// upstream u (n x 3, caller's order): L = sum_k u_k . F_k. With phi = A q (A
// symmetric), G(r) = sum_b q_b A(r, r_b) and psi(r) = sum_b p_b . d_2 A(r, r_b)
// the potential of the dipoles p_b = q_b u_b:
//   dL/dq_i = u_i . E_i - psi(r_i),   dL/dr_i = -q_i ((grad grad G)(r_i) u_i + grad psi(r_i)).
// The grid part of psi runs the dipole grid charge sum_b p_b . grad Phi_m(r_b)
// through the same restriction, stencils and prolongation as the charges.
// Consumes the workspace: a later msm_backward needs a new msm_forward.
static int run_force_vjp(Engine& E, void* ws, const float* u, float* dq, float* dpos, cudaStream_t s) {
  if (!E.have_fwd || ws != E.last_ws) return set_err(MSM_ERR_NO_FORWARD, "msm_force_vjp needs a prior msm_forward on this workspace");
  if (E.last_n > 0 && !u) return set_err(MSM_ERR_INVALID_ARG, "u must not be NULL");
  Work w = E.resolve(ws);
  Tables t = E.tables();
  const int nai = (int)E.atom_items.size();
  if ((E.last_flags & MSM_WANT_FORCES) == 0) {
    const bool had_w = (E.last_flags & MSM_WANT_VIRIAL) != 0;
    launch_short(w, t, E.d_atom_items, nai, true, had_w, s, E.p, E.short_code());
    launch_interp(w, t, E.d_atom_items, nai, true, s, E.p);
  }
  if (E.last_n > 0) {
    launch_sort_u(w, t, E.d_atom_items, nai, u, w.vjp_u, s);
    launch_interp_hess(w, t, E.d_atom_items, nai, w.vjp_u, s, E.p);  // f_sr <- ((H u)_grid, u . E)
    launch_short_fvjp(w, t, E.d_atom_items, nai, w.vjp_u, w.vjp_h, s, E.p, E.any_tri);
    launch_anterp_dipole(w, t, E.d_anterp_items, (int)E.anterp_items.size(), s, E.p, E.anterp_tz, w.vjp_u);
    for (int l = 1; l < E.maxcomp; l++) {
      int a = E.restrict_off[l - 1], b = E.restrict_off[l];
      launch_restrict(w, t, E.d_res_items + a, b - a, s, E.p);
    }
    E.stencils(w, t, s, false);
    for (int l = E.maxcomp - 1; l >= 1; l--) {
      int a = E.prolong_off[l - 1], b = E.prolong_off[l];
      launch_prolong(w, t, E.d_pro_items + a, b - a, s, E.p);
    }
    launch_interp(w, t, E.d_atom_items, nai, true, s, E.p);  // phi_lr <- psi_grid, f_lr <- -grad psi_grid
    launch_fvjp_final(w, t, E.d_atom_items, nai, w.vjp_h, dq, dpos, s);
  }
  E.have_fwd = false;
  return check_launch("msm_force_vjp");
}

// Vector-Jacobian product of the potentials of the last forward on ws for an
// upstream g (n, caller's order): L = sum_k g_k phi_k, phi = A q with A
// symmetric, so dL/dq = A g and dL/dr_k = -g_k E_k(q) - q_k E_k(g). The field
// of q is kept, the method runs once more with charges g on the forward's
// sorted positions and bins (short range on the second stream, overlapping
// the grid chain, as in the forward), and a last kernel combines the two.
// Consumes the workspace.
static int run_potential_vjp(Engine& E, void* ws, const float* g, float* dq, float* dpos, cudaStream_t s) {
  if (!E.have_fwd || ws != E.last_ws)
    return set_err(MSM_ERR_NO_FORWARD, "msm_potential_vjp needs a prior msm_forward on this workspace");
  if (E.last_n > 0 && !g) return set_err(MSM_ERR_INVALID_ARG, "g must not be NULL");
  Work w = E.resolve(ws);
  Tables t = E.tables();
  const int nai = (int)E.atom_items.size();
  if ((E.last_flags & MSM_WANT_FORCES) == 0) {
    const bool had_w = (E.last_flags & MSM_WANT_VIRIAL) != 0;
    launch_short(w, t, E.d_atom_items, nai, true, had_w, s, E.p, E.short_code());
    launch_interp(w, t, E.d_atom_items, nai, true, s, E.p);
  }
  if (E.last_n > 0) {
    launch_pvjp_prep(w, t, E.d_atom_items, nai, g, s);
    E.anterp(w, t, s);
    cudaEventRecord(E.ev_fork, s);
    cudaStreamWaitEvent(E.side, E.ev_fork, 0);
    launch_short(w, t, E.d_atom_items, nai, true, false, E.side, E.p, E.short_code());
    cudaEventRecord(E.ev_join, E.side);
    for (int l = 1; l < E.maxcomp; l++) {
      int a = E.restrict_off[l - 1], b = E.restrict_off[l];
      launch_restrict(w, t, E.d_res_items + a, b - a, s, E.p);
    }
    E.stencils(w, t, s, false);
    for (int l = E.maxcomp - 1; l >= 1; l--) {
      int a = E.prolong_off[l - 1], b = E.prolong_off[l];
      launch_prolong(w, t, E.d_pro_items + a, b - a, s, E.p);
    }
    launch_interp(w, t, E.d_atom_items, nai, true, s, E.p);
    cudaStreamWaitEvent(s, E.ev_join, 0);
    launch_pvjp_final(w, t, E.d_atom_items, nai, dq, dpos, s);
  }
  E.have_fwd = false;
  return check_launch("msm_potential_vjp");
}

int msm_potential_vjp(msm_plan plan, void* workspace, const float* g, float* dL_dq, float* dL_dpos, void* stream) {
  if (!plan) return set_err(MSM_ERR_INVALID_ARG, "plan must not be NULL");
  return run_potential_vjp(plan->eng, workspace, g, dL_dq, dL_dpos, (cudaStream_t)stream);
}

int msm_batch_potential_vjp(msm_batch batch, void* workspace, const float* g, float* dL_dq, float* dL_dpos,
                            void* stream) {
  if (!batch) return set_err(MSM_ERR_INVALID_ARG, "batch must not be NULL");
  return run_potential_vjp(batch->eng, workspace, g, dL_dq, dL_dpos, (cudaStream_t)stream);
}

int msm_force_vjp(msm_plan plan, void* workspace, const float* u, float* dL_dq, float* dL_dpos, void* stream) {
  if (!plan) return set_err(MSM_ERR_INVALID_ARG, "plan must not be NULL");
  return run_force_vjp(plan->eng, workspace, u, dL_dq, dL_dpos, (cudaStream_t)stream);
}

int msm_batch_force_vjp(msm_batch batch, void* workspace, const float* u, float* dL_dq, float* dL_dpos,
                        void* stream) {
  if (!batch) return set_err(MSM_ERR_INVALID_ARG, "batch must not be NULL");
  return run_force_vjp(batch->eng, workspace, u, dL_dq, dL_dpos, (cudaStream_t)stream);
}

int msm_plan_set_cell(msm_plan plan, const double* cell, void* stream) {
  if (!plan || !cell) return set_err(MSM_ERR_INVALID_ARG, "plan and cell must not be NULL");
  Engine& E = plan->eng;
  SysHost& S = E.sys[0];
  for (int i = 0; i < 9; i++)
    if (!std::isfinite(cell[i])) return set_err(MSM_ERR_INVALID_ARG, "cell has a non-finite entry");
  if (S.tri) {
    // a plan built for a tilted cell takes any right-handed cell within its capacity
    std::string err;
    int rc = E.set_cell_tilted(cell, (cudaStream_t)stream, &err);
    if (rc) return set_err(rc, "msm_plan_set_cell: " + err);
    E.have_fwd = false;
    return check_launch("msm_plan_set_cell");
  }
  for (int i = 0; i < 9; i++)
    if (i % 4 != 0 && cell[i] != 0.0)
      return set_err(MSM_ERR_UNSUPPORTED, "a plan built for a rectangular cell takes rectangular cells only");
  for (int d = 0; d < 3; d++)
    if (!(cell[4 * d] > 0.0)) return set_err(MSM_ERR_INVALID_ARG, "cell lengths must be > 0");
  double h1[3];
  int Snew[3];
  for (int d = 0; d < 3; d++) {
    h1[d] = cell[4 * d] / S.M[d];
    Snew[d] = std::max(0, (int)std::ceil(2.0 * S.a / h1[d]) - 1);
    // the plan's arrays hold samples out to R - hw (its sample radius at creation)
    if (Snew[d] > S.R[d] - S.hw)
      return set_err(MSM_ERR_CAPACITY, "cell compressed beyond the plan's stencil radius: create the plan for the "
                                       "most compressed cell it must serve");
  }
  SysDev D = E.hsys[0];
  for (int d = 0; d < 3; d++) {
    S.L[d] = cell[4 * d];
    S.h1[d] = h1[d];
    S.S[d] = Snew[d];
    S.edge[d] = S.L[d] / S.C[d];
    S.nnbr[d] = (int)std::ceil(S.a / S.edge[d]);
    D.Ld[d] = S.L[d];
    D.edged[d] = S.edge[d];
    D.edge[d] = (float)S.edge[d];
    D.invL[d] = (float)(1.0 / S.L[d]);
    D.inv_h1[d] = (float)(1.0 / S.h1[d]);
    D.Lf[d] = (float)S.L[d];
    D.h1f[d] = (float)S.h1[d];
    D.nnbr[d] = S.nnbr[d];
  }
  E.hsys[0] = D;
  E.have_fwd = false;  // the workspace holds results for the old cell
  bool device_path = S.pbc[0] && S.pbc[1] && S.pbc[2] && S.prefilter;
  for (const LevelHost& Lv : S.lev) device_path = device_path && Lv.kind == 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (device_path) {
    // every level a ball of raw samples: pointwise in h_1, computed on the device
    const int hz = (S.B[2] + 3) & ~3;
    launch_cell_update(E.d_sys, D, S.h1, S.a, S.p, S.B, hz, S.kball_off, S.dkh_off, S.wb_off, S.wh_off, E.d_kpool,
                       E.d_wpool, st);
    // the spectral level method's spectra, from the same raw samples (separable sums on the device)
    if (E.spec_ok)
      launch_spec_cell(S.h1, S.a, S.p, S.B, S.omh.data(), S.hw, (int)E.spec_n.size(), E.spec_n.data(),
                       E.spec_sp.data(), E.d_spec_scr_a, E.d_spec_scr_b, E.d_kpool, st);
  } else {
    // omega'-convolved stencils and folded boxes: rebuilt on the host with the
    // plan's sizes, copied through pinned staging buffers (stream-ordered)
    std::string err;
    int rc = E.set_cell_host(S.L, st, &err);
    if (rc) return set_err(rc, "msm_plan_set_cell: " + err);
    launch_set_sys(E.d_sys, D, st);
  }
  return check_launch("msm_plan_set_cell");
}

int msm_field(msm_plan plan, void* workspace, float* field, void* stream) {
  if (!plan) return set_err(MSM_ERR_INVALID_ARG, "plan must not be NULL");
  return run_field(plan->eng, workspace, field, (cudaStream_t)stream);
}

int msm_autotune(msm_plan plan, void* workspace, size_t workspace_bytes, int n, const float* pos, const float* q,
                 void* stream) {
  if (!plan) return set_err(MSM_ERR_INVALID_ARG, "plan must not be NULL");
  if (n < 0 || n > plan->eng.total_atoms) return set_err(MSM_ERR_CAPACITY, "n outside [0, max_atoms]");
  return run_autotune(plan->eng, workspace, workspace_bytes, n, pos, q, (cudaStream_t)stream);
}

static_assert(MSM_SHORT_CLUSTER == kShortCluster, "public and internal cluster-kernel codes agree");

static int set_tuning(Engine& E, int anterp_tz, int short_block) {
  if (short_block != kChunk && short_block != kChunk / 2 && short_block != kShortCluster)
    return set_err(MSM_ERR_INVALID_ARG, "short_block must be 128, 256 or MSM_SHORT_CLUSTER");
  if (short_block == kShortCluster && !E.cluster_ok())
    return set_err(MSM_ERR_INVALID_ARG,
                   "MSM_SHORT_CLUSTER needs rectangular cells, nnbr <= 4 along x and y and L_z >= a + 2 e_z");
  std::string err;
  int rc = E.set_anterp_tz(anterp_tz, &err);
  if (rc) return set_err(rc, err);
  E.short_block = short_block;
  return MSM_OK;
}

int msm_set_tuning(msm_plan plan, int anterp_tz, int short_block) {
  if (!plan) return set_err(MSM_ERR_INVALID_ARG, "plan must not be NULL");
  return set_tuning(plan->eng, anterp_tz, short_block);
}

int msm_status(msm_plan plan, void* workspace, void* stream, int* device_status) {
  if (!plan) return set_err(MSM_ERR_INVALID_ARG, "plan must not be NULL");
  return read_status(plan->eng, workspace, (cudaStream_t)stream, device_status);
}

int msm_debug_offset(msm_plan plan, int which, int level, size_t* offset_bytes, size_t* count) {
  if (!plan || !offset_bytes || !count) return set_err(MSM_ERR_INVALID_ARG, "NULL argument");
  const Engine& E = plan->eng;
  switch (which) {
    case 0: *offset_bytes = E.L_cell_start; *count = (size_t)E.total_cells + 1; return MSM_OK;
    case 1: *offset_bytes = E.L_perm; *count = (size_t)E.total_atoms; return MSM_OK;
    case 4: *offset_bytes = E.L_scell; *count = (size_t)E.total_atoms; return MSM_OK;
    case 2:
    case 3: {
      const SysHost& S = E.sys[0];
      if (level < 1 || level > S.ncomp) return set_err(MSM_ERR_INVALID_ARG, "level out of range");
      const LevDev& L = E.hlev[level - 1];
      *offset_bytes = E.L_grid + sizeof(float) * (size_t)(which == 2 ? L.q_off : L.e_off);
      *count = (size_t)L.n[0] * L.n[1] * L.n[2];
      return MSM_OK;
    }
    default: return set_err(MSM_ERR_INVALID_ARG, "unknown array");
  }
}

int msm_batch_create(const msm_params* per_sys, const int* n_per_sys, int nsys, msm_batch* out) {
  if (!per_sys || !n_per_sys || !out || nsys <= 0) return set_err(MSM_ERR_INVALID_ARG, "bad batch arguments");
  msm_batch b = new (std::nothrow) msm_batch_s;
  if (!b) return set_err(MSM_ERR_CUDA, "out of host memory");
  std::string err;
  int rc = b->eng.build(per_sys, n_per_sys, nsys, false, &err);
  if (rc) {
    delete b;
    return set_err(rc, err);
  }
  *out = b;
  g_err.clear();
  return MSM_OK;
}

int msm_batch_destroy(msm_batch batch) {
  delete batch;
  return MSM_OK;
}

int msm_batch_workspace_bytes(msm_batch batch, size_t* bytes) {
  if (!batch || !bytes) return set_err(MSM_ERR_INVALID_ARG, "batch and bytes must not be NULL");
  *bytes = batch->eng.ws_bytes;
  return MSM_OK;
}

int msm_batch_forward(msm_batch batch, void* workspace, size_t workspace_bytes, const float* pos, const float* q,
                      double* energy, float* phi, float* forces, int flags, void* stream) {
  if (!batch) return set_err(MSM_ERR_INVALID_ARG, "batch must not be NULL");
  return run_forward(batch->eng, workspace, workspace_bytes, -1, pos, q, energy, phi, forces, flags,
                     (cudaStream_t)stream);
}

int msm_batch_backward(msm_batch batch, void* workspace, const double* grad_energy, float* dE_dpos, float* dE_dq,
                       double* virial, void* stream) {
  if (!batch) return set_err(MSM_ERR_INVALID_ARG, "batch must not be NULL");
  return run_backward(batch->eng, workspace, grad_energy, dE_dpos, dE_dq, virial, (cudaStream_t)stream);
}

int msm_batch_field(msm_batch batch, void* workspace, float* field, void* stream) {
  if (!batch) return set_err(MSM_ERR_INVALID_ARG, "batch must not be NULL");
  return run_field(batch->eng, workspace, field, (cudaStream_t)stream);
}

int msm_batch_autotune(msm_batch batch, void* workspace, size_t workspace_bytes, const float* pos, const float* q,
                       void* stream) {
  if (!batch) return set_err(MSM_ERR_INVALID_ARG, "batch must not be NULL");
  return run_autotune(batch->eng, workspace, workspace_bytes, -1, pos, q, (cudaStream_t)stream);
}

int msm_batch_set_tuning(msm_batch batch, int anterp_tz, int short_block) {
  if (!batch) return set_err(MSM_ERR_INVALID_ARG, "batch must not be NULL");
  return set_tuning(batch->eng, anterp_tz, short_block);
}

int msm_batch_get_tuning(msm_batch batch, int* anterp_tz, int* short_block) {
  if (!batch || !anterp_tz || !short_block) return set_err(MSM_ERR_INVALID_ARG, "NULL argument");
  *anterp_tz = batch->eng.anterp_tz;
  *short_block = batch->eng.short_block;
  return MSM_OK;
}

int msm_batch_status(msm_batch batch, void* workspace, void* stream, int* device_status) {
  if (!batch) return set_err(MSM_ERR_INVALID_ARG, "batch must not be NULL");
  return read_status(batch->eng, workspace, (cudaStream_t)stream, device_status);
}

}  // extern "C"
