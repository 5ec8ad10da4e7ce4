/*
 * msm_gb300.h -- C ABI of the GB300 (sm_103a) multilevel summation method.
 *
 * The method is the B-spline multilevel summation method (MSM) of arXiv
 * 2510.05961 (msmJAX), Sec. 2 and 3: the Coulomb energy of N point charges,
 * U = 1/2 sum_i sum_(j != i) q_i q_j / r_ij (Eq. generic_pair_potential_sum),
 * split into a short-range part U^0 evaluated pair by pair (Eq. U_zero) and a
 * long-range part U^(1+) evaluated on a hierarchy of grids (Eqs. grid_charge,
 * u_oneplus_nested_eval, uoneplus_interpolation). Units are those of the
 * inputs; the Coulomb constant is 1 (Sec. 3.6).
 *
 * Conventions shared by every call:
 *  - Plain C types only. Device pointers point to CUDA device memory of the
 *    current device; host pointers are marked "host".
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call is stream-ordered and returns without waiting for the GPU,
 *    except msm_status, which synchronises the stream.
 *  - The caller owns and allocates every input, output and workspace buffer.
 *    A plan owns only its host settings and its device constant tables
 *    (stencils, work lists), allocated by msm_plan_create and freed by
 *    msm_plan_destroy.
 *  - Return value: MSM_OK (0) or an MSM_ERR_* code; msm_last_error() then
 *    holds a message (per thread). Problems found on the GPU while running
 *    (an atom outside an open cell, a non-finite input) do not fail the call:
 *    they set bits in a device status word that msm_status reads; the
 *    outputs of such a call are unspecified.
 *  - Positions are Cartesian, row-major n x 3 (x,y,z per atom), float32.
 *    Along a periodic axis any value is allowed (it is wrapped); along an open
 *    axis 0 <= x <= L is required.
 *  - All arithmetic on the GPU is float32 with float64 final sums of the
 *    energy and the virial.
 */
#ifndef MSM_GB300_H
#define MSM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define MSM_OK 0
#define MSM_ERR_INVALID_ARG 1  /* a NULL pointer, a size out of range, bad settings */
#define MSM_ERR_UNSUPPORTED 2  /* settings outside what this build implements */
#define MSM_ERR_CUDA 3         /* a CUDA runtime call failed */
#define MSM_ERR_NO_FORWARD 4   /* msm_backward without a prior msm_forward on the workspace */
#define MSM_ERR_CAPACITY 5     /* n above the plan's max_atoms, or a workspace too small */

/* bits of the device status word (msm_status) */
#define MSM_DEV_OUT_OF_CELL 1  /* an atom outside [0, L] along an open axis */
#define MSM_DEV_NONFINITE 2    /* a NaN or infinite position or charge */
/* A warning, not an error: a system with a periodic axis whose total charge
 * is not zero, |sum q| > 1e-5 sum |q| (set by msm_forward). The paper's
 * method assumes neutral periodic systems (Sec. 4.1: the dropped one-point
 * top level holds sum q); it prescribes no background correction, so none is
 * applied and the outputs are those of the method as defined (the dropped
 * top level, and the left-out lattice-sum constant of slabs and wires, then
 * omit a term proportional to (sum q)^2). */
#define MSM_DEV_NON_NEUTRAL 4
/* Debug builds only (compiled with -DMSM_CHECKS=1): a kernel found a
 * data-dependent index outside its array and skipped the access. A stand-in
 * for a device memory checker; normal builds never set it. */
#define MSM_DEV_CHECK 8
#define MSM_DEV_ERRORS (MSM_DEV_OUT_OF_CELL | MSM_DEV_NONFINITE | MSM_DEV_CHECK)  /* outputs unspecified */

/* msm_forward flags */
#define MSM_WANT_FORCES 1      /* compute forces in the forward pass */
#define MSM_WANT_VIRIAL 2      /* keep what msm_backward needs for the virial */

typedef struct msm_plan_s* msm_plan;
typedef struct msm_batch_s* msm_batch;

/* Settings of one system; the arguments of the paper's set_up_msm_params
 * (Sec. 3.5): cell, periodicity, level-one spacing, level-zero cutoff, order.
 *  cell[9]        row-major 3x3 cell matrix, rows = cell vectors a, b, c, a
 *                 right-handed basis. Off-diagonal entries (a tilted cell,
 *                 Sec. 3.2.2's transform to the unit cube: grids in the
 *                 fractional coordinates s = A^-T r) need pbc 1, 1, 1; L below
 *                 is then the length of each cell vector, the stencils follow
 *                 the cell's metric (ball kernels with shifted column
 *                 centres). A plan built for a tilted cell takes any later
 *                 right-handed cell in msm_plan_set_cell; a rectangular plan
 *                 only rectangular ones.
 *  pbc[3]         1 = periodic along that axis, 0 = open. Any combination:
 *                 three periodic axes drop the one-point top level (zero for
 *                 a neutral cell, Sec. 4.1); two (a slab) or one (a wire)
 *                 keep it, with the level-L kernel summed over the 2-D or
 *                 1-D lattice of the periodic axes (the divergent constant,
 *                 which multiplies the squared total charge, left out).
 *  h              target level-1 grid spacing h_1 (> 0 unless overridden).
 *                 Periodic axes use M = 2^round(log2(L/h)) intervals (all
 *                 periodic axes must give the same M); open axes M = ceil(L/h).
 *  grid_override  > 0: use exactly this many level-1 intervals on that axis
 *                 (a power of two on periodic axes).
 *  cutoff         level-zero cutoff a = r_cut^(0) (> 0).
 *  order          B-spline order p: 4, 6 or 8.
 *  levels         number of grid levels L; 0 = automatic. With any periodic
 *                 axis L = log2(M) + 1 is fixed (spacing doubles until one
 *                 point remains, Sec. 4.1) and any other value is rejected.
 *  qi_mode        interpolation of the grid kernels (Sec. 3.4, the omega'
 *                 coefficients of Eq. kernel_stencil_by_conv_with_universal_coeff):
 *                 0 = minimal quasi-interpolation (half-width p/2 - 1, the
 *                 default); 1 = exact interpolation, omega' = omega * omega with
 *                 omega the inverse of the sampled B-spline (Phi_p(n))_n,
 *                 truncated where |omega'_n| < 1e-12 |omega'_0| (half-width 23,
 *                 36, 49 for p = 4, 6, 8): an accuracy reference whose stencils
 *                 are wider than the ball kernels take, so every level runs the
 *                 dense folded-box kernel (practical for grids up to ~32^3).
 *  max_atoms      largest n a forward call may pass (sizes the workspace). */
typedef struct {
  double cell[9];
  int pbc[3];
  double h;
  int grid_override[3];
  double cutoff;
  int order;
  int levels;
  int qi_mode;
  int max_atoms;
} msm_params;

/* Derived sizes of a plan (msm_plan_get_info), for inspection and tests. */
typedef struct {
  int nlev;          /* grid levels L, top level included */
  int ncomp;         /* levels whose grids are evaluated (L, or L-1 when the
                        one-point top level of a periodic system is dropped) */
  int M[3];          /* level-1 interval counts */
  double h1[3];      /* level-1 spacings */
  int lo[20][3];     /* first grid index of each evaluated level */
  int n[20][3];      /* grid points of each evaluated level */
  int R[3];          /* stencil radius of the levels below the top */
  int C[3];          /* binning cells per axis */
  int nnbr[3];       /* neighbour-cell reach per axis */
  int stencil_kind[20]; /* 0 = ball stencil with wrap/zero, 1 = dense folded box */
  int anterp_tz;     /* anterpolation tile z-extent in use (16, 32, 64; msm_autotune) */
  int short_block;   /* short-range kernel in use: 128 or 256 threads per block of the per-atom
                        kernel, or MSM_SHORT_CLUSTER (cluster-pair tiles); msm_autotune */
  int anterp_kind;   /* anterpolation in use: 1 = by binning columns (column partials, then their
                        sum per grid point), 0 = gather by grid columns (footprints too wide for
                        the column kernel at this tile z-extent); -1 from msm_plan_describe */
  int level_method;  /* level stencils in use: MSM_LEVELS_BALL or MSM_LEVELS_SPECTRAL (0 from
                        msm_plan_describe) */
  int spectral_ok;   /* 1 if the plan allows MSM_LEVELS_SPECTRAL (0 from msm_plan_describe) */
} msm_plan_info;

/* Create a plan: validates the settings synchronously, builds the level
 * stencils K^l (Eq. kernel_stencil_by_conv_with_universal_coeff) and their
 * strain derivatives in FP64 on the host, and uploads them to the current
 * device. *out receives the plan; free it with msm_plan_destroy. */
int msm_plan_create(const msm_params* params, msm_plan* out);
int msm_plan_destroy(msm_plan plan);
int msm_plan_get_info(msm_plan plan, msm_plan_info* info);

/* Dynamic cell (Sec. 3.2.2: with a changing cell the stencils K^l must be
 * recomputed, as they sample the level kernels on grids that scale with the
 * cell; Sec. 4.1 lists the limits of fixed-size stencil arrays). Gives the
 * plan a new orthorhombic cell while keeping its grid counts M, level ranges,
 * binning cells and stencil array sizes: the level-1 spacings become
 * h_1 = L / M and the stencils, the virial weights, the column tables and
 * the system descriptor are recomputed, stream-ordered: on the device for a
 * periodic system of order 4 with qi_mode 0 (every level a ball of raw
 * samples, no host synchronisation), otherwise on the host with the plan's
 * array sizes and copied from pinned staging buffers (the call then waits
 * for the previous call's copy only).
 *  cell    host, 9 doubles, row-major, diagonal (as msm_params.cell;
 *          MSM_ERR_UNSUPPORTED for other cells).
 * The new cell may expand freely (coarser spacings lower the accuracy, as
 * the paper notes); it may be compressed only while ceil(2 a / h_1) - 1 stays
 * within the sample radius the plan was built with (MSM_ERR_CAPACITY
 * otherwise: create the plan for the most compressed cell it must serve).
 * Open axes need the positions inside the new cell. A later msm_backward
 * needs a new msm_forward. */
int msm_plan_set_cell(msm_plan plan, const double* cell, void* stream);

/* Host-only (no device needed): the plan msm_plan_create would build from
 * params, described in *info. Same validation and return codes. */
int msm_plan_describe(const msm_params* params, msm_plan_info* info);

/* Host-only: the stencil a plan applies on level `level` (1-based), as float
 * values on the offset box [lo, lo + sz) (z fastest), which = 0 for K^l
 * (Eq. kernel_stencil_by_conv_with_universal_coeff), 1..6 for the strain
 * derivatives dK^l/d eps_ab, ab = xx, yy, zz, xy, xz, yz. Ball levels are
 * returned unfolded on [-R, R] (the kernel wraps indices), box levels folded
 * along periodic axes onto [0, n). which = 7 .. 13: the spectra the spectral
 * level method (MSM_LEVELS_SPECTRAL) stores for the level, on the octant
 * k_d = 0 .. n_d / 2 (lo = 0, sz = n_d / 2 + 1): 7 the discrete Fourier
 * transform of the folded K^l times 1/N, 8 .. 13 those of dK^l/d eps_ab times
 * -1/2 (1/N), N the level's point count (MSM_ERR_UNSUPPORTED for levels
 * without it). out (host, capacity `cap` floats) may be NULL to query lo and
 * sz only. MSM_ERR_CAPACITY if cap is too small. */
int msm_plan_stencil(const msm_params* params, int level, int which, float* out, size_t cap, int lo[3], int sz[3]);

/* Bytes of device workspace a plan needs (for max_atoms atoms). The caller
 * allocates it (any device allocator; 256-byte alignment or better) and passes
 * it, unchanged between msm_forward and msm_backward, to every call. */
int msm_workspace_bytes(msm_plan plan, size_t* bytes);

/* Forward pass: energy, potentials and (optionally) forces of n atoms.
 *  pos     device, n x 3 float32 Cartesian positions (row-major).
 *  q       device, n float32 charges.
 *  energy  device, 1 double: E = 1/2 sum_i q_i phi_i.
 *  phi     device, n float32 or NULL: phi_i = dE/dq_i (Eq.
 *          analytic_uoneplus_charge_grad plus the short-range part and the
 *          self term).
 *  forces  device, n x 3 float32 or NULL: F_i = -dE/dr_i (Eq.
 *          analytic_uoneplus_position_grad plus the short-range part).
 *          Needs MSM_WANT_FORCES.
 *  flags   MSM_WANT_FORCES | MSM_WANT_VIRIAL.
 * Returns MSM_ERR_CAPACITY if n > max_atoms or workspace_bytes is too small. */
int msm_forward(msm_plan plan, void* workspace, size_t workspace_bytes, int n, const float* pos,
                const float* q, double* energy, float* phi, float* forces, int flags, void* stream);

/* Backward pass for an upstream gradient g = dL/dE (device, 1 double),
 * reusing the sorted bins, the level grids and the per-atom results the last
 * msm_forward left in the workspace. Outputs (any may be NULL):
 *  dE_dpos device, n x 3 float32: g * dE/dr_i = -g F_i.
 *  dE_dq   device, n float32: g * phi_i.
 *  virial  device, 9 doubles (row-major): g * W with W = -dE/d(eps) for the
 *          homogeneous strain r -> (1+eps) r, cell -> (1+eps) cell.
 * What the forward did not compute (forces, the short-range virial) is
 * computed here. Returns MSM_ERR_NO_FORWARD without a prior forward. */
int msm_backward(msm_plan plan, void* workspace, const double* grad_energy, float* dE_dpos, float* dE_dq,
                 double* virial, void* stream);

/* End-to-end evaluation on host buffers: copies the inputs to the device (into
 * the workspace), evaluates forward and backward with dL/dE = 1 (the forward
 * writes dE/dpos = -F and dE/dq = phi directly, the values msm_backward would
 * give), copies E, dE/dpos, dE/dq and, if virial_host is not NULL, W back, and
 * waits for the copies. The per-atom gradients are copied while the grid
 * virial is formed (a second stream). Unlike the other calls this one returns
 * only after the results are on the host.
 *  pos_host      host, n x 3 float32 (page-locked memory makes the copies asynchronous).
 *  q_host        host, n float32.
 *  energy_host   host, 1 double.
 *  dE_dpos_host  host, n x 3 float32; dE_dq_host host, n float32.
 *  virial_host   host, 9 doubles (row-major 3x3), or NULL to skip the virial.
 * The workspace must have msm_workspace_bytes (it includes the staging arrays);
 * afterwards it holds the forward's state like msm_forward (a later msm_field,
 * msm_force_vjp or msm_potential_vjp may follow). */
int msm_evaluate_host(msm_plan plan, void* workspace, size_t workspace_bytes, int n, const float* pos_host,
                      const float* q_host, double* energy_host, float* dE_dpos_host, float* dE_dq_host,
                      double* virial_host, void* stream);

/* The field E_i = -grad phi(r_i) of the MSM potential at every atom (the
 * gradient of Eq. U_total's phi with respect to the evaluation point, both
 * the short-range and the interpolated part; the force is F_i = q_i E_i),
 * from the last msm_forward on workspace.
 *  field  device, n x 3 float32, the caller's atom order.
 * It is what the gradient of sum_i g_i phi_i needs (phi = A q with A
 * symmetric: d/dq = A g, d/dr_k = -g_k E_k(q) - q_k E_k(g), the second field
 * from an evaluation with charges g), and it needs no division by q.
 * Stream-ordered; computes the field parts if that forward skipped forces.
 * Returns MSM_ERR_NO_FORWARD without a prior forward on workspace. */
int msm_field(msm_plan plan, void* workspace, float* field, void* stream);

/* Vector-Jacobian product of the forces of the last msm_forward on workspace
 * (the derivatives of Sec. 3.2.2 taken once more, for training through the
 * forces): for an upstream u, L = sum_k u_k . F_k,
 *   dL/dq_i = u_i . E_i - psi(r_i),
 *   dL/dr_i = -q_i ((grad grad G)(r_i) u_i + grad psi(r_i)),
 * with E the field (msm_field), G(r) = sum_b q_b A(r, r_b) the potential of
 * the charges as a function of the evaluation point and psi the potential of
 * the dipoles p_b = q_b u_b (phi = A q with A symmetric). The grid part of psi
 * sends the dipole grid charge sum_b p_b . grad Phi_m(r_b) through the same
 * restriction, stencils and prolongation as the charges; the short-range part
 * and the pair Hessians use k_0, k_0', k_0''.
 *  u        device, n x 3 float32, caller's order.
 *  dL_dq    device, n float32, or NULL.
 *  dL_dpos  device, n x 3 float32, or NULL.
 * Stream-ordered. Consumes the workspace: a later msm_backward needs a new
 * msm_forward. Returns MSM_ERR_NO_FORWARD without a prior forward. */
int msm_force_vjp(msm_plan plan, void* workspace, const float* u, float* dL_dq, float* dL_dpos, void* stream);

/* Vector-Jacobian product of the potentials of the last msm_forward on
 * workspace (Sec. 3.2.2's derivatives of phi, for training through the
 * potentials, e.g. an MLIP with predicted charges): for an upstream g,
 * L = sum_k g_k phi_k. phi = A q with A symmetric (the short-range kernel,
 * the self term and the grid chain Phi^T K Phi are symmetric), so
 *   dL/dq_i = (A g)_i                          (the potentials of charges g),
 *   dL/dr_i = -g_i E_i(q) - q_i E_i(g)          (E = -grad phi, the field).
 * The library keeps the field of q from the forward, evaluates the method
 * once more with charges g on the same sorted positions and bins (short
 * range, anterpolation, restrictions, stencils, prolongations,
 * interpolation, all in its kernels) and combines the two in a final kernel.
 *  g        device, n float32, caller's order.
 *  dL_dq    device, n float32, or NULL.
 *  dL_dpos  device, n x 3 float32, or NULL.
 * Stream-ordered. Consumes the workspace: a later msm_backward, msm_field or
 * msm_force_vjp needs a new msm_forward. Returns MSM_ERR_NO_FORWARD without
 * a prior forward, MSM_ERR_INVALID_ARG if g is NULL for n > 0. */
int msm_potential_vjp(msm_plan plan, void* workspace, const float* g, float* dL_dq, float* dL_dpos, void* stream);

/* Autotuner (no counterpart in the paper, whose JAX code leaves launch shapes
 * to XLA): runs one forward on (n, pos, q) to fill workspace, then times each
 * tunable launch shape on those inputs and keeps the fastest for every later
 * call on this plan: the z-extent of the anterpolation tiles (16, 32, 64
 * level-1 points) and the short-range kernel (the per-atom kernel with 256
 * threads per block, or 128 = two blocks per 256-atom item, or, where the plan
 * allows it, MSM_SHORT_CLUSTER: cluster-pair tiles) and, where the plan allows
 * the spectral method, the level method (the forward's stencils with the
 * backward's grid virial). Arguments as msm_forward. Synchronises stream
 * (not capturable into a graph); afterwards msm_backward needs a new
 * msm_forward. The choices are reported by msm_plan_get_info. */
int msm_autotune(msm_plan plan, void* workspace, size_t workspace_bytes, int n, const float* pos, const float* q,
                 void* stream);

/* Short-range kernel code for short_block: Eq. U_zero's pair sums as
 * cluster-pair tiles (one warp per cluster of 4 sorted atoms: candidates culled
 * against the cluster's bounding box into a shared-memory queue, then 4 x 8 pair
 * tiles). Allowed when every system of the plan has a rectangular cell, a
 * neighbour-cell reach nnbr of at most 4 along x and y and, when z is periodic,
 * L_z >= a + 2 e_z (e_z the binning cell edge along z); where a later
 * msm_plan_set_cell breaks this, the plan runs the per-atom kernel (256 threads)
 * until the condition holds again. Same sums, reproducible bit for bit. */
#define MSM_SHORT_CLUSTER 4

/* Sets the tuned launch shapes directly (for callers that keep earlier
 * msm_autotune results): anterp_tz in {16, 32, 64}, short_block in {128, 256,
 * MSM_SHORT_CLUSTER}; MSM_ERR_INVALID_ARG otherwise, or for MSM_SHORT_CLUSTER on
 * a plan that does not allow it. Host-side; affects the next calls. */
int msm_set_tuning(msm_plan plan, int anterp_tz, int short_block);

/* Level methods: how the level stencils K^l of Eq. action_of_K_as_convolution
 * (and, in the backward, the grid virial -1/2 q~^T dK^l q~ of every level) are
 * applied.
 *  MSM_LEVELS_BALL: stencil sums over a halo-padded copy of each level grid
 *    (ball kernels; every plan).
 *  MSM_LEVELS_SPECTRAL: on a periodic grid the stencil sum is a circular
 *    convolution with the stencil folded onto the grid, so it is applied as a
 *    product with the stencil's discrete Fourier transform (the unfolded
 *    stencil's transform sampled at k / n: the same operator, up to FP32
 *    rounding), between forward and inverse three-dimensional FFTs of the level
 *    grid; the virial is the sum over k of dK^(k) |Q(k)|^2 / N (Parseval),
 *    formed during the forward. Plans that allow it: a single system with a
 *    fully periodic rectangular cell whose evaluated levels have 2 .. 256 points
 *    per axis (the planner's periodic grids are powers of two), as reported by
 *    msm_plan_info.spectral_ok. The spectra are computed on the host (FP64) at
 *    plan creation; msm_plan_set_cell recomputes them with the stencils, on the
 *    device for p = 4 plans (separable sums over the raw samples, FP32) and on
 *    the host otherwise, whichever method the plan runs.
 * New plans run MSM_LEVELS_BALL; msm_autotune picks the faster method. */
#define MSM_LEVELS_BALL 0
#define MSM_LEVELS_SPECTRAL 1

/* Selects the level method of a single-system plan (host-side; affects the next
 * calls; a following msm_backward needs a new msm_forward). MSM_ERR_INVALID_ARG
 * for an unknown method, MSM_ERR_UNSUPPORTED for MSM_LEVELS_SPECTRAL on a plan
 * that does not allow it. */
int msm_set_level_method(msm_plan plan, int method);

/* Synchronises stream and returns the device status word (MSM_DEV_* bits)
 * of the last call on workspace in *device_status (host). */
int msm_status(msm_plan plan, void* workspace, void* stream, int* device_status);

/* Byte offset and element count, inside the workspace, of an internal array
 * (for tests): which = 0 cell_start (int32, cells+1), 1 perm (int32, sorted
 * slot -> atom), 2 grid charge of level `level` (float32, z fastest),
 * 3 grid potential e of level `level` (after prolongation: e^(l+)),
 * 4 sorted cell id of each sorted slot (int32). */
int msm_debug_offset(msm_plan plan, int which, int level, size_t* offset_bytes, size_t* count);

/* Phase timing. With profiling enabled, msm_forward / msm_backward record a
 * CUDA event pair on the call's stream around each phase; msm_profile_read
 * synchronises those events and returns, per phase, the milliseconds of the
 * most recent forward and backward (host, ms[MSM_NPHASE]) and the number of
 * kernels those two calls launched (host, *launches). enable = 1 keeps the
 * normal schedule (the short-range phase on the library's second stream,
 * overlapping the grid chain, so phase times include the contention);
 * enable = 2 runs every phase on the call's stream, one after the other, so
 * each phase's time is its own (same results); 0 turns profiling off.
 * Phases: */
#define MSM_PH_BIN 0        /* binning (counting sort) */
#define MSM_PH_SHORT 1      /* short-range pair sum */
#define MSM_PH_ANTERP 2     /* anterpolation */
#define MSM_PH_RESTRICT 3   /* restrictions, all levels */
#define MSM_PH_STENCIL 4    /* level stencils, all levels */
#define MSM_PH_PROLONG 5    /* prolongations, all levels */
#define MSM_PH_INTERP 6     /* interpolation */
#define MSM_PH_FINAL 7      /* outputs and energy */
#define MSM_PH_VIRIAL 8     /* grid virial (backward) */
#define MSM_PH_BSCALE 9     /* backward outputs */
#define MSM_NPHASE 10
int msm_profile(msm_plan plan, int enable);
int msm_profile_read(msm_plan plan, double* ms, int* launches);

/* Forward pass without a caller-allocated workspace. The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory themselves (a host application whose allocator owns all
 * device memory, a real-time loop that must not allocate). It behaves as
 * msm_forward but keeps its workspace in a fixed device array inside the
 * library, MSM_NOALLOC_SCRATCH_BYTES large, which every GPU that loads the
 * library holds until the process exits. It allocates nothing.
 *  - Plans whose msm_workspace_bytes exceeds MSM_NOALLOC_SCRATCH_BYTES are
 *    rejected with MSM_ERR_CAPACITY (about 250,000 atoms with modest grids fit).
 *  - The first call on a device looks up the array's device address on that
 *    device (cudaGetSymbolAddress); make that first call before any stream
 *    capture.
 *  - All calls share the one array: calls that overlap on the GPU (other
 *    streams, other threads) race and give wrong results; serialise them.
 *  - There is no matching backward pass (msm_backward needs a workspace the
 *    caller owns). Arguments and results are those of msm_forward. */
#define MSM_NOALLOC_SCRATCH_BYTES (32u << 20)
int msm_forward_noalloc(msm_plan plan, int n, const float* pos, const float* q, double* energy, float* phi,
                        float* forces, int flags, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* msm_last_error(void);

/* ---------------------------------------------------------------------------
 * Batches: many independent systems of uneven size and mixed periodicity in
 * one set of launches (one launch per MSM phase for all systems), for the
 * paper's vmap use (Sec. 4.1, batched Madelung evaluation).
 *  per_sys    host, nsys settings (max_atoms ignored).
 *  n_per_sys  host, nsys atom counts (fixed for the batch).
 * Atoms of all systems are packed back to back in system order: positions
 * (sum n) x 3, charges sum n; energy has nsys entries, virial 9 * nsys.
 * A batch applies each system's grid levels of at most 512 points as folded
 * dense stencils (a single-system plan applies them as ball stencils on the
 * prefiltered grid); the two are equal in exact arithmetic, so a system's
 * results in a batch and in its own plan agree to FP32 rounding, not bitwise.
 * ------------------------------------------------------------------------- */
int msm_batch_create(const msm_params* per_sys, const int* n_per_sys, int nsys, msm_batch* out);
int msm_batch_destroy(msm_batch batch);
int msm_batch_workspace_bytes(msm_batch batch, size_t* bytes);
int msm_batch_forward(msm_batch batch, void* workspace, size_t workspace_bytes, const float* pos, const float* q,
                      double* energy, float* phi, float* forces, int flags, void* stream);
int msm_batch_backward(msm_batch batch, void* workspace, const double* grad_energy, float* dE_dpos,
                       float* dE_dq, double* virial, void* stream);
/* msm_field for a batch: field (sum n) x 3, packed like the positions. */
int msm_batch_field(msm_batch batch, void* workspace, float* field, void* stream);
/* msm_force_vjp for a batch: u, dL_dpos (sum n) x 3 and dL_dq (sum n), packed like the positions. */
int msm_batch_force_vjp(msm_batch batch, void* workspace, const float* u, float* dL_dq, float* dL_dpos,
                        void* stream);
/* msm_potential_vjp for a batch: g, dL_dq (sum n) and dL_dpos (sum n) x 3, packed like the positions. */
int msm_batch_potential_vjp(msm_batch batch, void* workspace, const float* g, float* dL_dq, float* dL_dpos,
                            void* stream);
int msm_batch_status(msm_batch batch, void* workspace, void* stream, int* device_status);
/* msm_autotune for a batch (all systems share the tuned shapes), and the shapes in use. */
int msm_batch_autotune(msm_batch batch, void* workspace, size_t workspace_bytes, const float* pos, const float* q,
                       void* stream);
int msm_batch_set_tuning(msm_batch batch, int anterp_tz, int short_block);
int msm_batch_get_tuning(msm_batch batch, int* anterp_tz, int* short_block);

#ifdef __cplusplus
}
#endif

#endif /* MSM_GB300_H */
