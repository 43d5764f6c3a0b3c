/*
 * rte.h -- C ABI of the GB300 (sm_103a) library for ROM-enhanced source iteration with
 * synthetic acceleration (SISA) on the parametric steady radiative transfer equation,
 * after Peng, "Reduced Order Model Enhanced Source Iteration with Synthetic Acceleration for
 * Parametric Radiative Transfer Equation" (arXiv 2402.10488).
 *
 * Problem (paper Sec. 2, Eq. (1)/(2)): one energy group, isotropic scattering, isotropic
 * source G and isotropic inflow g,
 *     v . grad f + sigma_t f = sigma_s rho + G,   rho = normalised angular integral of f.
 * Discretisation: S_N in angle (Sec. 2.1; 1D Gauss-Legendre, 2D Chebyshev-Legendre
 * CL(N_phi, N_vz), weights summing to 1) and upwind DG with Q^1 elements and an orthonormal
 * basis on each cell (Sec. 2.2, Eq. (dg_matrix_vec)).
 *
 * Conventions shared by every call
 *   - Status: every call returns RTE_OK (0) or a negative RTE_E* code; rte_last_error() gives
 *     a message for the calling thread.  No C++ exception crosses this boundary.
 *   - Handles (rte_disc_t, rte_batch_t, rte_rom_t) are owned by the library; destroy them with
 *     the matching *_destroy call.  Arrays passed in are owned by the caller and are only read
 *     (or written) during the call, or -- for calls taking a stream -- until the stream reaches
 *     the work the call enqueued.
 *   - "device" pointers are CUDA global-memory pointers on the handle's device; "host"
 *     pointers are ordinary CPU memory.  Each argument states which it is.
 *   - Streams are passed as void* (a cudaStream_t; NULL = the legacy default stream).
 *   - Layouts: cell index c = j*nx + i (i along x).  A DG vector (rho, G, ...) of one instance
 *     is double[n_cells][P] with P = 2 in 1D (local index a, Legendre degree in x) and P = 4
 *     in 2D (local index k = a + 2b, a the degree in x, b in y).  A batch of B instances stores
 *     B such vectors back to back: double[B][n_dof], n_dof = n_cells*P.
 *   - Orthonormal cell basis: phi_a(x) = sqrt((2a+1)/h) P_a(2(x-x_c)/h), tensorised in 2D.
 *     Coefficient vectors are in this basis (rho's cell average is rho[c][0]/sqrt(|T_c|)).
 *   - FP64 is the interface precision.
 */
#ifndef RTE_GB300_H
#define RTE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTE_OK 0
#define RTE_EINVAL (-1)    /* bad shape, NaN/Inf, sigma_s > sigma_t, negative sigma, bad mode  */
#define RTE_ENOMEM (-2)    /* device allocation failed / admission refused by memory budget     */
#define RTE_ENOCONV (-3)   /* iteration cap reached; results are still written                  */
#define RTE_ETIMEOUT (-4)  /* a bounded device-side wait gave up; the context remains usable    */
#define RTE_ECUDA (-5)     /* a CUDA runtime call failed                                        */
#define RTE_ESTATE (-6)    /* call out of order (e.g. parameters not set, ROM not built)       */

typedef struct rte_disc_s* rte_disc_t;
typedef struct rte_batch_s* rte_batch_t;
typedef struct rte_rom_s* rte_rom_t;

/* ---- library ------------------------------------------------------------------------- */

/* ABI version of this header (major*10000 + minor*100 + patch). */
int rte_version(void);
/* Message of the last failed call on this thread ("" if none).  Pointer valid until the next
 * call on the same thread. */
const char* rte_last_error(void);

/* Library-wide counters: out (HOST int64[1]) = number of kernels this library has launched in
 * this process so far (every launch site increments it). */
int rte_counters(int64_t* out);

/* ---- discretisation -------------------------------------------------------------------- */

/* Mesh, angular rule and material map, shared by every instance of a batch.
 *   dim            1 (slab geometry, Eq. (2)) or 2 (X-Y geometry on S^2)
 *   nx, ny         cells along x and y (ny = 1 when dim == 1); uniform mesh
 *   x0,x1,y0,y1    domain [x0,x1] (x [y0,y1] in 2D)
 *   n_phi, n_vz    1D: n_phi = number of Gauss-Legendre points, n_vz = 0
 *                  2D: the CL(n_phi, n_vz) rule of Sec. 2.1; n_phi must be even (reflection
 *                  symmetry used by the 2D DSA moments)
 *   n_mat          number of materials (a material's cross sections are one value per instance)
 *   mat_id         HOST int32[n_cells], material of each cell, copied during the call      */
typedef struct {
  int dim;
  int nx, ny;
  double x0, x1, y0, y1;
  int n_phi, n_vz;
  int n_mat;
  const int32_t* mat_id;
  const double* dx;   /* 1D only, HOST double[nx] or NULL: cell widths of a non-uniform mesh
                         (positive, summing to x1 - x0); NULL = uniform.  Ignored in 2D.         */
  const int32_t* mat_id_right;
                      /* 1D only, HOST int32[nx] or NULL: the material at each cell's right
                         end.  Cross sections are then linear across cell c, from the values of
                         material mat_id[c] at its left end to those of mat_id_right[c] at its
                         right end (the paper's cross-regime problem, Sec. 4.1.1, has sigma_s
                         linear in x); NULL = mat_id (cellwise constant).  Must be NULL in 2D.
                         Copied during the call.                                                */
} rte_disc_desc;

/* Creates the discretisation on CUDA device `device`: builds the quadrature (Sec. 2.1), the
 * list of distinct sweep directions (in X-Y geometry f_j depends only on (v_x, v_y), so the
 * +-v_z pair of a CL direction is swept once with the pair's summed weight) and uploads the
 * material map.  Errors: RTE_EINVAL for bad sizes, RTE_ECUDA/RTE_ENOMEM. */
int rte_disc_create(const rte_disc_desc* desc, int device, rte_disc_t* out);
int rte_disc_destroy(rte_disc_t disc);

/* info (HOST int64[8]): n_cells, n_dof, P, n_angles, n_dirs (distinct swept directions),
 * n_mat, dim, device. */
int rte_disc_info(rte_disc_t disc, int64_t* info);

/* The S_N rule: v (HOST double[n_angles][3]) and omega (HOST double[n_angles]), in the paper's
 * index order j = (j2-1) N_phi + j1 for CL; 1D: v[j] = (xi_j, 0, 0), ascending xi. */
int rte_disc_quadrature(rte_disc_t disc, double* v, double* omega);

/* ---- batches of parametric instances ------------------------------------------------ */

/* A batch of B instances on one discretisation.  Allocates all per-instance device state
 * (parameters, sweep tables, DSA operators, iteration scratch).  RTE_ENOMEM if it does not
 * fit.  `stream` is used for every later call that takes no stream of its own. */
int rte_batch_create(rte_disc_t disc, int B, rte_batch_t* out);
int rte_batch_destroy(rte_batch_t batch);

/* Sets the parameters mu of every instance (Sec. 3.1: cross sections, source, inflow) and
 * runs the per-instance set-up kernels (sweep cell tables, source moments, DSA operator):
 *   sigma_t, sigma_s  HOST double[B][n_mat]; 0 <= sigma_s <= sigma_t, sigma_t > 0
 *   source            HOST double[B][n_cells], cellwise-constant isotropic G
 *   inflow            HOST double[B][2*dim], isotropic inflow g on the sides (x-, x+[, y-, y+])
 * Errors: RTE_EINVAL (NaN/Inf, negative values, sigma_s > sigma_t), RTE_ECUDA.
 * Synchronous with respect to the host (returns after the set-up has run). */
int rte_batch_set_params(rte_batch_t batch, const double* sigma_t, const double* sigma_s,
                         const double* source, const double* inflow);

/* The same as rte_batch_set_params with the parameters already in DEVICE memory of the batch's
 * device (for example tensors resident in HBM), in the same layouts:
 *   sigma_t, sigma_s  DEVICE double[B][n_mat];  source DEVICE double[B][n_cells];
 *   inflow            DEVICE double[B][2*dim]
 * Asynchronous on `stream`: a kernel copies the tables, forms the source moments and checks every
 * value (finite, sigma_t > 0, 0 <= sigma_s <= sigma_t) on the device, then the per-instance
 * set-up kernels run; the call returns without waiting.  The check's outcome is read by the host
 * in the next call that uses the parameters (rte_sweep, rte_solve, rte_pgmres, rte_dsa_correction,
 * ...): that call waits for the set-up and returns RTE_EINVAL, leaving the batch without
 * parameters, if a value was invalid.  Invalid values cause no fault (they only enter
 * arithmetic).  The caller keeps the arrays unchanged until the stream has passed the call;
 * work on other streams must be ordered after it by the caller.  Errors (immediate): RTE_EINVAL
 * for null arguments, RTE_ECUDA. */
int rte_batch_set_params_device(rte_batch_t batch, const double* sigma_t, const double* sigma_s,
                                const double* source, const double* inflow, void* stream);

/* Sets the parameters of some instances (slots) only, leaving the others untouched -- the
 * admission step of continuous batching.  Same meaning as rte_batch_set_params for n instances:
 *   slots             HOST int[n], distinct, each in [0, B)
 *   sigma_t, sigma_s  HOST double[n][n_mat]
 *   source            HOST double[n][n_cells]
 *   inflow            HOST double[n][2*dim]
 * The host arrays may be reused when the call returns (they are staged in pinned memory).  The
 * uploads and the per-slot set-up kernels are asynchronous on `stream`; a later call on the same
 * batch waits until the previous call's staging has been consumed.  The batch counts as having
 * parameters once every slot has been set (by this call or rte_batch_set_params).
 * Errors: as rte_batch_set_params. */
int rte_batch_set_slots(rte_batch_t batch, int n, const int* slots, const double* sigma_t,
                        const double* sigma_s, const double* source, const double* inflow,
                        void* stream);

/* Red-black block Gauss-Seidel sweeps per level before and after the coarse correction in the
 * 2D DSA multigrid (default 2; 1..8).  Changes only the convergence rate of the DSA solve (the
 * fixed point of Alg. 1 does not depend on the DSA).  Errors: RTE_EINVAL. */
int rte_batch_dsa_smoothing(rte_batch_t batch, int nu);

/* Form of the red-black block Gauss-Seidel smoother of the 2D DSA multigrid -- the solver of the
 * consistent DSA system (App. B, carried to X-Y geometry) -- on the levels that run one launch per
 * step (levels of at most 32 x 32 cells run inside one fused kernel per instance).  Changes only
 * how the same sweeps are scheduled: all three compute the same values bit for bit:
 *   RTE_SMOOTHER_GLOBAL   one launch per half sweep, each cell reading its neighbours from global
 *                         memory
 *   RTE_SMOOTHER_TILED    one launch per half sweep on 16 x 16 tiles: the other colour's cells of a
 *                         tile and a one-cell halo are loaded into shared memory once
 *   RTE_SMOOTHER_BLOCKED  the nu sweeps in one launch on 16 x 16 tiles with a halo of 2 nu cells
 *                         in shared memory (temporal blocking, nu <= 4): x and b read once, but
 *                         1.4x the cell updates (the shrinking halo)
 * Default: the measured fastest on GB300 (see the library's design notes).  Errors: RTE_EINVAL. */
#define RTE_SMOOTHER_GLOBAL 0
#define RTE_SMOOTHER_TILED 1
#define RTE_SMOOTHER_BLOCKED 2
int rte_batch_dsa_smoother(rte_batch_t batch, int kind);

/* info (HOST int64[6]): B, device bytes held by the batch, directions per warp (preferred),
 * the smallest directions per warp its sweep partial sums are sized for, 1 if the
 * decomposition is picked per launch, 1 if every slot has parameters.  The device bytes of a
 * one-instance batch bound the memory one more slot costs (used for admission by memory). */
int rte_batch_info(rte_batch_t batch, int64_t* info);

/* ---- hot path: one source iteration --------------------------------------------------- */

/* Transport sweep fused with the scalar-flux reduction (Alg. 1; Eq. (transport_sweep)):
 *     f_j = (D_j + Sigma_t)^{-1} (Sigma_s rho_in + [G + g^bc_j]),   rho_out = sum_j omega_j f_j
 * for every instance of the batch.  with_source = 0 drops G and g^bc (rho_out = L rho_in,
 * Eq. (rho_matrix_vec_def)).  f_j itself is not stored unless psi_out != NULL.
 *   rho_in   DEVICE double[B][n_dof]
 *   rho_out  DEVICE double[B][n_dof] (must not alias rho_in)
 *   psi_out  DEVICE double[B][n_dirs][n_dof] or NULL: f of each distinct swept direction, in
 *            the order of rte_batch_directions()
 *   active   DEVICE uint8[B] or NULL: instances with active[b] == 0 are skipped (outputs
 *            untouched)
 * Asynchronous on `stream`.  Errors: RTE_ESTATE (no parameters), RTE_EINVAL, RTE_ECUDA. */
int rte_sweep(rte_batch_t batch, const double* rho_in, double* rho_out, double* psi_out,
              int with_source, const uint8_t* active, void* stream);

/* One FP32 sweep (the precision variant's sweep, rte_solve_opts.fp32_switch): the operator of
 * rte_sweep with source, evaluated with FP32 sweep tables, FP32 cell sources Sigma_s rho_in + G, FP32
 * cell solves and FP32 per-group partial sums, which are added in FP32 and returned in FP64:
 *     rho_out ~ sum_j omega_j (D_j + Sigma_t)^{-1} (Sigma_s rho_in + G + g^bc_j)
 * to FP32 rounding (a few 1e-7 relative per cell solve, carried along the sweep).
 *   rho_in, rho_out  DEVICE double[B][n_dof], not aliased
 *   active           DEVICE uint8[B] or NULL (instances with active[b] == 0 are skipped)
 * 2D only.  Asynchronous on `stream`.  Errors: RTE_ESTATE, RTE_EINVAL, RTE_ECUDA. */
int rte_sweep_f32(rte_batch_t batch, const double* rho_in, double* rho_out, const uint8_t* active,
                  void* stream);

/* One float-float sweep (the precision variant's outer sweep, rte_solve_opts.outer_ff; no
 * counterpart in the paper, which computes in FP64): the operator of rte_sweep with source, each
 * cell solve in float-float arithmetic -- every value an unevaluated sum of two FP32 numbers,
 * about 48 significant bits, from Knuth's TwoSum and Dekker's exact product in FMA form -- on the
 * FP32 units, with cell sources formed in FP64 and the per-group partial sums reduced in FP64:
 *     rho_out = sum_j omega_j (D_j + Sigma_t)^{-1} (Sigma_s rho_in + G + g^bc_j)
 * to within 3e-11 of ||rho_out||_inf (the tested bound: the FP64 sweep's 1e-12 scaled by the ratio
 * 32 of the two unit roundoffs; one float-float FMA rounds to ~1e-14 relative).
 *   rho_in, rho_out  DEVICE double[B][n_dof], 16-byte aligned, not aliased
 *   active           DEVICE uint8[B] or NULL (instances with active[b] == 0 are skipped)
 * 2D only; 1, 2 or 4 directions per warp (the sweep's choice, 8 narrowed to 4; where the batch's
 * partial-sum buffer holds only the groups of 8, the FP64 sweep runs instead).  Asynchronous on
 * `stream`.  Errors: RTE_ESTATE, RTE_EINVAL, RTE_ENOMEM, RTE_ECUDA. */
int rte_sweep_ff(rte_batch_t batch, const double* rho_in, double* rho_out, const uint8_t* active,
                 void* stream);

/* Work decomposition of the 2D sweep: dirs_per_warp in {1, 2, 4, 8} sets how many directions of
 * one quadrant a warp sweeps together (more directions: more instruction-level parallelism and
 * fewer partial sums; fewer: more warps in flight).  0 (the default) picks per launch the largest
 * value that still gives at least four resident warps per SM for the number of running
 * instances, but never fewer directions per warp than keep one instance's partial sums within
 * 64 MB (large meshes with many directions).  Set before sweeping.  Errors: RTE_EINVAL. */
int rte_batch_tune(rte_batch_t batch, int dirs_per_warp);

/* Empirical autotuner of the same choice: for B, B/2, B/4, ..., 1 running instances it times one
 * sweep with every allowed directions-per-warp value (CUDA events on `stream`, on the batch's
 * current parameters) and keeps the fastest per count; for the FP64 sweep every value is also
 * timed with 2, 4 and 8 warps per direction group (the pipelined form, row blocks shared
 * round-robin, as far as the mesh has row blocks of 32 rows).  Later sweeps pick the entry for the
 * smallest timed count >= their running instances.  2D batches get a second table, measured the
 * same way with the FP32 sweep of the precision variant (kept internally).  Uses the batch's
 * iteration scratch only.
 *   n_entries  HOST int out (may be NULL); table HOST int[2*32] or NULL: (count, dirs_per_warp)
 * Synchronous.  rte_batch_tune resets it.  1D batches: no-op.  Errors: RTE_ESTATE (no
 * parameters), RTE_ECUDA. */
int rte_batch_autotune(rte_batch_t batch, void* stream, int* n_entries, int* table);

/* The FP64 sweep decomposition rte_batch_autotune chose, per timed count of running instances:
 *   n_entries  HOST int out: 0 when the batch is not autotuned
 *   table      HOST int[3*32] or NULL: (count, dirs_per_warp, warps per direction group)
 * Errors: RTE_EINVAL (null batch). */
int rte_batch_tuned(rte_batch_t batch, int* n_entries, int* table);

/* Allocation-free variant of rte_sweep (the paper has no counterpart: this is a library service).
 * For callers that cannot allocate device memory while they run (for example under a host
 * framework whose caching allocator has reserved the device's memory, or inside a latency-bound
 * service loop where an allocation, which may synchronise the device, is not allowed).  Computes
 * the same sweep and scalar-flux reduction as rte_sweep for every instance (no active mask, no psi
 * output), equal to rounding: it always uses the batch's preferred directions per warp and one
 * warp per direction group, while rte_sweep may group directions per launch, so the partial sums
 * can be added in another order (1e-12 relative).  It keeps the partial scalar-flux sums in one
 * fixed 16 MiB device array that belongs to the library image instead of memory owned by the
 * batch.  The array is taken on a device when the first batch is created there
 * (rte_batch_create loads it and looks up its address); the call itself allocates nothing and
 * looks the address up again each time.
 *   rho_in, rho_out  DEVICE double[B][n_dof], 16-byte aligned, not aliased
 * Limit: B * (number of sweep work groups) * n_dof <= 2^21 doubles, else RTE_EINVAL (e.g. at most
 * 4 instances of a 128x128 CL(16,4) batch swept with 4 directions per warp, see
 * rte_batch_tune; any 1D slab batch of moderate size).
 * Every GPU that loads the library's device code holds the 16 MiB array until the process exits.
 * All calls share the one array: calls that overlap on the GPU (on different streams, or from
 * different threads) race and give wrong results; serialise them.
 * Asynchronous on `stream`.  Errors: RTE_EINVAL, RTE_ESTATE, RTE_ECUDA. */
int rte_sweep_static(rte_batch_t batch, const double* rho_in, double* rho_out, int with_source,
                     void* stream);

/* Residual and particle balance of a solution, in FP64 (one extra sweep; no counterpart call in
 * the paper, which reports the residual R^rho_inf = ||(I - L) rho - b-bar||_inf of Eq.
 * (rho_matrix_vec) averaged over its test sets, the notation table of Sec. 4).  For every instance
 * b (in `active`, or all when NULL) one FP64 sweep rho* = L rho + b-bar of rho gives
 *   out[b][0] = ||rho - rho*||_inf                          (R^rho_inf of this instance)
 *   out[b][1] = max_T |bal_T|, bal_T = net outflow_T + int_T sigma_t rho* - int_T sigma_s rho
 *               - int_T G: the particle balance of the sweep in cell T (the DG equation tested
 *               with T's indicator function), the net outflow summed over directions with their
 *               weights from the upwind face traces the sweep passes between cells; it vanishes
 *               for an exact sweep whatever rho is
 *   out[b][2] = leakage + int sigma_a rho* - int G over the domain (absorption + net leakage =
 *               source), which tends to 0 as rho converges: it equals sum_T bal_T minus
 *               int sigma_s (rho* - rho)
 *   out[b][3] = int G over the domain
 *   rho           DEVICE double[B][n_dof], 16-byte aligned
 *   out           DEVICE double[B][4]
 *   cell_balance  DEVICE double[B][n_cells] or NULL: bal_T per cell
 *   active        DEVICE uint8[B] or NULL
 * Uses the batch's iteration scratch (not to overlap rte_solve on the same batch) and, from the
 * first call, B x (directions / 8 in 2D, directions in 1D) x n_cells doubles the batch keeps for
 * the face outflows.  Asynchronous on `stream`.  Errors: RTE_ESTATE, RTE_EINVAL, RTE_ENOMEM,
 * RTE_ECUDA. */
int rte_residual(rte_batch_t batch, const double* rho, double* out, double* cell_balance,
                 const uint8_t* active, void* stream);

/* Sweep-kernel timing for throughput and roofline accounting.  Each 2D/1D sweep kernel launched
 * for this batch while timing is on is bracketed by CUDA events recorded on the stream it is
 * launched on, and so is each DSA correction, each ROM step (ROMSA correction, ROMIG, reduced
 * operator assembly), each per-instance set-up and each FP32 or float-float sweep (sources, sweep,
 * no reduction).  out (HOST double[15], may be NULL) receives (FP64 sweep-kernel ms, timed FP64
 * sweep launches, cell x distinct-direction local solves they performed, DSA ms, DSA calls, ROM
 * ms, ROM calls, set-up ms, set-up calls, FP32 sweep ms, FP32 sweep calls, their cell x direction
 * solves, float-float sweep ms, float-float sweep calls, their cell x direction solves); the
 * call waits for the recorded events.  enable = 1 resets and starts, 0 resets and stops, -1 only
 * reads.  Errors: RTE_EINVAL, RTE_ECUDA. */
int rte_batch_timing(rte_batch_t batch, int enable, double* out);

/* Measured FMA throughput of the device's arithmetic pipes, for roofline accounting (a library
 * service; the paper has no counterpart): kind 0 = FP64 DFMA (the 2D FP64 sweep's bound), 1 = FP32
 * FFMA (the FP32 sweep's).  Independent FMA chains in 4 blocks of 256 threads per SM; best of five
 * launches of a few milliseconds, timed with CUDA events on `stream` after two untimed ones.
 * tflops: HOST double out (2 FLOP per FMA).  Synchronous.  Errors: RTE_EINVAL, RTE_ECUDA. */
int rte_fma_peak(int device, int kind, double* tflops, void* stream);

/* The distinct swept directions: dirs (HOST double[n_dirs][4]) = (v_x, v_y, summed weight,
 * multiplicity), in the order used by psi_out and the ROM bases. */
int rte_batch_directions(rte_batch_t batch, double* dirs);

/* Stop-test norms (Alg. 1): norms[b] = (||rho_star_b - rho_prev_b||_inf, ||rho_star_b||_inf)
 * over the coefficient vectors.  norms: DEVICE double[B][2].  Asynchronous. */
int rte_change_norm(rte_batch_t batch, const double* rho_star, const double* rho_prev,
                    double* norms, void* stream);

/* Consistent DSA correction (App. B; 2D by the same P1-ansatz moment derivation):
 * solves the diffusion system for delta rho given R = Sigma_s (rho^(l,*) - rho^(l-1)).
 *   R      DEVICE double[B][n_dof];  drho  DEVICE double[B][n_dof]
 *   rtol   2D: > 0 -- flexible GMRES on the FP64 system, preconditioned by one FP32 multigrid
 *          V-cycle per iteration, to this relative residual; == 0 -- exactly max_it FP32
 *          multigrid V-cycles x <- x + V(b - A x) with no host round trip (an approximate DSA:
 *          the SI fixed point does not depend on it).  1D is always a direct solve.
 *   max_it iteration cap (rtol > 0) or number of V-cycles (rtol == 0); iters (HOST int[B], may
 *          be NULL) receives iterations used
 *   active DEVICE uint8[B] or NULL
 * Synchronises `stream` (the 2D Krylov solve reads residual norms on the host).
 * Errors: RTE_ENOCONV if max_it was reached for some instance (drho still written). */
int rte_dsa_correction(rte_batch_t batch, const double* R, double* drho, double rtol,
                       int max_it, const uint8_t* active, int* iters, void* stream);

/* Forms R = Sigma_s (rho_star - rho_prev) (the source of the kinetic correction equation,
 * Eq. (discrete_correction)).  All DEVICE double[B][n_dof].  Asynchronous. */
int rte_correction_source(rte_batch_t batch, const double* rho_star, const double* rho_prev,
                          double* R, void* stream);

/* ---- reduced order models (Sec. 3) ------------------------------------------------------ */

typedef struct {
  double eps_train;   /* SISA tolerance of the training solves (absolute, Alg. 1)           */
  int window;         /* window size w for correction snapshots (Sec. 3.2.1)                 */
  int rank_p;         /* POD rank of the parametric ROM (0: use eps_pod)                     */
  int rank_c;         /* POD rank of the correction ROM (0: use eps_pod)                     */
  double eps_pod;     /* truncation tolerance of Eq. (pod_truncation) when a rank is 0       */
  int max_iter;       /* iteration cap of the training solves                                */
  double dsa_rtol;    /* DSA solve tolerance used in the training solves                     */
  int correction_start; /* 0: correction snapshots from training runs started at zero;
                           1: from runs started at the ROMIG guess of the parametric ROM, for
                           ROMIG followed by ROMSAD (remark after Alg. 2)                       */
} rte_rom_opts;

/* Offline stage (Sec. 3.1.1, 3.2.1) on the GPU: SI-DSA solves of every training instance of
 * `train` (f stored), snapshot matrices F and delta F (window w), thin SVD by a Gram-Schmidt QR
 * on the device (applied twice per column) and a one-sided Jacobi SVD of the small factor R,
 * truncation,
 * U^rho, U^iso and the affine reduced operators A_{k,r} = U^T A_k U.  Produces the parametric ROM (rom_p, for ROMIG) and
 * the correction ROM (rom_c, for ROMSA).  Either output pointer may be NULL.  Synchronous. */
int rte_rom_build(rte_batch_t train, const rte_rom_opts* opts, rte_rom_t* rom_p,
                  rte_rom_t* rom_c, void* stream);
int rte_rom_destroy(rte_rom_t rom);

/* info (HOST double[6]): r, n_snapshots, eps_pod of the kept rank (1 - sum_{k<=r} s_k /
 * sum s_k), n_dirs, n_dof, sum of singular values.  sv (HOST double[n_snapshots] or NULL):
 * singular values of the snapshot matrix. */
int rte_rom_info(rte_rom_t rom, double* info, double* sv);

/* Writes the online part of a ROM (U^rho, U^iso, the reduced operators, singular values and the
 * discretisation it was built on) to a file, and reads it back for a discretisation with the
 * same mesh, domain, quadrature and material map.  The full basis U is not stored (the online
 * stage never reads it).  Errors: RTE_EINVAL (path, mismatching discretisation, bad file),
 * RTE_ENOMEM, RTE_ECUDA. */
int rte_rom_save(rte_rom_t rom, const char* path);
int rte_rom_load(rte_disc_t disc, const char* path, rte_rom_t* rom);

/* ROMIG (Sec. 3.1.1): rho0 = U^rho c with (sum_k psi_k(mu) A_{k,r}) c = U^T b_mu, for every
 * instance of `batch` (same discretisation as the ROM).  rho0: DEVICE double[B][n_dof]. */
int rte_rom_initial_guess(rte_rom_t rom_p, rte_batch_t batch, double* rho0,
                          const uint8_t* active, void* stream);

/* ROMSA correction (Eq. (rom_correction)): delta rho = dU^rho dc with
 * (dU^T A_mu dU) dc = (dU^iso)^T R.  R, drho: DEVICE double[B][n_dof]. */
int rte_romsa_correction(rte_rom_t rom_c, rte_batch_t batch, const double* R, double* drho,
                         const uint8_t* active, void* stream);

/* Dense POD projections on the tensor cores: the products behind ROMSA's and ROMIG's project and
 * lift steps (Eq. (rom_correction); Sec. 3.1.2) for a basis of r <= 32 vectors of length n,
 *   rte_pod_project_bf16:  out[b][i] = sum_e U[i][e] X[b][e]     (i < r, e < n, b < B)
 *   rte_pod_lift_bf16:     Y[b][e]   = sum_i U[i][e] C[b][i]
 * with U, X, C rounded to BF16 and products summed in FP32 (tcgen05.mma, accumulators in tensor
 * memory); the projection sums its K chunks in FP64 in a fixed order, so results are
 * deterministic.  Exact when the operands are BF16 values whose partial sums stay exact in FP32.
 *   U    DEVICE double[r][n];  X DEVICE double[B][n];  C DEVICE double[B][r]
 *   out  DEVICE double[B][r];  Y DEVICE double[B][n] (rows of inactive instances untouched)
 *   active  DEVICE uint8[B] or NULL (instances with active[b] == 0 are skipped)
 *   work DEVICE, 16-byte aligned, rte_pod_workspace_bytes(r, n, B) bytes (the lift uses its first
 *        word only).  work's first int32 is a status word: a device-side wait that gave up sets it
 *        to 1 (the result is then invalid); the caller zeroes it before the first call.
 * Asynchronous on `stream`; calls sharing `work` must not overlap.  Errors: RTE_EINVAL (r > 32,
 * bad sizes, null or misaligned pointers), RTE_ECUDA. */
int rte_pod_workspace_bytes(int r, int n, int B, int64_t* bytes);
int rte_pod_project_bf16(const double* U, int r, int n, const double* X, int B,
                         const uint8_t* active, double* out, void* work, void* stream);
int rte_pod_lift_bf16(const double* U, int r, int n, const double* C, int B, const uint8_t* active,
                      double* Y, void* work, void* stream);

/* Fault injection for tests of the failure path (no counterpart in the paper).  The device-side
 * waits of the library (the tensor-core products' mbarrier waits) give up after about one second
 * and set the caller's status word instead of hanging.  RTE_FAULT_LIFT_NO_MMA makes the next
 * rte_pod_lift_bf16 launch (directly or inside a ROMSA correction with rom_bf16) issue no MMA, so
 * its wait runs out: its status word becomes 1, its output is invalid, nothing is left in flight
 * and the context stays usable.  One-shot; 0 clears.  Errors: RTE_EINVAL. */
#define RTE_FAULT_LIFT_NO_MMA 1
int rte_fault_inject(int what);

/* ---- full solves (Alg. 1 with the SA of choice, Alg. 2) --------------------------------- */

#define RTE_SA_NONE 0
#define RTE_SA_DSA 1
#define RTE_SA_ROMSA 2
#define RTE_SA_ROMSAD 3

typedef struct {
  double eps;          /* stop tolerance eps_SISA                                           */
  int rel;             /* 0: ||rho* - rho||_inf < eps (Alg. 1); 1: divided by ||rho*||_inf   */
  int max_iter;        /* N_iter                                                             */
  int sa;              /* RTE_SA_*                                                           */
  int theta;           /* ROMSAD: ROMSA allowed after iterations 1..theta (Alg. 2)           */
  double eps_romsad;   /* ROMSAD threshold on the absolute change (Eq. (romsad_parameters)) */
  double dsa_rtol;     /* 2D DSA: Krylov tolerance (> 0) or 0 for dsa_max_it V-cycles          */
  int dsa_max_it;      /* 2D DSA: iteration cap, or the number of V-cycles when dsa_rtol == 0  */
  const uint8_t* schedule; /* HOST uint8[max_iter] or NULL: forces ROMSAD's choice per
                              iteration (1 = ROMSA, 0 = DSA), for reproducibility tests      */
  double fp32_switch;  /* precision variant (2D): 0 -- every sweep in FP64; > 0 -- an instance
                          sweeps in FP32 until its stop-test quantity falls below fp32_switch,
                          then in FP64 until the stop test fires, so the FP64 sweeps supply the
                          final digits (the fixed point is the FP64 one)                      */
  double refine_kappa; /* FP64 outer residual correction (2D): 0 -- off; > 0 -- an FP64 sweep
                          of the iterate x0 that does not stop the instance gives y0 = L x0 + b
                          and the residual r = y0 - x0 (Eq. (rho_matrix_vec): (I - L) e = r for
                          the error e of x0).  The following sweeps iterate e alone in FP32
                          (rho^(l,*) = y0 + L (rho^(l-1) - x0), so FP32 rounding only touches the
                          small e; the corrections are Alg. 1's), until the change falls below
                          refine_kappa x the FP64 change or refine_inner FP32 sweeps are done;
                          then the next sweep is FP64 again.  Only FP64 sweeps (float-float
                          ones with outer_ff) take the stop test.  Combines with fp32_switch
                          (its FP32 phase comes first).                                       */
  int refine_inner;    /* cap on the FP32 sweeps per outer step (>= 1 when refine_kappa > 0) */
  int rom_bf16;        /* 1: ROMSA's project and lift products (Eq. (rom_correction)) in BF16
                          on the tensor cores with FP32 accumulation (rte_pod_project_bf16,
                          rte_pod_lift_bf16); the r x r solve stays FP64.  The correction is
                          then accurate to ~1e-3 relative, which changes how fast the iteration
                          converges, never its FP64 fixed point.  0: FP64.                    */
  int gang_wait;       /* precision variant: 0 -- every instance sweeps at every iteration;
                          > 0 -- an instance due for an FP64 sweep while other running instances
                          still sweep in FP32 waits (no sweep, no correction) for up to gang_wait
                          iterations, so that FP64 sweeps run in fewer, fuller launches.  Its
                          own sequence of iterates is unchanged; only when it runs changes.   */
  int verify;          /* 1: after the solve, one more FP64 sweep of each result gives its
                          residual R^rho_inf and particle balance (rte_residual) in the report;
                          the result must be in device memory.  0: not computed (zeros).      */
  uint8_t* sa_history; /* HOST uint8[B][max_iter] or NULL, written: per sweep l of an instance,
                          the correction that followed it -- RTE_SA_NONE (none: plain SI, or the
                          stop test fired), RTE_SA_DSA or RTE_SA_ROMSA (Alg. 2's choice) --
                          plus 0x10 when sweep l ran in FP32.  Entries past n_sweep untouched. */
  int outer_ff;        /* precision variant (fp32_switch or refine_kappa > 0): 1 -- its sweeps
                          that would run in FP64 run as float-float sweeps (rte_sweep_ff) on the
                          FP32 units, so eps must stay above their rounding (a relative change
                          of 1e-11 is tested to converge to the FP64 solution); 0 -- FP64.    */
} rte_solve_opts;

typedef struct {
  int n_sweep;         /* sweeps performed                                                  */
  int converged;       /* 1 if the stop test fired                                          */
  int n_romsa;         /* corrections done by ROMSA                                         */
  int n_dsa;           /* corrections done by DSA                                           */
  int dsa_iters;       /* total DSA Krylov iterations                                       */
  double last_change;  /* last ||rho* - rho||_inf                                           */
  double rho_inf;      /* ||rho*||_inf at exit                                              */
  int n_sweep32;       /* of the n_sweep sweeps, those done in FP32                          */
  int pad;
  /* with rte_solve_opts.verify (else 0), from one FP64 sweep rho* of the result rho:          */
  double r_inf;        /* ||(I - L) rho - b-bar||_inf = ||rho - rho*||_inf (R^rho_inf, Sec. 4) */
  double balance_cell; /* max over cells of |net outflow + int sigma_t rho* - int sigma_s rho
                          - int G| (zero for an exact sweep; see rte_residual)               */
  double balance;      /* leakage + int sigma_a rho* - int G (absorption + net leakage =
                          source; -> 0 as rho converges)                                      */
} rte_solve_report;

/* Runs Alg. 1 on every instance of the batch, each stopping on its own test.
 *   rho      DEVICE double[B][n_dof]: in = initial guess rho^(0), out = solution (rho^(l,*) of
 *            the sweep at which the test fired; the last corrected iterate otherwise)
 *   rom_c    correction ROM for RTE_SA_ROMSA / RTE_SA_ROMSAD (NULL otherwise)
 *   reports  HOST rte_solve_report[B] (may be NULL)
 *   history  HOST double[B][max_iter] or NULL: ||rho^(l,*) - rho^(l-1)||_inf per iteration
 * Synchronous.  Returns RTE_ENOCONV if some instance hit max_iter. */
int rte_solve(rte_batch_t batch, const rte_solve_opts* opts, rte_rom_t rom_c, double* rho,
              rte_solve_report* reports, double* history, void* stream);

/* ---- the paper's comparison system: DSA-preconditioned GMRES (Sec. 2.3, App. A) ---------- */

typedef struct {
  double rtol;      /* stop when ||M^{-1}(b-bar - (I - L) x)|| <= rtol ||M^{-1} b-bar||            */
  int restart;      /* m: Arnoldi steps per cycle (the paper uses 25); 1..200                       */
  int max_iter;     /* cap on the total Arnoldi steps per instance                                 */
  int precond;      /* 1: left preconditioner M^{-1} = I + C Sigma_s (C: the DSA correction of
                       Alg. 1, i.e. one SI-DSA step is a Richardson step); 0: none                */
  double dsa_rtol;  /* 2D DSA inside M^{-1}, as in rte_solve_opts                                 */
  int dsa_max_it;
  int zero_start;   /* 1: start from x = 0 (rho is output only); 0: rho holds the start (one
                       extra sweep for its residual), e.g. a ROMIG guess                           */
} rte_gmres_opts;

/* Restarted GMRES on (I - L) rho = b-bar for every instance of the batch (Eq. (rho_matrix_vec)),
 * applying I - L by a transport sweep without source and b-bar by one sweep from rho = 0.
 *   rho      DEVICE double[B][n_dof]: start (unless zero_start) and solution
 *   reports  HOST rte_solve_report[B] or NULL: n_sweep (one for b-bar, one per Arnoldi step, one
 *            per residual of a nonzero iterate -- the paper's count), converged, n_dsa = applications
 *            of M^{-1}, dsa_iters, last_change = the final relative preconditioned residual
 * Synchronous.  RTE_ENOCONV if an instance reached max_iter. */
int rte_pgmres(rte_batch_t batch, const rte_gmres_opts* opts, double* rho,
               rte_solve_report* reports, void* stream);

/* rte_solve on n batches at once (typically one per discretisation of a mixed-size workload),
 * each on its own stream: one host thread keeps every batch's iteration going, relaunching a
 * batch as soon as its stop-test norms are back, so the batches' kernels overlap on the device.
 * Arrays of length n: batches (distinct), opts, roms (array or NULL; a ROM may serve one batch
 * only), rho (DEVICE double[B_k][n_dof_k] each, in/out as in rte_solve), reports (HOST arrays of
 * rte_solve_report[B_k], the array or an entry may be NULL), streams (array or NULL).
 * Synchronous.  Returns RTE_ENOCONV if some instance hit its iteration cap. */
int rte_solve_many(int n, const rte_batch_t* batches, const rte_solve_opts* opts,
                   const rte_rom_t* roms, double* const* rho, rte_solve_report* const* reports,
                   void* const* streams);

/* rte_solve_many with the batches iterating in lockstep, for mixed-size workloads: at every iteration
 * ONE sweep launch covers the running instances of all batches -- a persistent grid of warps taking
 * (batch, instance, direction group) work items from a shared counter, longest sweeps first -- so
 * that instances of every mesh and quadrature size fill the GPU together and the launch's tail is
 * short; then each batch's stop test and corrections (Alg. 1 / Alg. 2) run on its own stream, and
 * the next sweep waits for them all.  Every batch sweeps 4 directions per warp (8 where its partial
 * sums need wider groups); with the same decomposition (rte_batch_tune) the results equal
 * rte_solve_many's bit for bit.  The sweeps run on the first batch's stream.  Arguments as in
 * rte_solve_many; 2D batches and FP64 sweeps only (no fp32_switch / refine_kappa).  Synchronous.
 * Errors: RTE_EINVAL, RTE_ENOCONV (some instance hit its cap), RTE_ECUDA. */
int rte_solve_lockstep(int n, const rte_batch_t* batches, const rte_solve_opts* opts,
                       const rte_rom_t* roms, double* const* rho, rte_solve_report* const* reports,
                       void* const* streams);

/* rte_solve_many with the SWEEPS of all batches on one internal stream of the highest priority, one
 * after another in the order the batches' stop tests come back, and each batch's stop test and
 * corrections (Alg. 1 / Alg. 2: DSA V-cycles, ROM products) on its own stream: while one batch
 * sweeps, the corrections of the others run beside it.  The FP64 sweep is bound by the FP64 pipe and
 * leaves the FP32 pipe and the memory system mostly idle, so splitting one batch of instances into
 * sub-batches (separate rte_batch_t of one discretisation, each with its own ROM handle, e.g. from
 * rte_rom_save / rte_rom_load) and solving them this way hides most of the correction time.  A
 * batch's corrections are issued only after the sweep queued behind its own has been dispatched
 * (sweeps placed on a GPU busy with other kernels crowd onto some SM sub-partitions and run up to
 * 3x slower).  Every batch runs exactly the iterations it runs under rte_solve_many; the results
 * equal rte_solve_many's bit for bit.  Arguments and errors as in rte_solve_many; streams: n
 * distinct streams for the corrections (NULL: the legacy default stream, which serialises them
 * with everything else and gives no overlap).  Synchronous. */
int rte_solve_interleaved(int n, const rte_batch_t* batches, const rte_solve_opts* opts,
                          const rte_rom_t* roms, double* const* rho, rte_solve_report* const* reports,
                          void* const* streams);

/* ---- serving: continuous batching of parametric solves ---------------------------------- */

typedef struct rte_server_s* rte_server_t;

typedef struct {
  rte_solve_report solve;  /* iteration report of the request's solve                         */
  int status;              /* RTE_OK, RTE_ENOCONV, or the error that ended the request         */
  int bucket, slot;        /* where it ran                                                    */
  int pad;
  double t_submit, t_admit, t_done;  /* seconds since rte_server_start (steady clock); t_done
                                        is when the result was in host memory                 */
} rte_serve_report;

/* A server drives buckets -- one per discretisation -- from one worker thread, each bucket on its
 * own stream.  A bucket's batch supplies its slots (B = the most requests of that bucket on the
 * device at once; size it by device memory with rte_batch_info).  Requests queue per bucket; at
 * every iteration boundary of a bucket its finished slots are returned and queued requests are
 * admitted into free slots, so new requests join the running ones without waiting for them.
 * Every slot runs Alg. 1 with the bucket's options (ROMSAD of Alg. 2 with rom_c, etc.) and the
 * request's own tolerance; rom_p (or NULL for a zero initial iterate) gives the ROMIG guess.
 * Handles passed to a bucket must outlive the server and not be used elsewhere meanwhile. */
int rte_server_create(int device, rte_server_t* out);
/* opts.schedule and opts.sa_history must be NULL and opts.verify 0; opts.eps is replaced by each
 * request's tolerance. */
int rte_server_add_bucket(rte_server_t server, rte_batch_t slots, rte_rom_t rom_p,
                          rte_rom_t rom_c, const rte_solve_opts* opts, int* bucket);
int rte_server_start(rte_server_t server);
/* Queues one request (parameters as one instance of rte_batch_set_slots; host arrays copied
 * before the call returns).  ticket: HOST uint64 out.  Thread-safe. */
int rte_server_submit(rte_server_t server, int bucket, const double* sigma_t,
                      const double* sigma_s, const double* source, const double* inflow,
                      double eps, uint64_t* ticket);
/* Waits up to timeout_s seconds for a request; on completion copies the solution (HOST
 * double[n_dof], may be NULL) and the report, and releases the ticket.  RTE_ETIMEOUT if it has
 * not finished (the ticket stays valid).  Thread-safe. */
int rte_server_wait(rte_server_t server, uint64_t ticket, double timeout_s, double* rho,
                    rte_serve_report* report);
/* stats (HOST double[8]): sweep launches, admitted, completed, queued now, largest queue,
 * largest number of running slots of one bucket, worker seconds with work in flight, seconds
 * since start. */
int rte_server_stats(rte_server_t server, double* stats);
/* Drops queued requests, lets running ones finish, stops the worker and frees the server (not
 * the batches or ROMs given to it). */
int rte_server_destroy(rte_server_t server);

#ifdef __cplusplus
}
#endif
#endif /* RTE_GB300_H */
