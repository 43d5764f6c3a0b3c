// Internal declarations shared by the translation units of the RTE library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include "../../include/rte.h"

namespace rte {

// ---- launch accounting: every kernel launch of the library is counted ------------------------
extern std::atomic<long long> g_launches;
#define RTE_NOTE_LAUNCH() (::rte::g_launches.fetch_add(1, std::memory_order_relaxed))

// ---- error plumbing ------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define RTE_CUDA_TRY(expr)                                                                    \
  do {                                                                                        \
    cudaError_t _e = (expr);                                                                  \
    if (_e != cudaSuccess)                                                                    \
      return ::rte::fail(_e == cudaErrorMemoryAllocation ? RTE_ENOMEM : RTE_ECUDA,            \
                         std::string(#expr) + ": " + cudaGetErrorString(_e));                 \
  } while (0)

#define RTE_TRY(expr)                                                                         \
  do {                                                                                        \
    int _s = (expr);                                                                          \
    if (_s != RTE_OK) return _s;                                                              \
  } while (0)

// Switches the calling thread to the handle's device for the scope of a call, and clears an
// error that other code on this thread left in the runtime's last-error slot (the library checks
// its launches with cudaGetLastError, which would otherwise report that stale error).
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    cudaGetLastError();
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// A 1D cross section linear across a cell, from `left` at its left end to `right` at its right
// end, acts on the cell's orthonormal P1 moments as the symmetric 2x2 [[mean, off], [off, mean]]
// with mean = (left + right) / 2 and off = (right - left) / (2 sqrt 3).
__host__ __device__ __forceinline__ void linear_sigma(double left, double right, double& mean,
                                                      double& off) {
  mean = 0.5 * (left + right);
  off = (right - left) * 0.28867513459481288225;   // 1 / (2 sqrt 3)
}

// Device buffer owned by a handle.
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  int alloc(size_t count) {
    release();
    if (count == 0) return RTE_OK;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(e == cudaErrorMemoryAllocation ? RTE_ENOMEM : RTE_ECUDA,
                  std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    n = count;
    return RTE_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  ~DevBuf() { release(); }
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

constexpr int kTab2D = 16;  // doubles per (material, direction) sweep table in 2D: M^-1 (4x4)
constexpr int kTab1D = 8;   // ... in 1D, per (instance, cell, direction): Minv 2x2, inflow 2x1, 1/sqrt(h)
constexpr int kMaxDirsPerWarp = 8;
constexpr size_t kPartialBytes = size_t(64) << 20;  // per-instance sweep partial sums, upper bound

// A distinct swept direction: X-Y geometry depends on (v_x, v_y) only.
struct Dir {
  double vx, vy, w;  // w = summed weight of the merged quadrature directions
  int mult;          // how many quadrature directions were merged
  int quad;          // (v_x < 0) + 2 (v_y < 0)
};

// Consistent-DSA quadrature moments (2D); in 1D only abs_x, xx, abs3_x are used.
struct DsaMoments {
  double abs_x, abs_y, xx, yy, abs3_x, abs3_y, xx_absy, yy_absx;
};

struct SweepGroup {
  int d0, nd, quad, pad;
};

}  // namespace rte

// ---- handles -----------------------------------------------------------------------------
struct rte_disc_s {
  int device = 0;
  int dim = 2, nx = 0, ny = 1, n_cells = 0, P = 4, n_dof = 0;
  double x0 = 0, x1 = 1, y0 = 0, y1 = 1, hx = 0, hy = 0;
  int n_phi = 0, n_vz = 0, n_angles = 0, n_dirs = 0, n_mat = 0;
  std::vector<double> v, w;           // full rule, paper index order
  std::vector<rte::Dir> dirs;         // distinct directions sorted by quadrant
  std::vector<int32_t> mat_host;
  rte::DsaMoments mom{};
  rte::DevBuf<int32_t> mat_id;        // [n_cells]
  rte::DevBuf<double> dir_dev;        // [n_dirs][4] vx, vy, w, mult
  std::vector<double> dx;             // 1D: cell widths (uniform: hx each)
  rte::DevBuf<double> dx_dev;         // 1D: [nx]
  // 1D cross sections linear across cells: material at each cell's right end (matr_host is
  // mat_host when they are cellwise constant; mat_r is then not allocated and linear is false)
  std::vector<int32_t> matr_host;
  rte::DevBuf<int32_t> mat_r;         // 1D linear: [nx]
  bool linear = false;
};

namespace rte {
struct DsaState;   // 2D/1D DSA per-batch state (dsa.cu)
void dsa_state_free(DsaState*);
int dsa_setup(rte_batch_t batch, cudaStream_t st, const uint8_t* mask = nullptr);
}

struct rte_batch_s {
  rte_disc_s* disc = nullptr;
  int B = 0;
  bool params_set = false;
  int dpw = 4;                        // directions per warp in the 2D sweep (preferred / fixed)
  int min_dpw = 1;                    // smallest dpw the partial-sum buffer is sized for
  std::vector<rte::SweepGroup> groups;
  rte::DevBuf<rte::SweepGroup> groups_dev;
  // group tables for dpw = 1, 2, 4, 8; with dpw_dynamic each launch picks the largest dpw (up to
  // the preferred one) that still keeps four warps per SM busy for its number of active instances
  bool dpw_dynamic = true;
  int n_sm = 148;
  int gcount[4] = {0, 0, 0, 0}, goff[4] = {0, 0, 0, 0};
  rte::DevBuf<rte::SweepGroup> groups_all_dev;
  // measured choice of the empirical autotuner: (largest number of running instances, dpw),
  // ascending; empty = the occupancy rule above
  std::vector<std::pair<int, int>> tuned;
  std::vector<std::pair<int, int>> tuned32;   // the same, measured with the FP32 sweep
  int force_dpw = 0;                  // autotuner trials: this dpw for every launch
  int force_nw = 0;                   // autotuner trials: this many warps per direction group
  // measured warps per direction group of the FP64 sweep for each entry of `tuned` (1: one warp
  // walks all row blocks; more: the pipelined sweep2d_kba_kernel); empty = the cost model
  std::vector<int> tuned_nw;
  bool kba = true;                    // several warps per direction group when warps are scarce
  std::vector<double> sigma_t_h, sigma_s_h, source_h, inflow_h;
  // parameters taken from device memory (rte_batch_set_params_device) are validated on the device;
  // the host reads the flag when a later call first needs them (params_ready)
  rte::DevBuf<int> param_bad;
  int* param_bad_h = nullptr;             // pinned copy of param_bad
  cudaEvent_t param_ev = nullptr;         // recorded after the set-up and the flag copy
  bool param_pending = false;
  rte::DevBuf<double> sigma_t, sigma_s;   // [B][n_mat]
  rte::DevBuf<double> G0;                 // [B][n_cells] zeroth source moment int G phi_0
  rte::DevBuf<double> inflow;             // [B][4] (2D) or [B][2] (1D)
  rte::DevBuf<double> tables;             // [B][n_mat][n_dirs][kTab*]
  rte::DevBuf<double> partial;            // [B][n_groups][n_dof] per-group scalar-flux partials
  rte::DevBuf<double> S;                  // [B][n_dof] cell sources of the current sweep (2D)
  // FP32 sweep state (precision variant), allocated on first use
  rte::DevBuf<float> tables32, S32, partial32;
  bool tables32_stale = true;
  double sweep32_units = 0.0;
  // float-float sweep state (the precision variant's outer sweeps), allocated on first use
  rte::DevBuf<float> tablesff, Sff;
  bool tablesff_stale = true;
  double sweepff_units = 0.0;
  rte::DevBuf<unsigned long long> norms;  // [B][2] stop-test norms as ordered bit patterns
  rte::DevBuf<double> work;               // [B][n_dof] x 4 iteration scratch for rte_solve
  rte::DevBuf<double> outer;              // [2][B][n_dof] x0, y0 of the FP64 outer residual
                                          // correction (rte_solve_opts.refine_kappa), on first use
  rte::DevBuf<double> leak;               // [B][groups][n_cells] net face outflow partials and
  rte::DevBuf<double> vout;               // [B][4] outputs of the residual / balance check
                                          // (rte_residual, rte_solve_opts.verify), on first use
  rte::DsaState* dsa = nullptr;
  int dsa_nu = 2;                         // red-black smoothing sweeps per multigrid level (2D DSA)
  bool dsa_blocking = false;              // smoothing sweeps of a level in one temporally blocked launch
  bool dsa_tiled = false;                 // half sweeps on shared-memory tiles (rbgs_tiled_kernel)
  // pinned host staging for per-slot parameter uploads (rte_batch_set_slots), allocated on use
  double* stage = nullptr;
  uint8_t* stage_mask = nullptr;
  rte::DevBuf<uint8_t> slot_mask;         // [B] instances touched by the last slot upload
  std::vector<uint8_t> slot_set;          // parameters uploaded for this instance
  cudaEvent_t stage_ev = nullptr;         // the last upload's copies have been issued before it
  // when set, the next sweep launch records it on its stream right before its first sweep kernel
  // and clears it (rte_solve_interleaved: the host learns that the sweep has been dispatched)
  cudaEvent_t started_ev = nullptr;
  // when set (the solve loop, 2D), the sweeps' partial-sum reductions also write the correction
  // source R = sigma_s (rho_out - rho_in) of every swept instance there
  double* fuse_R = nullptr;
  // optional phase timing with CUDA events on the launching stream (rte_batch_timing)
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> sweep_ev;
  double sweep_units = 0.0;   // cell x distinct-direction solves in the timed sweeps
  long long sweep_launches = 0;
  struct PhaseEv { int phase; cudaEvent_t a, b; };
  std::vector<PhaseEv> phase_ev;   // phases: 0 FP32 sweep, 1 DSA, 2 ROM, 3 set-up, 4 float-float sweep
  long long phase_calls[5] = {0, 0, 0, 0, 0};
  size_t bytes() const;                   // device memory held by the batch
  ~rte_batch_s();
};

namespace rte {
// RTE_OK when the batch has parameters; RTE_ESTATE ("<who>: parameters not set") otherwise.
// Parameters set from device memory are checked here the first time: the host waits for their
// set-up and reads the device's validation flag (RTE_EINVAL, and no parameters, if it failed).
int params_ready(rte_batch_t b, const char* who);

// Brackets one phase of work on `st` with CUDA events when the batch is timing (no-op otherwise).
struct PhaseScope {
  rte_batch_t b;
  int phase;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  PhaseScope(rte_batch_t b_, int phase_, cudaStream_t st_) : b(b_), phase(phase_), st(st_) {
    if (b->timing && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, st);
  }
  ~PhaseScope() {
    if (!a) return;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) == cudaSuccess) {
      cudaEventRecord(e, st);
      b->phase_ev.push_back({phase, a, e});
      b->phase_calls[phase] += 1;
    } else {
      cudaEventDestroy(a);
    }
  }
};
void make_groups(rte_batch_t b);
int auto_dpw(const rte_disc_s* disc, int B);
// groups of one launch: dpw, number of groups and their device table
void pick_groups(rte_batch_t b, int n_active, int* dpw, int* n_groups, const SweepGroup** dev,
                 bool f32 = false);
// sweep.cu
int sweep_launch(rte_batch_t b, const double* rho_in, double* rho_out, double* psi_out,
                 int with_source, const uint8_t* active, cudaStream_t st, bool fuse_norms,
                 int n_active = -1, bool zero_norms = true);
int norms_to_host(rte_batch_t b, double* host, cudaStream_t st);
// Arguments of the 2D FP64 sweep kernels (sweep.cu): one batch's arrays and sizes for one launch.
struct Sweep2DArgs {
  const double* rho_in;     // or, when the kernel is instantiated with PRESRC, the sources S
  double* partial;
  double* psi_out;
  const uint8_t* active;
  const double* tables;
  const double* sigma_s;
  const double* G0;
  const double* inflow;
  const int32_t* mat;
  const double* dirs;
  const SweepGroup* groups;
  int nx, ny, n_cells, n_dof, n_mat, n_dirs, n_groups, with_source;
  double sq_area;
  double ihx, ihy;          // 1 / h_x, 1 / h_y
  // balance accounting (kernels instantiated with LEAK only): per (running instance, group, cell)
  // the omega-weighted net outflow through the cell's faces; lx = sqrt(h_y / h_x) and
  // ly = sqrt(h_x / h_y) turn a face trace's zeroth coefficient into the face integral
  double* leak = nullptr;
  double lx = 0.0, ly = 0.0;
};

// A work item of the multi-batch sweep: one direction group of one instance of one batch.
struct SweepItem {
  int batch, group, inst, pad;
};

// one FP64 sweep of several 2D batches in one work-queue launch (sweep.cu)
struct MultiSweepScratch {
  DevBuf<Sweep2DArgs> descs;
  DevBuf<SweepItem> items;
  DevBuf<int> counter;
  std::vector<Sweep2DArgs> h_descs;
  std::vector<SweepItem> h_items;
};
int sweep_launch_multi(const std::vector<rte_batch_t>& bts, const std::vector<const double*>& rho_in,
                       const std::vector<double*>& rho_out, const std::vector<const uint8_t*>& act,
                       const std::vector<const uint8_t*>& host_act, MultiSweepScratch& ws,
                       cudaStream_t st);
// FP32 sweep; the instances flagged in `inner` sweep the error rho_in - x0 without sources and
// get y0 added in the reduction (the correction sweeps of the FP64 outer residual correction)
int sweep_launch_f32(rte_batch_t bt, const double* rho_in, double* rho_out, const uint8_t* active,
                     cudaStream_t st, int n_active, bool zero_norms = true,
                     const uint8_t* inner = nullptr, const double* x0 = nullptr,
                     const double* y0 = nullptr);
// float-float sweep with source (the precision variant's outer sweeps), reduced in FP64
int sweep_launch_ff(rte_batch_t bt, const double* rho_in, double* rho_out, const uint8_t* active,
                    cudaStream_t st, int n_active, bool fuse_norms, bool zero_norms = true);
int setup_tables(rte_batch_t b, cudaStream_t st, const uint8_t* mask = nullptr);
// one FP64 sweep with source that also records each cell's net face outflow (bt->leak)
int sweep_launch_leak(rte_batch_t bt, const double* rho_in, double* rho_out, const uint8_t* active,
                      cudaStream_t st, int* n_groups);
// verify.cu: residual ||(I - L) rho - b||_inf and particle balance of every instance in `active`
// (all when null): out DEVICE double[B][4], cell_balance DEVICE double[B][n_cells] or null
int residual_launch(rte_batch_t bt, const double* rho, double* out, double* cell_balance,
                    const uint8_t* active, cudaStream_t st);
size_t dsa_bytes(const rte_batch_s* b);
// noalloc.cu: looks up the allocation-free sweep's static scratch on the current device, which
// loads (and allocates) it there if it was not loaded yet; called when a batch is created
int static_scratch_preload();
// per-slot parameter upload: instances slots[0..n) take the given parameters (host arrays)
int set_slots(rte_batch_t b, int n, const int* slots, const double* sigma_t, const double* sigma_s,
              const double* source, const double* inflow, cudaStream_t st);
int correction_source_launch(rte_batch_t b, const double* rs, const double* rp, double* R,
                             const uint8_t* active, cudaStream_t st);
int axpy_launch(rte_batch_t b, const double* x, const double* y, double* out,
                const uint8_t* active, cudaStream_t st);  // out = x + y (x when y is null)
int dsa_apply(rte_batch_t b, const double* R, double* drho, double rtol, int max_it,
              const uint8_t* active, int* iters, cudaStream_t st);
// A single FP32 V-cycle (2D, dsa_rtol 0, one cycle) whose result goes straight into the SI update:
// rho_out = rho_star + delta rho for the instances in `active` (no delta-rho array)
bool dsa_update_fusable(rte_batch_t b, double rtol, int max_it);
int dsa_apply_update(rte_batch_t b, const double* R, const double* rho_star, double* rho_out,
                     const uint8_t* active, cudaStream_t st);
}  // namespace rte

namespace rte { struct RomOnline; }

struct rte_rom_s {
  rte_disc_s* disc = nullptr;
  int r = 0, n_snap = 0;
  std::vector<double> sv;
  double eps_equiv = 0;
  rte::DevBuf<double> U;       // [r][n_dirs][n_dof]: basis vectors (offline only, then freed)
  rte::DevBuf<double> U_rho;   // [r][n_dof]
  rte::DevBuf<double> U_iso;   // [r][n_dof]
  rte::DevBuf<double> U_iso0;  // [r][n_cells] zeroth-moment rows of U_iso
  rte::DevBuf<double> a_side;  // [4][r] projection of a unit isotropic inflow through each side
  std::vector<double> A0;      // [r][r]
  std::vector<double> Aa, As;  // [n_mat][r][r]
  rte::DevBuf<double> A0_dev, Aa_dev, As_dev;
  rte::RomOnline* online = nullptr;
  ~rte_rom_s();
};

namespace rte {
int rom_prepare(rte_rom_t rom, rte_batch_t bt, cudaStream_t st, const uint8_t* mask = nullptr);
int rom_correction(rte_rom_t rom, rte_batch_t bt, const double* R, double* drho,
                   const uint8_t* active, cudaStream_t st, bool bf16 = false);
// status word of the BF16 tensor-core products of this ROM's online state (0 if never used):
// nonzero when a device-side wait gave up; read after the stream is synchronised, then cleared
int rom_tc_status(rte_rom_t rom, int* status);
// podtc.cu: BF16 tensor-core POD products (see rte_pod_project_bf16 / rte_pod_lift_bf16)
size_t pod_project_ws_bytes(int n, int B, int n_sm);
int pod_project_bf16(const double* U, int r, int n, const double* X, int B, const uint8_t* active,
                     double* out, void* ws, int n_sm, cudaStream_t st);
int pod_lift_bf16(const double* U, int r, int n, const double* C, int B, const uint8_t* active,
                  double* Y, int* status, cudaStream_t st);
// ROMIG initial guess rho0 = U^rho A_{mu,r}^{-1} (U^iso)^T G for the instances in `mask`
int rom_guess_launch(rte_rom_t rom, rte_batch_t bt, double* rho0, const uint8_t* mask,
                     cudaStream_t st);

// Per-batch state of Alg. 1 / Alg. 2 for instances that may start and finish at different
// times: one instance is one slot of the batch, with its own iteration count, tolerance and
// report.  si_launch issues one sweep of every running instance and the asynchronous copy of
// the stop-test norms; si_finish waits for those norms, applies the stop test and issues the
// corrections.  Both only enqueue work on the stream, so several batches on several streams
// progress concurrently from one host thread.
struct SiState {
  rte_batch_t bt = nullptr;
  int B = 0;
  rte_solve_opts o{};
  rte_rom_t rom = nullptr;
  bool mixed = false;                 // FP32 sweeps until the change drops below fp32_switch
  bool refine = false;                // FP64 outer residual correction with FP32 inner sweeps
  uint8_t* hm = nullptr;              // pinned [10][B]: act, lo, hi, inner (sweep) | act, rom,
                                      // dsa, enter (correction) | converged, expired (result
                                      // copies); enter = the FP64 sweep just done is an outer point
  unsigned long long* hn = nullptr;   // pinned [2B] stop-test norms (ordered bit patterns)
  DevBuf<uint8_t> dm;                 // device copy of hm
  cudaEvent_t ev = nullptr;           // recorded after the norms copy
  cudaEvent_t started = nullptr;      // rte_solve_interleaved: recorded before the sweep kernel
  cudaEvent_t corr = nullptr;         // rte_solve_interleaved: recorded after the corrections
  bool r_fused = false;               // the launch in flight also formed the correction source
  std::vector<uint8_t> act, lowp, done;
  std::vector<uint8_t> inner;         // the next sweep is an FP32 correction sweep
  std::vector<uint8_t> swept;         // swept in the launch in flight (not waiting, gang_wait)
  std::vector<int> it, status, n_inner, waited;
  std::vector<double> eps, outer_test;  // outer_test: stop-test quantity of the last FP64 sweep
  std::vector<rte_solve_report> rep;
  bool in_flight = false;
  double* result = nullptr;           // [B][n_dof] destination of finished instances (device or pinned host)
  bool result_dev = false;            // result is device memory: one masked copy kernel per iteration
  int init(rte_batch_t b, const rte_solve_opts& opts, rte_rom_t rom_c, double* result_dst);
  void begin(int b, double eps_b);    // the instance's initial iterate is already in slot b of work
  int n_active() const;
  ~SiState();
};
int si_launch(SiState& s, cudaStream_t st, double* psi_cur, cudaEvent_t wait_ev = nullptr);
int event_ready(cudaEvent_t ev, bool* ready);
int si_finish(SiState& s, cudaStream_t st, double* history);
}  // namespace rte
