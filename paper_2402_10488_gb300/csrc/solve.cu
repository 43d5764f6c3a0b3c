// Source iteration with synthetic acceleration (paper Alg. 1) with the ROMSAD switch (Alg. 2).
//
// Every instance of a batch runs its own Alg. 1: sweep (fused scalar-flux reduction and stop-
// test norms), stop test, then the correction chosen for it -- DSA (App. B), ROMSA
// (Eq. (rom_correction)) or, for ROMSAD, ROMSA iff 1 <= l <= theta and the change is at least
// eps_ROMSAD.  Instances that have converged drop out of every later launch through a device
// mask.  The only host round trip per iteration is the 2*B stop-test norms.
//
// Precision variant: an instance may sweep in FP32 while its change is above fp32_switch, and with
// refine_kappa > 0 every FP64 sweep that does not stop it opens an outer residual-correction step:
// the FP64 sweep y0 = L x0 + b of the iterate x0 gives the residual r = y0 - x0 of
// (I - L) rho = b (Eq. (rho_matrix_vec)), and the following sweeps solve (I - L) e = r for the
// error e = rho - x0 by the same SI iterations (DSA / ROMSA corrections unchanged) with the sweep of
// e in FP32, rho^(l,*) = y0 + L (rho^(l-1) - x0), until the change is refine_kappa times smaller
// than the FP64 one; then the next FP64 sweep evaluates the new residual.  FP32 rounding thus only
// enters through e, which shrinks from one outer step to the next, and the stop test sees FP64
// sweeps only (with outer_ff those FP64-grade sweeps run in float-float arithmetic, sweep.cu).
//
// The iteration is a small state machine per batch (SiState): instances are slots that may
// start at different iterations (serving), and si_launch / si_finish only enqueue work, so one
// host thread keeps several batches of different discretisations busy on their own streams
// (rte_solve_many, the serving loop).
#include <deque>
#include <thread>

#include "common.cuh"

namespace rte {

int SiState::init(rte_batch_t b, const rte_solve_opts& opts, rte_rom_t rom_c, double* result_dst) {
  bt = b;
  B = b->B;
  o = opts;
  rom = rom_c;
  result = result_dst;
  mixed = o.fp32_switch > 0.0 && b->disc->dim == 2;
  refine = o.refine_kappa > 0.0 && b->disc->dim == 2;
  if (refine && b->outer.n < 2 * (size_t)B * b->disc->n_dof)
    RTE_TRY(b->outer.alloc(2 * (size_t)B * b->disc->n_dof));
  if (!hm) {
    RTE_CUDA_TRY(cudaHostAlloc((void**)&hm, 10 * (size_t)B, cudaHostAllocDefault));
    RTE_CUDA_TRY(cudaHostAlloc((void**)&hn, sizeof(unsigned long long) * 2 * B, cudaHostAllocDefault));
    RTE_TRY(dm.alloc(10 * (size_t)B));
    RTE_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  std::memset(hm, 0, 10 * (size_t)B);
  cudaPointerAttributes pa{};
  result_dev = cudaPointerGetAttributes(&pa, result) == cudaSuccess &&
               pa.type == cudaMemoryTypeDevice;
  cudaGetLastError();   // a pointer the runtime does not know is not an error here
  act.assign(B, 0);
  lowp.assign(B, 0);
  done.assign(B, 0);
  inner.assign(B, 0);
  swept.assign(B, 0);
  it.assign(B, 0);
  n_inner.assign(B, 0);
  waited.assign(B, 0);
  status.assign(B, RTE_OK);
  eps.assign(B, o.eps);
  outer_test.assign(B, 0.0);
  rep.assign(B, rte_solve_report{});
  in_flight = false;
  return RTE_OK;
}

void SiState::begin(int b, double eps_b) {
  act[b] = 1;
  lowp[b] = mixed ? 1 : 0;
  done[b] = 0;
  inner[b] = 0;
  swept[b] = 0;
  it[b] = 0;
  n_inner[b] = 0;
  waited[b] = 0;
  status[b] = RTE_OK;
  eps[b] = eps_b;
  rep[b] = rte_solve_report{};
}

int SiState::n_active() const {
  int n = 0;
  for (int b = 0; b < B; ++b) n += act[b];
  return n;
}

SiState::~SiState() {
  if (hm) cudaFreeHost(hm);
  if (hn) cudaFreeHost(hn);
  if (ev) cudaEventDestroy(ev);
  if (started) cudaEventDestroy(started);
  if (corr) cudaEventDestroy(corr);
}

// One sweep of every running instance: rho^(l,*) = L rho^(l-1) + b (FP32 for instances still in
// the low-precision phase or inside an outer residual-correction step), then the asynchronous copy
// of the stop-test norms.  With wait_ev the stream first waits for that event (the batch's
// corrections when they run on another stream); with s.started set, that event is recorded right
// before the first sweep kernel.
int si_launch(SiState& s, cudaStream_t st, double* psi_cur, cudaEvent_t wait_ev) {
  rte_batch_t bt = s.bt;
  const int B = s.B;
  const size_t nb = (size_t)B * bt->disc->n_dof;
  double* rho_prev = bt->work.p;
  double* rho_star = bt->work.p + nb;
  uint8_t *h_act = s.hm, *h_lo = s.hm + B, *h_hi = s.hm + 2 * B, *h_in = s.hm + 3 * B;
  int n_lo = 0, n_hi = 0, n_in = 0;
  for (int b = 0; b < B; ++b) {
    const bool in = s.act[b] && s.inner[b] && psi_cur == nullptr;
    const bool lo = s.act[b] && (s.lowp[b] || in) && psi_cur == nullptr;
    s.swept[b] = s.act[b];
    h_lo[b] = lo;
    h_hi[b] = s.act[b] && !lo;
    h_in[b] = in;
    n_lo += h_lo[b], n_hi += h_hi[b], n_in += in;
  }
  if (s.o.gang_wait > 0 && n_lo > 0 && n_hi > 0) {
    // instances due for an FP64 sweep wait while others still sweep in FP32 (bounded)
    for (int b = 0; b < B; ++b)
      if (h_hi[b] && s.waited[b] < s.o.gang_wait) {
        h_hi[b] = 0, s.swept[b] = 0, n_hi--;
        s.waited[b]++;
      }
  }
  for (int b = 0; b < B; ++b) {
    h_act[b] = s.swept[b];
    if (h_hi[b]) s.waited[b] = 0;
  }
  if (n_lo + n_hi == 0) return RTE_OK;
  if (wait_ev) RTE_CUDA_TRY(cudaStreamWaitEvent(st, wait_ev, 0));
  RTE_CUDA_TRY(cudaMemcpyAsync(s.dm.p, s.hm, 4 * (size_t)B, cudaMemcpyHostToDevice, st));
  bt->started_ev = s.started;
  // the reductions form the correction source of the next correction as they go (2D, not for the
  // training solves' psi capture)
  s.r_fused = s.o.sa != RTE_SA_NONE && bt->disc->dim == 2 && psi_cur == nullptr;
  bt->fuse_R = s.r_fused ? bt->work.p + 2 * nb : nullptr;
  // the precision variant's FP64-grade sweeps in float-float arithmetic (rte_solve_opts.outer_ff)
  const bool ff = s.o.outer_ff && (s.mixed || s.refine) && psi_cur == nullptr;
  if (n_lo == 0) {
    RTE_TRY(ff ? sweep_launch_ff(bt, rho_prev, rho_star, s.dm.p, st, n_hi, true)
               : sweep_launch(bt, rho_prev, rho_star, psi_cur, 1, s.dm.p, st, true, n_hi));
  } else {
    RTE_CUDA_TRY(cudaMemsetAsync(bt->norms.p, 0, sizeof(unsigned long long) * 2 * B, st));
    const double* x0 = bt->outer.p;
    const double* y0 = bt->outer.p ? bt->outer.p + nb : nullptr;
    RTE_TRY(sweep_launch_f32(bt, rho_prev, rho_star, s.dm.p + B, st, n_lo, false,
                             n_in ? s.dm.p + 3 * B : nullptr, x0, y0));
    if (n_hi > 0)
      RTE_TRY(ff ? sweep_launch_ff(bt, rho_prev, rho_star, s.dm.p + 2 * B, st, n_hi, true, false)
                 : sweep_launch(bt, rho_prev, rho_star, psi_cur, 1, s.dm.p + 2 * B, st, true, n_hi, false));
  }
  bt->started_ev = nullptr;
  bt->fuse_R = nullptr;
  RTE_CUDA_TRY(cudaMemcpyAsync(s.hn, bt->norms.p, sizeof(unsigned long long) * 2 * B,
                               cudaMemcpyDeviceToHost, st));
  RTE_CUDA_TRY(cudaEventRecord(s.ev, st));
  s.in_flight = true;
  return RTE_OK;
}

// dst[b] = src[b] for the instances flagged in `mask` (results of finished instances).
__global__ void copy_rows_kernel(double* dst, const double* src, const uint8_t* mask, int n_dof) {
  const int b = blockIdx.y;
  if (!mask[b]) return;
  const size_t o = (size_t)b * n_dof;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_dof; e += gridDim.x * blockDim.x)
    dst[o + e] = src[o + e];
}

// Copies the rows of the finished instances flagged in hflag (host) / dflag (device) from src to
// s.result: one kernel when the result is in device memory, else one copy per instance.
static int copy_finished(SiState& s, const double* src, const uint8_t* hflag, const uint8_t* dflag,
                         int n_fin, cudaStream_t st) {
  if (n_fin == 0) return RTE_OK;
  const int n = s.bt->disc->n_dof;
  if (s.result_dev) {
    dim3 grid(std::min((n + 255) / 256, 256), s.B);
    copy_rows_kernel<<<grid, 256, 0, st>>>(s.result, src, dflag, n); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
  }
  for (int b = 0; b < s.B; ++b)
    if (hflag[b])
      RTE_CUDA_TRY(cudaMemcpyAsync(s.result + (size_t)b * n, src + (size_t)b * n,
                                   sizeof(double) * n, cudaMemcpyDefault, st));
  return RTE_OK;
}

// Stop test and correction of the iteration launched by si_launch.  Finished instances (converged,
// or at the iteration cap) have their result copied to s.result and are flagged in s.done.
int si_finish(SiState& s, cudaStream_t st, double* history) {
  if (!s.in_flight) return RTE_OK;
  RTE_CUDA_TRY(cudaEventSynchronize(s.ev));
  s.in_flight = false;
  rte_batch_t bt = s.bt;
  const rte_solve_opts& o = s.o;
  const int B = s.B;
  const size_t n = bt->disc->n_dof, nb = (size_t)B * n;
  double* rho_prev = bt->work.p;
  double* rho_star = bt->work.p + nb;
  double* R = bt->work.p + 2 * nb;
  double* drho = bt->work.p + 3 * nb;
  uint8_t *h_corr = s.hm + 4 * B, *h_rom = s.hm + 5 * B, *h_dsa = s.hm + 6 * B;
  uint8_t *h_enter = s.hm + 7 * B, *h_conv = s.hm + 8 * B, *h_exp = s.hm + 9 * B;
  int n_conv = 0, n_exp = 0, n_enter = 0;
  bool any = false, anyd = false, anyr = false;
  for (int b = 0; b < B; ++b) {
    h_corr[b] = h_rom[b] = h_dsa[b] = h_enter[b] = h_conv[b] = h_exp[b] = 0;
    if (!s.act[b] || !s.swept[b]) continue;
    const int l = ++s.it[b];
    double delta, rinf;
    std::memcpy(&delta, &s.hn[2 * b], sizeof(double));
    std::memcpy(&rinf, &s.hn[2 * b + 1], sizeof(double));
    if (history) history[(size_t)b * o.max_iter + (l - 1)] = delta;
    if (o.sa_history) o.sa_history[(size_t)b * o.max_iter + (l - 1)] = s.hm[B + b] ? 0x10 : 0;
    rte_solve_report& rp = s.rep[b];
    rp.n_sweep = l;
    rp.last_change = delta;
    rp.rho_inf = rinf;
    const double test = o.rel ? delta / rinf : delta;
    if (s.lowp[b]) {
      rp.n_sweep32++;
      if (test < o.fp32_switch) s.lowp[b] = 0;  // later sweeps of this instance in FP64
    } else if (s.inner[b]) {
      // FP32 sweep of the correction equation: back to FP64 once the error equation's change is
      // refine_kappa times below the outer residual, or after refine_inner sweeps
      rp.n_sweep32++;
      if (++s.n_inner[b] >= o.refine_inner || test < o.refine_kappa * s.outer_test[b])
        s.inner[b] = 0;
    } else if (test < s.eps[b]) {
      rp.converged = 1;
      s.act[b] = 0;
      s.done[b] = 1;
      s.status[b] = RTE_OK;
      h_conv[b] = 1, n_conv++;
      continue;
    } else if (s.refine) {
      // this FP64 sweep is the outer point: x0 = rho^(l-1), y0 = rho^(l,*)
      s.inner[b] = 1;
      s.n_inner[b] = 0;
      s.outer_test[b] = test;
      h_enter[b] = 1, n_enter++;
    }
    if (l >= o.max_iter) h_exp[b] = 1, n_exp++;
    any = true;
    h_corr[b] = 1;
    if (o.sa == RTE_SA_NONE) {
      if (o.sa_history) o.sa_history[(size_t)b * o.max_iter + (l - 1)] = s.hm[B + b] ? 0x10 : 0;
      continue;
    }
    bool romsa = o.sa == RTE_SA_ROMSA;
    if (o.sa == RTE_SA_ROMSAD)
      romsa = o.schedule ? o.schedule[l - 1] != 0 : (l <= o.theta && delta >= o.eps_romsad);
    if (romsa) h_rom[b] = 1, rp.n_romsa++, anyr = true;
    else h_dsa[b] = 1, rp.n_dsa++, anyd = true;
    if (o.sa_history)   // the correction that follows sweep l; 0x10 marks an FP32 sweep
      o.sa_history[(size_t)b * o.max_iter + (l - 1)] =
          (uint8_t)((romsa ? RTE_SA_ROMSA : RTE_SA_DSA) | (s.hm[B + b] ? 0x10 : 0));
  }
  if (any || n_conv || n_exp)
    RTE_CUDA_TRY(cudaMemcpyAsync(s.dm.p + 4 * B, h_corr, 6 * (size_t)B, cudaMemcpyHostToDevice, st));
  RTE_TRY(copy_finished(s, rho_star, h_conv, s.dm.p + 8 * B, n_conv, st));
  if (n_enter) {
    // keep the outer point and its FP64 sweep before the correction overwrites rho_prev
    const int n = bt->disc->n_dof;
    dim3 grid(std::min((n + 255) / 256, 256), B);
    copy_rows_kernel<<<grid, 256, 0, st>>>(bt->outer.p, rho_prev, s.dm.p + 7 * B, n); RTE_NOTE_LAUNCH();
    copy_rows_kernel<<<grid, 256, 0, st>>>(bt->outer.p + nb, rho_star, s.dm.p + 7 * B, n); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
  }
  if (any) {
    const uint8_t* d_corr = s.dm.p + 4 * B;
    if (o.sa == RTE_SA_NONE) {
      // plain SI: rho^(l) = rho^(l,*)
      RTE_TRY(axpy_launch(bt, rho_star, nullptr, rho_prev, d_corr, st));
    } else {
      if (!s.r_fused) RTE_TRY(correction_source_launch(bt, rho_star, rho_prev, R, d_corr, st));
      // a single V-cycle writes rho^(l) = rho^(l,*) + delta rho^(l) itself (after R is formed from
      // rho_prev), so only the ROMSA instances need the separate update below
      const bool fused = anyd && dsa_update_fusable(bt, o.dsa_rtol, o.dsa_max_it);
      if (anyd) {
        std::vector<int> iters(B, 0);
        PhaseScope ps(bt, 1, st);
        int e = fused ? dsa_apply_update(bt, R, rho_star, rho_prev, s.dm.p + 6 * B, st)
                      : dsa_apply(bt, R, drho, o.dsa_rtol, o.dsa_max_it, s.dm.p + 6 * B, iters.data(), st);
        if (e != RTE_OK && e != RTE_ENOCONV) return e;
        for (int b = 0; b < B; ++b)
          if (h_dsa[b]) s.rep[b].dsa_iters += fused ? 1 : iters[b];
      }
      if (anyr) {
        PhaseScope ps(bt, 2, st);
        RTE_TRY(rom_correction(s.rom, bt, R, drho, s.dm.p + 5 * B, st, o.rom_bf16 != 0));
      }
      // rho^(l) = rho^(l,*) + delta rho^(l), written into the rho_prev slot
      if (!fused || anyr) RTE_TRY(axpy_launch(bt, rho_star, drho, rho_prev, fused ? s.dm.p + 5 * B : d_corr, st));
    }
  }
  for (int b = 0; b < B; ++b)
    if (h_exp[b]) {
      s.act[b] = 0;
      s.done[b] = 1;
      s.status[b] = RTE_ENOCONV;
    }
  RTE_TRY(copy_finished(s, rho_prev, h_exp, s.dm.p + 9 * B, n_exp, st));
  return RTE_OK;
}

// rte_solve_opts.verify: R^rho_inf and the particle balance of every instance's result (in DEVICE
// memory) into its report.  Synchronises the stream.
static int verify_results(SiState& s, cudaStream_t st) {
  rte_batch_t bt = s.bt;
  if (!s.result_dev) return fail(RTE_EINVAL, "verify: the result must be in device memory");
  if (bt->vout.n < 4 * (size_t)s.B) RTE_TRY(bt->vout.alloc(4 * (size_t)s.B));
  RTE_TRY(residual_launch(bt, s.result, bt->vout.p, nullptr, nullptr, st));
  std::vector<double> v(4 * (size_t)s.B);
  RTE_CUDA_TRY(cudaMemcpyAsync(v.data(), bt->vout.p, sizeof(double) * v.size(),
                               cudaMemcpyDeviceToHost, st));
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  for (int b = 0; b < s.B; ++b) {
    s.rep[b].r_inf = v[4 * b];
    s.rep[b].balance_cell = v[4 * b + 1];
    s.rep[b].balance = v[4 * b + 2];
  }
  return RTE_OK;
}

// All instances of the batch from the initial iterates in `rho` (overwritten with the results).
// With psi_cur the angular flux of the latest sweep is kept, and the first `window` sweeps are
// also copied to psi_win (training solves of the offline stage).
int run_si(rte_batch_t bt, const rte_solve_opts* o, rte_rom_t rom_c, double* rho,
           rte_solve_report* reports, double* history, cudaStream_t st, double* psi_cur,
           double* psi_win, int window) {
  const rte_disc_s* d = bt->disc;
  const int B = bt->B;
  const size_t n = d->n_dof;
  if ((o->sa == RTE_SA_ROMSA || o->sa == RTE_SA_ROMSAD) && !rom_c)
    return fail(RTE_EINVAL, "ROMSA/ROMSAD need a correction ROM");
  SiState s;
  rte_solve_opts oo = *o;
  if (psi_cur) oo.fp32_switch = 0.0, oo.refine_kappa = 0.0;
  RTE_TRY(s.init(bt, oo, rom_c, rho));
  RTE_CUDA_TRY(cudaMemcpyAsync(bt->work.p, rho, sizeof(double) * B * n, cudaMemcpyDeviceToDevice, st));
  for (int b = 0; b < B; ++b) s.begin(b, o->eps);
  if (rom_c) {
    PhaseScope ps(bt, 2, st);
    RTE_TRY(rom_prepare(rom_c, bt, st));
  }
  const size_t psi_per = (size_t)d->n_dirs * n;
  for (int l = 1; s.n_active() > 0; ++l) {
    RTE_TRY(si_launch(s, st, psi_cur));
    if (psi_win && l <= window)
      for (int b = 0; b < B; ++b)
        if (s.act[b])
          RTE_CUDA_TRY(cudaMemcpyAsync(psi_win + ((size_t)(l - 1) * B + b) * psi_per,
                                       psi_cur + (size_t)b * psi_per, sizeof(double) * psi_per,
                                       cudaMemcpyDeviceToDevice, st));
    RTE_TRY(si_finish(s, st, history));
  }
  if (o->verify) RTE_TRY(verify_results(s, st));
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  int status = RTE_OK;
  for (int b = 0; b < B; ++b)
    if (s.status[b] != RTE_OK) status = s.status[b];
  if (rom_c && o->rom_bf16) {
    int tc = 0;
    RTE_TRY(rom_tc_status(rom_c, &tc));
    if (tc) return fail(RTE_ETIMEOUT, "BF16 ROM product: a device-side wait gave up");
  }
  if (reports)
    for (int b = 0; b < B; ++b) reports[b] = s.rep[b];
  return status;
}

// Readiness of an event without leaving cudaErrorNotReady in the thread's last-error slot.
int event_ready(cudaEvent_t ev, bool* ready) {
  const cudaError_t q = cudaEventQuery(ev);
  if (q == cudaSuccess) {
    *ready = true;
    return RTE_OK;
  }
  if (q == cudaErrorNotReady) {
    cudaGetLastError();
    *ready = false;
    return RTE_OK;
  }
  return fail(RTE_ECUDA, std::string("cudaEventQuery: ") + cudaGetErrorString(q));
}

}  // namespace rte

using namespace rte;

static int check_opts(rte_batch_t b, const rte_solve_opts* o, rte_rom_t rom_c) {
  RTE_TRY(params_ready(b, "rte_solve"));
  if (!(o->eps >= 0) || o->max_iter < 1 || o->sa < 0 || o->sa > 3 || !(o->fp32_switch >= 0) ||
      !(o->refine_kappa >= 0) || (o->refine_kappa > 0 && o->refine_inner < 1) || o->gang_wait < 0 ||
      o->verify < 0 || o->verify > 1 || o->outer_ff < 0 || o->outer_ff > 1)
    return fail(RTE_EINVAL, "rte_solve: bad options");
  if (o->sa != RTE_SA_NONE && b->disc->dim == 2 && (!(o->dsa_rtol >= 0) || o->dsa_max_it < 1))
    return fail(RTE_EINVAL, "rte_solve: bad DSA tolerance");
  if (rom_c && rom_c->disc != b->disc) return fail(RTE_EINVAL, "ROM built on another discretisation");
  if ((o->sa == RTE_SA_ROMSA || o->sa == RTE_SA_ROMSAD) && !rom_c)
    return fail(RTE_EINVAL, "ROMSA/ROMSAD need a correction ROM");
  return RTE_OK;
}

extern "C" int rte_solve(rte_batch_t b, const rte_solve_opts* o, rte_rom_t rom_c, double* rho,
                         rte_solve_report* reports, double* history, void* stream) {
  if (!b || !o || !rho) return fail(RTE_EINVAL, "rte_solve: null argument");
  RTE_TRY(check_opts(b, o, rom_c));
  DeviceGuard g(b->disc->device);
  return run_si(b, o, rom_c, rho, reports, history, (cudaStream_t)stream, nullptr, nullptr, 0);
}

// Arguments of rte_solve_many / rte_solve_interleaved.
static int check_many(const char* who, int n, const rte_batch_t* batches, const rte_solve_opts* opts,
                      const rte_rom_t* roms, double* const* rho) {
  const std::string w(who);
  if (n < 1 || !batches || !opts || !rho) return fail(RTE_EINVAL, w + ": null argument");
  for (int k = 0; k < n; ++k) {
    if (!batches[k] || !rho[k]) return fail(RTE_EINVAL, w + ": null batch or rho");
    if (batches[k]->disc->device != batches[0]->disc->device)
      return fail(RTE_EINVAL, w + ": batches on different devices");
    for (int j = 0; j < k; ++j) {
      if (batches[j] == batches[k]) return fail(RTE_EINVAL, w + ": batch listed twice");
      if (roms && roms[k] && roms[j] == roms[k])
        return fail(RTE_EINVAL, w + ": a ROM serves one batch at a time");
    }
    RTE_TRY(check_opts(batches[k], &opts[k], roms ? roms[k] : nullptr));
  }
  return RTE_OK;
}

// The end of a multi-batch solve: verification, stream synchronisation, reports, status.
static int finish_many(std::vector<SiState>& S, const std::vector<cudaStream_t>& st,
                       const rte_solve_opts* opts, const rte_rom_t* roms,
                       rte_solve_report* const* reports) {
  const int n = (int)S.size();
  int status = RTE_OK;
  for (int k = 0; k < n; ++k) {
    if (opts[k].verify) RTE_TRY(verify_results(S[k], st[k]));
    RTE_CUDA_TRY(cudaStreamSynchronize(st[k]));
    if (roms && roms[k] && opts[k].rom_bf16) {
      int tc = 0;
      RTE_TRY(rom_tc_status(roms[k], &tc));
      if (tc) return fail(RTE_ETIMEOUT, "BF16 ROM product: a device-side wait gave up");
    }
    for (int b = 0; b < S[k].B; ++b) {
      if (S[k].status[b] != RTE_OK) status = S[k].status[b];
      if (reports && reports[k]) reports[k][b] = S[k].rep[b];
    }
  }
  return status;
}

// Whether the next sweep of s is a wide FP64 launch: every running instance sweeps in FP64 and at
// least half the batch is running.  Such launches keep every SM sub-partition's FP64 pipe busy on
// their own; narrower ones (the convergence tail) and FP32 sweeps are latency-bound.
static bool wide_fp64(const SiState& s) {
  int hi = 0;
  for (int b = 0; b < s.B; ++b) {
    if (!s.act[b]) continue;
    if (s.lowp[b] || s.inner[b]) return false;
    ++hi;
  }
  return 2 * hi >= s.B;
}

// rte_solve_many with the wide FP64 sweeps of all batches on one stream of the highest priority,
// one after another, and each batch's stop test and corrections on its own stream: while one batch
// sweeps, the others' corrections (DSA V-cycles on the FP32 pipe and the memory system, ROM
// products) run beside it on the SMs that the FP64-bound sweep leaves idle.  Narrow and FP32
// sweeps, latency-bound, run on the batch's own stream, concurrently with the others.  A sweep's
// one-warp CTAs must be placed on an idle GPU -- dispatched while other kernels fill the SMs they
// crowd onto some SM sub-partitions, whose FP64 pipes then carry two to three times their share
// (measured: a half-batch sweep 2.45 ms alone, 7.1 ms dispatched together with a V-cycle) -- so
// a batch's corrections are issued only once the wide sweep queued next on the priority stream
// has recorded `started` (after its cell sources, before its sweep kernel).
extern "C" int rte_solve_interleaved(int n, const rte_batch_t* batches, const rte_solve_opts* opts,
                                     const rte_rom_t* roms, double* const* rho,
                                     rte_solve_report* const* reports, void* const* streams) {
  RTE_TRY(check_many("rte_solve_interleaved", n, batches, opts, roms, rho));
  DeviceGuard g(batches[0]->disc->device);
  int prio_low = 0, prio_high = 0;
  RTE_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  cudaStream_t sw = nullptr;
  RTE_CUDA_TRY(cudaStreamCreateWithPriority(&sw, cudaStreamNonBlocking, prio_high));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  } sg{sw};
  std::vector<SiState> S(n);
  std::vector<cudaStream_t> st(n);
  std::deque<int> wide;   // batches whose sweep in flight is queued on sw, in queue order
  // queue the next sweep of batch k behind its corrections: wide FP64 sweeps on sw, others on st[k]
  auto launch = [&](int k) -> int {
    if (wide_fp64(S[k])) {
      RTE_CUDA_TRY(cudaEventRecord(S[k].corr, st[k]));
      RTE_TRY(si_launch(S[k], sw, nullptr, S[k].corr));
      if (S[k].in_flight) wide.push_back(k);
    } else {
      RTE_TRY(si_launch(S[k], st[k], nullptr));
    }
    return RTE_OK;
  };
  for (int k = 0; k < n; ++k) {
    rte_batch_t bt = batches[k];
    rte_rom_t rom = roms ? roms[k] : nullptr;
    st[k] = streams ? (cudaStream_t)streams[k] : nullptr;
    RTE_TRY(S[k].init(bt, opts[k], rom, rho[k]));
    if (!S[k].started) RTE_CUDA_TRY(cudaEventCreateWithFlags(&S[k].started, cudaEventDisableTiming));
    if (!S[k].corr) RTE_CUDA_TRY(cudaEventCreateWithFlags(&S[k].corr, cudaEventDisableTiming));
    RTE_CUDA_TRY(cudaMemcpyAsync(bt->work.p, rho[k], sizeof(double) * bt->B * bt->disc->n_dof,
                                 cudaMemcpyDeviceToDevice, st[k]));
    for (int b = 0; b < bt->B; ++b) S[k].begin(b, opts[k].eps);
    if (rom) RTE_TRY(rom_prepare(rom, bt, st[k]));
    RTE_TRY(launch(k));
  }
  int running = n;
  while (running > 0) {
    bool progress = false;
    running = 0;
    for (int k = 0; k < n; ++k) {
      if (!S[k].in_flight) continue;
      bool ready = false;
      RTE_TRY(event_ready(S[k].ev, &ready));
      if (ready) {
        // the wide sweep that runs next on sw -- the one queued after k's, or the oldest one when
        // k swept on its own stream (sw runs in order, so the ones before k's have finished) --
        // is dispatched before these corrections are issued; it waits only for work already
        // issued, so this wait ends
        int next = -1;
        for (auto it = wide.begin(); it != wide.end(); ++it)
          if (*it == k) {
            it = wide.erase(it);
            if (it != wide.end()) next = *it;
            break;
          }
        if (next < 0 && !wide.empty() && wide.front() != k) next = wide.front();
        if (next >= 0) RTE_CUDA_TRY(cudaEventSynchronize(S[next].started));
        RTE_TRY(si_finish(S[k], st[k], nullptr));
        RTE_TRY(launch(k));
        progress = true;
      }
      running += S[k].in_flight;
    }
    if (!progress && running > 0) std::this_thread::yield();
  }
  return finish_many(S, st, opts, roms, reports);
}

extern "C" int rte_solve_many(int n, const rte_batch_t* batches, const rte_solve_opts* opts,
                              const rte_rom_t* roms, double* const* rho,
                              rte_solve_report* const* reports, void* const* streams) {
  RTE_TRY(check_many("rte_solve_many", n, batches, opts, roms, rho));
  DeviceGuard g(batches[0]->disc->device);
  std::vector<SiState> S(n);
  std::vector<cudaStream_t> st(n);
  for (int k = 0; k < n; ++k) {
    rte_batch_t bt = batches[k];
    rte_rom_t rom = roms ? roms[k] : nullptr;
    st[k] = streams ? (cudaStream_t)streams[k] : nullptr;
    RTE_TRY(S[k].init(bt, opts[k], rom, rho[k]));
    RTE_CUDA_TRY(cudaMemcpyAsync(bt->work.p, rho[k], sizeof(double) * bt->B * bt->disc->n_dof,
                                 cudaMemcpyDeviceToDevice, st[k]));
    for (int b = 0; b < bt->B; ++b) S[k].begin(b, opts[k].eps);
    if (rom) RTE_TRY(rom_prepare(rom, bt, st[k]));
    RTE_TRY(si_launch(S[k], st[k], nullptr));
  }
  // event-driven round robin: whichever batch has its norms back is decided and relaunched
  int running = n;
  while (running > 0) {
    bool progress = false;
    running = 0;
    for (int k = 0; k < n; ++k) {
      if (!S[k].in_flight) continue;
      bool ready = false;
      RTE_TRY(event_ready(S[k].ev, &ready));
      if (ready) {
        RTE_TRY(si_finish(S[k], st[k], nullptr));
        RTE_TRY(si_launch(S[k], st[k], nullptr));
        progress = true;
      }
      running += S[k].in_flight;
    }
    if (!progress && running > 0) std::this_thread::yield();
  }
  return finish_many(S, st, opts, roms, reports);
}

// rte_solve_many with every batch iterating in lockstep: at each iteration one sweep launch covers
// the running instances of all batches (sweep_launch_multi: a work queue over (batch, instance,
// direction group), longest first), so that instances of any size fill the GPU together; then each
// batch's stop test and corrections run on its own stream, and the next sweep waits for all of
// them.  FP64 sweeps (no precision variant) and 2D batches only.
extern "C" int rte_solve_lockstep(int n, const rte_batch_t* batches, const rte_solve_opts* opts,
                                  const rte_rom_t* roms, double* const* rho,
                                  rte_solve_report* const* reports, void* const* streams) {
  RTE_TRY(check_many("rte_solve_lockstep", n, batches, opts, roms, rho));
  for (int k = 0; k < n; ++k) {
    if (batches[k]->disc->dim != 2) return fail(RTE_EINVAL, "rte_solve_lockstep: 2D batches only");
    if (opts[k].fp32_switch > 0.0 || opts[k].refine_kappa > 0.0)
      return fail(RTE_EINVAL, "rte_solve_lockstep: FP64 sweeps only (no precision variant)");
  }
  DeviceGuard g(batches[0]->disc->device);
  std::vector<SiState> S(n);
  std::vector<cudaStream_t> st(n);
  std::vector<cudaEvent_t> done(n, nullptr);
  struct EvGuard {
    std::vector<cudaEvent_t>& e;
    ~EvGuard() {
      for (auto x : e)
        if (x) cudaEventDestroy(x);
    }
  } evg{done};
  for (int k = 0; k < n; ++k) {
    rte_batch_t bt = batches[k];
    rte_rom_t rom = roms ? roms[k] : nullptr;
    st[k] = streams ? (cudaStream_t)streams[k] : nullptr;
    RTE_CUDA_TRY(cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming));
    RTE_TRY(S[k].init(bt, opts[k], rom, rho[k]));
    RTE_CUDA_TRY(cudaMemcpyAsync(bt->work.p, rho[k], sizeof(double) * bt->B * bt->disc->n_dof,
                                 cudaMemcpyDeviceToDevice, st[k]));
    for (int b = 0; b < bt->B; ++b) S[k].begin(b, opts[k].eps);
    if (rom) RTE_TRY(rom_prepare(rom, bt, st[k]));
    RTE_CUDA_TRY(cudaEventRecord(done[k], st[k]));
  }
  // the sweeps run on the first batch's stream, after every batch's set-up and corrections
  cudaStream_t s0 = st[0];
  MultiSweepScratch ws;
  for (;;) {
    std::vector<int> run;
    for (int k = 0; k < n; ++k)
      if (S[k].n_active() > 0) run.push_back(k);
    if (run.empty()) break;
    std::vector<rte_batch_t> bts;
    std::vector<const double*> rin;
    std::vector<double*> rout;
    std::vector<const uint8_t*> act, hact;
    for (int k : run) {
      SiState& s = S[k];
      rte_batch_t bt = batches[k];
      const size_t nb = (size_t)bt->B * bt->disc->n_dof;
      RTE_CUDA_TRY(cudaStreamWaitEvent(s0, done[k], 0));
      for (int b = 0; b < s.B; ++b) {
        s.swept[b] = s.act[b];
        s.hm[b] = s.act[b];
      }
      RTE_CUDA_TRY(cudaMemcpyAsync(s.dm.p, s.hm, (size_t)s.B, cudaMemcpyHostToDevice, s0));
      bts.push_back(bt);
      rin.push_back(bt->work.p);
      rout.push_back(bt->work.p + nb);
      act.push_back(s.dm.p);
      hact.push_back(s.hm);
    }
    RTE_TRY(sweep_launch_multi(bts, rin, rout, act, hact, ws, s0));
    for (int k : run) {
      SiState& s = S[k];
      RTE_CUDA_TRY(cudaMemcpyAsync(s.hn, batches[k]->norms.p, sizeof(unsigned long long) * 2 * s.B,
                                   cudaMemcpyDeviceToHost, s0));
      RTE_CUDA_TRY(cudaEventRecord(s.ev, s0));
      s.in_flight = true;
    }
    for (int k : run) {
      RTE_TRY(si_finish(S[k], st[k], nullptr));
      RTE_CUDA_TRY(cudaEventRecord(done[k], st[k]));
    }
  }
  return finish_many(S, st, opts, roms, reports);
}
