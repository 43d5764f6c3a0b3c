// Source iteration with synthetic acceleration (paper Alg. 1) with the ROMSAD switch (Alg. 2).
//
// Every instance of a batch runs its own Alg. 1: sweep (fused scalar-flux reduction and stop-
// test norms), stop test, then the correction chosen for it -- DSA (App. B), ROMSA
// (Eq. (rom_correction)) or, for ROMSAD, ROMSA iff 1 <= l <= theta and the change is at least
// eps_ROMSAD.  Instances that have converged drop out of every later launch through a device
// mask.  The only host round trip per iteration is the 2*B stop-test norms.
#include "common.cuh"

namespace rte {
int rom_prepare(rte_rom_t rom, rte_batch_t bt, cudaStream_t st);
int rom_correction(rte_rom_t rom, rte_batch_t bt, const double* R, double* drho,
                   const uint8_t* active, cudaStream_t st);

int run_si(rte_batch_t bt, const rte_solve_opts* o, rte_rom_t rom_c, double* rho,
           rte_solve_report* reports, double* history, cudaStream_t st, double* psi_cur,
           double* psi_win, int window) {
  const rte_disc_s* d = bt->disc;
  const int B = bt->B;
  const size_t n = d->n_dof, nb = (size_t)B * n;
  double* rho_prev = bt->work.p;
  double* rho_star = bt->work.p + nb;
  double* R = bt->work.p + 2 * nb;
  double* drho = bt->work.p + 3 * nb;
  RTE_CUDA_TRY(cudaMemcpyAsync(rho_prev, rho, sizeof(double) * nb, cudaMemcpyDeviceToDevice, st));
  std::vector<uint8_t> act(B, 1), use_rom(B, 0), use_dsa(B, 0);
  // precision variant: instances start with FP32 sweeps and switch to FP64 below fp32_switch
  const bool mixed = o->fp32_switch > 0.0 && d->dim == 2 && psi_cur == nullptr;
  std::vector<uint8_t> lowp(B, mixed ? 1 : 0), act_lo(B, 0), act_hi(B, 0);
  DevBuf<uint8_t> act_dev, rom_dev, dsa_dev, lo_dev, hi_dev;
  RTE_TRY(act_dev.alloc(B));
  RTE_TRY(lo_dev.alloc(B));
  RTE_TRY(hi_dev.alloc(B));
  RTE_TRY(rom_dev.alloc(B));
  RTE_TRY(dsa_dev.alloc(B));
  std::vector<rte_solve_report> rep(B);
  for (auto& r : rep) r = rte_solve_report{0, 0, 0, 0, 0, 0.0, 0.0, 0};
  if ((o->sa == RTE_SA_ROMSA || o->sa == RTE_SA_ROMSAD) && !rom_c)
    return fail(RTE_EINVAL, "ROMSA/ROMSAD need a correction ROM");
  if (rom_c) {
    PhaseScope ps(bt, 2, st);
    RTE_TRY(rom_prepare(rom_c, bt, st));
  }
  std::vector<double> norms(2 * B);
  std::vector<int> iters(B);
  int status = RTE_OK;
  const size_t psi_per = (size_t)d->n_dirs * n;
  for (int l = 1; l <= o->max_iter; ++l) {
    RTE_CUDA_TRY(cudaMemcpyAsync(act_dev.p, act.data(), B, cudaMemcpyHostToDevice, st));
    double* psi = psi_cur;
    int n_lo = 0, n_hi = 0;
    for (int b = 0; b < B; ++b) {
      act_lo[b] = act[b] && lowp[b];
      act_hi[b] = act[b] && !lowp[b];
      n_lo += act_lo[b], n_hi += act_hi[b];
    }
    if (n_lo == 0) {
      RTE_TRY(sweep_launch(bt, rho_prev, rho_star, psi, 1, act_dev.p, st, true, n_hi));
    } else {
      RTE_CUDA_TRY(cudaMemsetAsync(bt->norms.p, 0, sizeof(unsigned long long) * 2 * B, st));
      RTE_CUDA_TRY(cudaMemcpyAsync(lo_dev.p, act_lo.data(), B, cudaMemcpyHostToDevice, st));
      RTE_TRY(sweep_launch_f32(bt, rho_prev, rho_star, lo_dev.p, st, n_lo, false));
      if (n_hi > 0) {
        RTE_CUDA_TRY(cudaMemcpyAsync(hi_dev.p, act_hi.data(), B, cudaMemcpyHostToDevice, st));
        RTE_TRY(sweep_launch(bt, rho_prev, rho_star, psi, 1, hi_dev.p, st, true, n_hi, false));
      }
    }
    if (psi_win && l <= window)
      for (int b = 0; b < B; ++b)
        if (act[b])
          RTE_CUDA_TRY(cudaMemcpyAsync(psi_win + ((size_t)(l - 1) * B + b) * psi_per,
                                       psi_cur + (size_t)b * psi_per, sizeof(double) * psi_per,
                                       cudaMemcpyDeviceToDevice, st));
    RTE_TRY(norms_to_host(bt, norms.data(), st));
    bool any = false;
    for (int b = 0; b < B; ++b) {
      use_rom[b] = use_dsa[b] = 0;
      if (!act[b]) continue;
      const double delta = norms[2 * b], rinf = norms[2 * b + 1];
      if (history) history[(size_t)b * o->max_iter + (l - 1)] = delta;
      rep[b].n_sweep = l;
      rep[b].last_change = delta;
      rep[b].rho_inf = rinf;
      const double test = o->rel ? delta / rinf : delta;
      if (lowp[b]) {
        rep[b].n_sweep32++;
        if (test < o->fp32_switch) lowp[b] = 0;  // later sweeps of this instance in FP64
      } else if (test < o->eps) {
        rep[b].converged = 1;
        act[b] = 0;
        RTE_CUDA_TRY(cudaMemcpyAsync(rho + (size_t)b * n, rho_star + (size_t)b * n,
                                     sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        continue;
      }
      any = true;
      bool romsa = o->sa == RTE_SA_ROMSA;
      if (o->sa == RTE_SA_ROMSAD)
        romsa = o->schedule ? o->schedule[l - 1] != 0 : (l <= o->theta && delta >= o->eps_romsad);
      if (o->sa == RTE_SA_NONE) continue;
      if (romsa) use_rom[b] = 1, rep[b].n_romsa++;
      else use_dsa[b] = 1, rep[b].n_dsa++;
    }
    if (!any) break;
    RTE_CUDA_TRY(cudaMemcpyAsync(act_dev.p, act.data(), B, cudaMemcpyHostToDevice, st));
    if (o->sa == RTE_SA_NONE) {
      // plain SI: rho^(l) = rho^(l,*)
      std::swap(rho_prev, rho_star);
      continue;
    }
    RTE_TRY(correction_source_launch(bt, rho_star, rho_prev, R, act_dev.p, st));
    bool anyd = false, anyr = false;
    for (int b = 0; b < B; ++b) anyd |= use_dsa[b] != 0, anyr |= use_rom[b] != 0;
    if (anyd) {
      RTE_CUDA_TRY(cudaMemcpyAsync(dsa_dev.p, use_dsa.data(), B, cudaMemcpyHostToDevice, st));
      PhaseScope ps(bt, 1, st);
      int s = dsa_apply(bt, R, drho, o->dsa_rtol, o->dsa_max_it, dsa_dev.p, iters.data(), st);
      if (s != RTE_OK && s != RTE_ENOCONV) return s;
      for (int b = 0; b < B; ++b)
        if (use_dsa[b]) rep[b].dsa_iters += iters[b];
    }
    if (anyr) {
      RTE_CUDA_TRY(cudaMemcpyAsync(rom_dev.p, use_rom.data(), B, cudaMemcpyHostToDevice, st));
      PhaseScope ps(bt, 2, st);
      RTE_TRY(rom_correction(rom_c, bt, R, drho, rom_dev.p, st));
    }
    // rho^(l) = rho^(l,*) + delta rho^(l), written into the rho_prev slot
    RTE_TRY(axpy_launch(bt, rho_star, drho, rho_prev, act_dev.p, st));
  }
  for (int b = 0; b < B; ++b)
    if (act[b]) {
      status = RTE_ENOCONV;
      RTE_CUDA_TRY(cudaMemcpyAsync(rho + (size_t)b * n, rho_prev + (size_t)b * n,
                                   sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    }
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  if (reports)
    for (int b = 0; b < B; ++b) reports[b] = rep[b];
  return status;
}

}  // namespace rte

using namespace rte;

extern "C" int rte_solve(rte_batch_t b, const rte_solve_opts* o, rte_rom_t rom_c, double* rho,
                         rte_solve_report* reports, double* history, void* stream) {
  if (!b || !o || !rho) return fail(RTE_EINVAL, "rte_solve: null argument");
  if (!b->params_set) return fail(RTE_ESTATE, "rte_solve: parameters not set");
  if (!(o->eps >= 0) || o->max_iter < 1 || o->sa < 0 || o->sa > 3 || !(o->fp32_switch >= 0))
    return fail(RTE_EINVAL, "rte_solve: bad options");
  if (o->sa != RTE_SA_NONE && b->disc->dim == 2 && (!(o->dsa_rtol >= 0) || o->dsa_max_it < 1))
    return fail(RTE_EINVAL, "rte_solve: bad DSA tolerance");
  if (rom_c && rom_c->disc != b->disc) return fail(RTE_EINVAL, "ROM built on another discretisation");
  DeviceGuard g(b->disc->device);
  return run_si(b, o, rom_c, rho, reports, history, (cudaStream_t)stream, nullptr, nullptr, 0);
}
