// DSA-preconditioned restarted GMRES for (I - L) rho = b-bar (paper Sec. 2.3; App. A): the
// paper's second comparison system, for a batch of instances.
//
// Left preconditioner M^{-1} = I + C Sigma_s, where C Sigma_s v is the DSA correction for the
// source Sigma_s v (the same correction Alg. 1 applies; with it one SI-DSA step is a Richardson
// step on the preconditioned system).  Each instance runs its own GMRES(m): Arnoldi on
// w = M^{-1} (I - L) v, Givens rotations on the host for the preconditioned residual, x = x0 + V y
// when that estimate relative to ||M^{-1} b-bar|| is below rtol or after m steps; then the residual
// is recomputed from x and decides convergence (or starts the next cycle).  All instances
// advance in lockstep, one Arnoldi step per launch sequence; finished instances drop out through a
// device mask.  Orthogonalisation is classical Gram-Schmidt applied twice (two batched dot
// launches instead of i+1 dependent ones), which gives modified Gram-Schmidt's orthogonality.
// Host round trip: one per Arnoldi step (the new Hessenberg column and norm of every instance).
// Sweep accounting as in the paper: one sweep for b-bar, one per operator application, one per
// recomputed residual (end of every cycle, and the start when it is not zero).
#include "common.cuh"

namespace rte {

// w = v - Lv (or v when Lv is null); R = Sigma_s w.  With 1D cross sections linear across cells
// (matr non-null, P = 2) a thread takes one cell and applies the 2x2 of linear_sigma; both moments
// are read before either is written, so w may alias v.
__global__ void amv_kernel(const double* v, const double* Lv, double* w, double* R,
                           const double* sigma_s, const int32_t* mat, const int32_t* matr,
                           const uint8_t* active, int n_dof, int P, int n_mat) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  if (matr) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_dof / 2; c += gridDim.x * blockDim.x) {
      const size_t o = (size_t)b * n_dof + 2 * c;
      const double t0 = Lv ? v[o] - Lv[o] : v[o], t1 = Lv ? v[o + 1] - Lv[o + 1] : v[o + 1];
      double sb, so;
      linear_sigma(sigma_s[(size_t)b * n_mat + mat[c]], sigma_s[(size_t)b * n_mat + matr[c]], sb, so);
      w[o] = t0;
      w[o + 1] = t1;
      R[o] = fma(sb, t0, so * t1);
      R[o + 1] = fma(so, t0, sb * t1);
    }
    return;
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_dof; e += gridDim.x * blockDim.x) {
    const size_t o = (size_t)b * n_dof + e;
    const double t = Lv ? v[o] - Lv[o] : v[o];
    w[o] = t;
    R[o] = sigma_s[(size_t)b * n_mat + mat[e / P]] * t;
  }
}

// d = bbar - x + Lx  (the residual b-bar - (I - L) x)
__global__ void resid_kernel(const double* bbar, const double* x, const double* Lx, double* d,
                             const uint8_t* active, int n_dof) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_dof; e += gridDim.x * blockDim.x) {
    const size_t o = (size_t)b * n_dof + e;
    d[o] = bbar[o] - x[o] + Lx[o];
  }
}

// out[b][j] = <w_b, V_j,b> for j < nvec; one block per (j, b), fixed-order tree reduction
__global__ void kdots_kernel(const double* w, const double* V, size_t vstride, double* out,
                             int ldo, const uint8_t* active, int n_dof) {
  const int j = blockIdx.x, b = blockIdx.y;
  if (active && !active[b]) return;
  __shared__ double sh[256];
  const double* wb = w + (size_t)b * n_dof;
  const double* vb = V + (size_t)j * vstride + (size_t)b * n_dof;
  double s = 0.0;
  for (int e = threadIdx.x; e < n_dof; e += blockDim.x) s = fma(wb[e], vb[e], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(size_t)b * ldo + j] = sh[0];
}

// w_b -= sum_{j < nvec} h[b][j] V_j,b
__global__ void kupdate_kernel(double* w, const double* V, size_t vstride, int nvec,
                               const double* h, int ldh, const uint8_t* active, int n_dof) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_dof; e += gridDim.x * blockDim.x) {
    const size_t o = (size_t)b * n_dof + e;
    double s = w[o];
    for (int j = 0; j < nvec; ++j) s = fma(-h[(size_t)b * ldh + j], V[(size_t)j * vstride + o], s);
    w[o] = s;
  }
}

// out_b = c[b] w_b
__global__ void kscale_kernel(const double* w, double* out, const double* c, const uint8_t* active,
                              int n_dof) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const double s = c[b];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_dof; e += gridDim.x * blockDim.x) {
    const size_t o = (size_t)b * n_dof + e;
    out[o] = s * w[o];
  }
}

// x_b += sum_{j < k} y[b][j] V_j,b
__global__ void kcombine_kernel(double* x, const double* V, size_t vstride, int k, const double* y,
                                int ldy, const uint8_t* active, int n_dof) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_dof; e += gridDim.x * blockDim.x) {
    const size_t o = (size_t)b * n_dof + e;
    double s = x[o];
    for (int j = 0; j < k; ++j) s = fma(y[(size_t)b * ldy + j], V[(size_t)j * vstride + o], s);
    x[o] = s;
  }
}

namespace {

struct Gmres {
  rte_batch_t bt;
  const rte_gmres_opts* o;
  cudaStream_t st;
  int B, n, m, P, n_mat;
  dim3 grid;
  DevBuf<double> V, w, scal, coef;     // V: [m+1][B][n]; scal: [B][2(m+1) + 2]; coef: [B][m+1]
  DevBuf<uint8_t> mask;                // [2][B]: step mask, combine mask
  double* hs = nullptr;                // pinned [B][2(m+1) + 2]
  uint8_t* hm = nullptr;               // pinned [2][B]
  double* hy = nullptr;                // pinned [B][m+1] (y), then [B] scale factors
  std::vector<int> dsa_iters;
  // a pinned region is rewritten only after the copy that last read it has run
  cudaEvent_t ev_mask[2] = {nullptr, nullptr}, ev_y = nullptr;
  ~Gmres() {
    if (hs) cudaFreeHost(hs);
    if (hm) cudaFreeHost(hm);
    if (hy) cudaFreeHost(hy);
    for (auto e : {ev_mask[0], ev_mask[1], ev_y})
      if (e) cudaEventDestroy(e);
  }
  int init_events() {
    for (auto* e : {&ev_mask[0], &ev_mask[1], &ev_y}) {
      RTE_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
      RTE_CUDA_TRY(cudaEventRecord(*e, st));
    }
    return RTE_OK;
  }
  // host y / scale factors -> coef (count doubles); call wait_y() before writing hy
  int wait_y() {
    RTE_CUDA_TRY(cudaEventSynchronize(ev_y));
    return RTE_OK;
  }
  int upload_y(size_t count) {
    RTE_CUDA_TRY(cudaMemcpyAsync(coef.p, hy, sizeof(double) * count, cudaMemcpyHostToDevice, st));
    RTE_CUDA_TRY(cudaEventRecord(ev_y, st));
    return RTE_OK;
  }
  size_t ld() const { return 2 * (size_t)(m + 1) + 2; }
  double* bbar() const { return bt->work.p; }
  double* lx() const { return bt->work.p + (size_t)B * n; }
  double* R() const { return bt->work.p + 2 * (size_t)B * n; }
  double* drho() const { return bt->work.p + 3 * (size_t)B * n; }
  double* Vj(int j) const { return V.p + (size_t)j * B * n; }

  int upload_mask(int which, const std::vector<uint8_t>& act) {
    RTE_CUDA_TRY(cudaEventSynchronize(ev_mask[which]));
    std::memcpy(hm + (size_t)which * B, act.data(), B);
    RTE_CUDA_TRY(cudaMemcpyAsync(mask.p + (size_t)which * B, hm + (size_t)which * B, B,
                                 cudaMemcpyHostToDevice, st));
    RTE_CUDA_TRY(cudaEventRecord(ev_mask[which], st));
    return RTE_OK;
  }
  // out = M^{-1} in  (in may equal out)
  int apply_minv(const double* in, double* out, const uint8_t* act) {
    amv_kernel<<<grid, 256, 0, st>>>(in, nullptr, out, R(), bt->sigma_s.p, bt->disc->mat_id.p,
                                     bt->disc->mat_r.p, act,
                                     n, P, n_mat); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
    if (o->precond) {
      PhaseScope ps(bt, 1, st);
      int e = dsa_apply(bt, R(), drho(), o->dsa_rtol, o->dsa_max_it, act, dsa_iters.data(), st);
      if (e != RTE_OK && e != RTE_ENOCONV) return e;
      RTE_TRY(axpy_launch(bt, out, drho(), out, act, st));
    }
    return RTE_OK;
  }
  // norms ||v_b|| into host hs[b*ld + slot]
  int norms(const double* v, int slot, const uint8_t* act) {
    kdots_kernel<<<dim3(1, B), 256, 0, st>>>(v, v, 0, scal.p + slot, (int)ld(), act, n); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
  }
};

}  // namespace

static int run_pgmres(rte_batch_t bt, const rte_gmres_opts* o, double* x,
                      rte_solve_report* reports, cudaStream_t st) {
  const rte_disc_s* d = bt->disc;
  Gmres G;
  G.bt = bt, G.o = o, G.st = st;
  G.B = bt->B, G.n = d->n_dof, G.m = o->restart, G.P = d->P, G.n_mat = d->n_mat;
  const int B = G.B, n = G.n, m = G.m;
  const size_t ld = G.ld(), vstride = (size_t)B * n;
  G.grid = dim3(std::min((n + 255) / 256, 1024), B);
  RTE_TRY(G.V.alloc((size_t)(m + 1) * B * n));
  RTE_TRY(G.w.alloc((size_t)B * n));
  RTE_TRY(G.scal.alloc((size_t)B * ld));
  RTE_TRY(G.coef.alloc((size_t)B * (m + 1)));
  // unused basis columns enter x = x0 + V y with y = 0: keep them finite
  RTE_CUDA_TRY(cudaMemsetAsync(G.V.p, 0, sizeof(double) * G.V.n, st));
  RTE_TRY(G.mask.alloc(2 * (size_t)B));
  RTE_CUDA_TRY(cudaHostAlloc((void**)&G.hs, sizeof(double) * B * ld, cudaHostAllocDefault));
  RTE_CUDA_TRY(cudaHostAlloc((void**)&G.hm, 2 * (size_t)B, cudaHostAllocDefault));
  RTE_CUDA_TRY(cudaHostAlloc((void**)&G.hy, sizeof(double) * B * (m + 1), cudaHostAllocDefault));
  RTE_TRY(G.init_events());
  G.dsa_iters.assign(B, 0);
  std::vector<rte_solve_report> rep(B, rte_solve_report{});
  std::vector<uint8_t> act(B, 1);
  RTE_TRY(G.upload_mask(0, act));
  const uint8_t* m0 = G.mask.p;
  auto count_precond = [&](const std::vector<uint8_t>& a) {
    for (int b = 0; b < B; ++b)
      if (a[b] && o->precond) rep[b].n_dsa++, rep[b].dsa_iters += G.dsa_iters[b];
  };
  auto pull = [&]() -> int {
    RTE_CUDA_TRY(cudaMemcpyAsync(G.hs, G.scal.p, sizeof(double) * B * ld, cudaMemcpyDeviceToHost, st));
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    return RTE_OK;
  };
  // b-bar = L 0 + b (one sweep); x0 = 0 unless the caller supplied a start
  RTE_CUDA_TRY(cudaMemsetAsync(G.w.p, 0, sizeof(double) * vstride, st));
  RTE_TRY(sweep_launch(bt, G.w.p, G.bbar(), nullptr, 1, m0, st, false, B));
  for (auto& r : rep) r.n_sweep = 1;
  // reference ||M^{-1} b-bar|| and the first residual r = M^{-1}(b-bar - A x0) in V_0
  RTE_TRY(G.apply_minv(G.bbar(), G.Vj(0), m0));
  count_precond(act);
  RTE_TRY(G.norms(G.Vj(0), (int)ld - 2, m0));
  RTE_TRY(pull());
  std::vector<double> ref(B);
  for (int b = 0; b < B; ++b) ref[b] = std::sqrt(std::max(G.hs[b * ld + ld - 2], 0.0));
  // residual of the current x into V_0 for the instances in `a` (one sweep each)
  auto residual = [&](const std::vector<uint8_t>& a) -> int {
    RTE_TRY(G.upload_mask(0, a));
    int na = 0;
    for (int b = 0; b < B; ++b) na += a[b];
    RTE_TRY(sweep_launch(bt, x, G.lx(), nullptr, 0, m0, st, false, na));
    resid_kernel<<<G.grid, 256, 0, st>>>(G.bbar(), x, G.lx(), G.Vj(0), m0, n); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
    RTE_TRY(G.apply_minv(G.Vj(0), G.Vj(0), m0));
    count_precond(a);
    for (int b = 0; b < B; ++b)
      if (a[b]) rep[b].n_sweep++;
    return RTE_OK;
  };
  if (o->zero_start) {
    RTE_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * vstride, st));
  } else {
    RTE_TRY(residual(act));
  }
  std::vector<double> H((size_t)B * (m + 1) * m), g((size_t)B * (m + 1)), cs((size_t)B * m),
      sn((size_t)B * m);
  std::vector<int> kb(B, 0), steps(B, 0);
  std::vector<uint8_t> cyc(B, 0);
  int status = RTE_OK;
  while (true) {
    // beta = ||r||: converged instances stop; the others start a cycle from V_0 = r / beta
    RTE_TRY(G.upload_mask(0, act));
    RTE_TRY(G.norms(G.Vj(0), (int)ld - 1, m0));
    RTE_TRY(pull());
    bool any = false;
    RTE_TRY(G.wait_y());
    for (int b = 0; b < B; ++b) {
      if (!act[b]) continue;
      const double beta = std::sqrt(std::max(G.hs[b * ld + ld - 1], 0.0));
      rep[b].last_change = ref[b] > 0 ? beta / ref[b] : 0.0;
      if (ref[b] == 0.0 || beta <= o->rtol * ref[b]) {
        act[b] = 0, rep[b].converged = 1;
        continue;
      }
      if (steps[b] >= o->max_iter) {
        act[b] = 0, status = RTE_ENOCONV;
        continue;
      }
      any = true;
      std::fill(&g[(size_t)b * (m + 1)], &g[(size_t)b * (m + 1)] + m + 1, 0.0);
      g[(size_t)b * (m + 1)] = beta;
      G.hy[b] = 1.0 / beta;
    }
    if (!any) break;
    RTE_TRY(G.upload_mask(0, act));
    RTE_TRY(G.upload_y(B));
    kscale_kernel<<<G.grid, 256, 0, st>>>(G.Vj(0), G.Vj(0), G.coef.p, m0, n); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
    cyc = act;
    std::fill(kb.begin(), kb.end(), 0);
    for (int i = 0; i < m; ++i) {
      int na = 0;
      for (int b = 0; b < B; ++b) na += cyc[b];
      if (na == 0) break;
      RTE_TRY(G.upload_mask(0, cyc));
      // w = M^{-1} (I - L) V_i
      RTE_TRY(sweep_launch(bt, G.Vj(i), G.lx(), nullptr, 0, m0, st, false, na));
      amv_kernel<<<G.grid, 256, 0, st>>>(G.Vj(i), G.lx(), G.w.p, G.R(), bt->sigma_s.p, d->mat_id.p,
                                         d->mat_r.p, m0, n, G.P, G.n_mat); RTE_NOTE_LAUNCH();
      RTE_CUDA_TRY(cudaGetLastError());
      if (o->precond) {
        PhaseScope ps(bt, 1, st);
        int e = dsa_apply(bt, G.R(), G.drho(), o->dsa_rtol, o->dsa_max_it, m0, G.dsa_iters.data(), st);
        if (e != RTE_OK && e != RTE_ENOCONV) return e;
        RTE_TRY(axpy_launch(bt, G.w.p, G.drho(), G.w.p, m0, st));
      }
      count_precond(cyc);
      // classical Gram-Schmidt twice; coefficients of both passes land in scal[b][0..2(i+1))
      for (int pass = 0; pass < 2; ++pass) {
        double* h = G.scal.p + (size_t)pass * (m + 1);
        kdots_kernel<<<dim3(i + 1, B), 256, 0, st>>>(G.w.p, G.V.p, vstride, h, (int)ld, m0, n); RTE_NOTE_LAUNCH();
        kupdate_kernel<<<G.grid, 256, 0, st>>>(G.w.p, G.V.p, vstride, i + 1, h, (int)ld, m0, n); RTE_NOTE_LAUNCH();
        RTE_CUDA_TRY(cudaGetLastError());
      }
      RTE_TRY(G.norms(G.w.p, (int)ld - 1, m0));
      RTE_TRY(pull());
      RTE_TRY(G.wait_y());
      bool cont = false;
      for (int b = 0; b < B; ++b) {
        if (!cyc[b]) continue;
        rep[b].n_sweep++;
        steps[b]++;
        double* Hb = &H[(size_t)b * (m + 1) * m];
        double* gb = &g[(size_t)b * (m + 1)];
        double* cb = &cs[(size_t)b * m];
        double* sb = &sn[(size_t)b * m];
        const double* hb = &G.hs[b * ld];
        for (int j = 0; j <= i; ++j) Hb[j * m + i] = hb[j] + hb[(m + 1) + j];
        const double hn = std::sqrt(std::max(hb[ld - 1], 0.0));
        Hb[(i + 1) * m + i] = hn;
        for (int j = 0; j < i; ++j) {
          const double t = cb[j] * Hb[j * m + i] + sb[j] * Hb[(j + 1) * m + i];
          Hb[(j + 1) * m + i] = -sb[j] * Hb[j * m + i] + cb[j] * Hb[(j + 1) * m + i];
          Hb[j * m + i] = t;
        }
        const double dd = std::hypot(Hb[i * m + i], Hb[(i + 1) * m + i]);
        cb[i] = dd > 0 ? Hb[i * m + i] / dd : 1.0;
        sb[i] = dd > 0 ? Hb[(i + 1) * m + i] / dd : 0.0;
        Hb[i * m + i] = dd;
        Hb[(i + 1) * m + i] = 0.0;
        gb[i + 1] = -sb[i] * gb[i];
        gb[i] = cb[i] * gb[i];
        kb[b] = i + 1;
        rep[b].last_change = std::fabs(gb[i + 1]) / ref[b];
        const bool fin = std::fabs(gb[i + 1]) <= o->rtol * ref[b] || hn == 0.0 ||
                         steps[b] >= o->max_iter;
        if (fin) {
          cyc[b] = 0;
        } else {
          G.hy[b] = 1.0 / hn;
          cont = true;
        }
      }
      if (!cont || i + 1 == m) break;
      // V_{i+1} = w / h_{i+1,i} for the instances that continue
      RTE_TRY(G.upload_mask(1, cyc));
      RTE_TRY(G.upload_y(B));
      kscale_kernel<<<G.grid, 256, 0, st>>>(G.w.p, G.Vj(i + 1), G.coef.p, G.mask.p + B, n); RTE_NOTE_LAUNCH();
      RTE_CUDA_TRY(cudaGetLastError());
    }
    // x += V y with H y = g (back substitution per instance)
    RTE_TRY(G.wait_y());
    for (int b = 0; b < B; ++b) {
      double* yb = G.hy + (size_t)b * (m + 1);
      if (!act[b]) continue;
      const int k = kb[b];
      const double* Hb = &H[(size_t)b * (m + 1) * m];
      const double* gb = &g[(size_t)b * (m + 1)];
      for (int r = k - 1; r >= 0; --r) {
        double s = gb[r];
        for (int c = r + 1; c < k; ++c) s -= Hb[r * m + c] * yb[c];
        yb[r] = s / Hb[r * m + r];
      }
      for (int r = k; r <= m; ++r) yb[r] = 0.0;
    }
    RTE_TRY(G.upload_mask(1, act));
    RTE_TRY(G.upload_y((size_t)B * (m + 1)));
    kcombine_kernel<<<G.grid, 256, 0, st>>>(x, G.V.p, vstride, m, G.coef.p, m + 1, G.mask.p + B, n); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
    // the residual of the updated x, recomputed (one sweep): the next pass of the loop decides
    // convergence on it and otherwise starts a new cycle from it (App. A recomputes it after
    // every update; with an inexactly applied M^{-1} the Arnoldi estimate drifts from it)
    RTE_TRY(residual(act));
  }
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  for (int b = 0; b < B; ++b) {
    if (!rep[b].converged) status = RTE_ENOCONV;
    if (reports) reports[b] = rep[b];
  }
  return status;
}

}  // namespace rte

using namespace rte;

extern "C" int rte_pgmres(rte_batch_t b, const rte_gmres_opts* o, double* rho,
                          rte_solve_report* reports, void* stream) {
  if (!b || !o || !rho) return fail(RTE_EINVAL, "rte_pgmres: null argument");
  RTE_TRY(params_ready(b, "rte_pgmres"));
  if (!(o->rtol > 0) || o->restart < 1 || o->restart > 200 || o->max_iter < 1 ||
      (o->precond != 0 && o->precond != 1))
    return fail(RTE_EINVAL, "rte_pgmres: bad options");
  if (o->precond && b->disc->dim == 2 && (!(o->dsa_rtol >= 0) || o->dsa_max_it < 1))
    return fail(RTE_EINVAL, "rte_pgmres: bad DSA tolerance");
  DeviceGuard g(b->disc->device);
  return run_pgmres(b, o, rho, reports, (cudaStream_t)stream);
}
