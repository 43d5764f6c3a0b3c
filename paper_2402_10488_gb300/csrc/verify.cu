// Checks of a computed solution, in FP64 on the device: the residual of the discrete fixed-point
// problem and the particle balance.
//
// Residual (paper Sec. 2.3.1, Eq. (rho_matrix_vec)): rho solves (I - L) rho = b-bar exactly when
// one more sweep returns it unchanged, since sweep(rho) = L rho + b-bar (Eq. (rho_matrix_vec_def)).
// So ||(I - L) rho - b-bar||_inf = ||rho - sweep(rho)||_inf, the quantity the paper averages over
// its test set as R^rho_inf (the notation table of Sec. 4), costs one sweep.
//
// Particle balance: testing the upwind DG equation of one direction (Eq. (DG)) with the indicator
// function of a cell T, whose gradient vanishes, leaves
//     int_{dT} (v.n) f_hat + int_T sigma_t f = int_T (sigma_s rho_prev + G)   (+ inflow through f_hat),
// and the omega-weighted sum over directions gives, per cell, for the sweep rho* = sweep(rho_prev),
//     bal_T = net outflow_T + int_T sigma_t rho* - int_T sigma_s rho_prev - int_T G = 0.
// The sweep kernel records the net outflow from the face traces it passes between cells (the
// upwind values f_hat), so bal_T checks every cell solve against its own traces.  Summed over the
// cells, the interior faces cancel and
//     leakage + int sigma_a rho* - int G = - int sigma_s (rho* - rho_prev) + sum_T bal_T,
// the global balance (absorption + net leakage = source) that holds at the converged solution.
#include "common.cuh"

namespace rte {

namespace {
constexpr int kVerifyThreads = 256;

// One block per instance.  out[b] = (||rho - rho*||_inf, max_T |bal_T|, global balance defect
// leakage + int sigma_a rho* - int G, int G).  Each thread takes cells t, t + 256, ...; the sums are
// then combined in a fixed tree order, so the result does not depend on scheduling.
__global__ void __launch_bounds__(kVerifyThreads)
residual_balance_kernel(const double* __restrict__ rho, const double* __restrict__ rho_star,
                        const double* __restrict__ leak, int n_groups,
                        const double* __restrict__ sigma_t, const double* __restrict__ sigma_s,
                        const double* __restrict__ G0, const int32_t* __restrict__ mat,
                        const int32_t* __restrict__ matr, const double* __restrict__ dx,
                        double sq_area, const uint8_t* active, int n_cells, int P, int n_mat,
                        double* out, double* cell_balance) {
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  int rank = b;
  if (active) {   // leak partials are indexed by the rank among the swept instances
    rank = 0;
    for (int i = 0; i < b; ++i) rank += active[i] != 0;
  }
  const size_t n_dof = (size_t)n_cells * P;
  const double* r = rho + (size_t)b * n_dof;
  const double* rs = rho_star + (size_t)b * n_dof;
  const double* lk = leak + (size_t)rank * n_groups * n_cells;
  const double* st = sigma_t + (size_t)b * n_mat;
  const double* ss = sigma_s + (size_t)b * n_mat;
  double rmax = 0.0, bmax = 0.0, gsum = 0.0, src = 0.0;
  for (int c = threadIdx.x; c < n_cells; c += kVerifyThreads) {
    for (int k = 0; k < P; ++k) rmax = fmax(rmax, fabs(r[(size_t)c * P + k] - rs[(size_t)c * P + k]));
    double out_c = 0.0;
    for (int g = 0; g < n_groups; ++g) out_c += lk[(size_t)g * n_cells + c];
    const double sq = dx ? sqrt(dx[c]) : sq_area;   // int_T u = sqrt|T| u_0 (orthonormal basis)
    const double g0 = G0[(size_t)b * n_cells + c];   // int_T G phi_0 = G sqrt|T|
    const double u0 = rs[(size_t)c * P], p0 = r[(size_t)c * P];
    double tot, sca, sca_star;   // int sigma_t rho*, int sigma_s rho_prev, int sigma_s rho* (over sqrt|T|)
    if (matr) {   // 1D, cross sections linear across the cell: [[mean, off], [off, mean]]
      double tm, to, sm, so;
      linear_sigma(st[mat[c]], st[matr[c]], tm, to);
      linear_sigma(ss[mat[c]], ss[matr[c]], sm, so);
      const double u1 = rs[(size_t)c * P + 1], p1 = r[(size_t)c * P + 1];
      tot = fma(tm, u0, to * u1);
      sca = fma(sm, p0, so * p1);
      sca_star = fma(sm, u0, so * u1);
    } else {
      const double t = st[mat[c]], s = ss[mat[c]];
      tot = t * u0;
      sca = s * p0;
      sca_star = s * u0;
    }
    const double bal = out_c + sq * (tot - sca - g0);
    if (cell_balance) cell_balance[(size_t)b * n_cells + c] = bal;
    bmax = fmax(bmax, fabs(bal));
    gsum += out_c + sq * (tot - sca_star - g0);
    src += sq * g0;
  }
  __shared__ double s_r[kVerifyThreads], s_b[kVerifyThreads], s_g[kVerifyThreads], s_s[kVerifyThreads];
  const int t = threadIdx.x;
  s_r[t] = rmax, s_b[t] = bmax, s_g[t] = gsum, s_s[t] = src;
  __syncthreads();
  for (int h = kVerifyThreads / 2; h > 0; h >>= 1) {
    if (t < h) {
      s_r[t] = fmax(s_r[t], s_r[t + h]);
      s_b[t] = fmax(s_b[t], s_b[t + h]);
      s_g[t] += s_g[t + h];
      s_s[t] += s_s[t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
    out[4 * (size_t)b] = s_r[0];
    out[4 * (size_t)b + 1] = s_b[0];
    out[4 * (size_t)b + 2] = s_g[0];
    out[4 * (size_t)b + 3] = s_s[0];
  }
}
}  // namespace

int residual_launch(rte_batch_t bt, const double* rho, double* out, double* cell_balance,
                    const uint8_t* active, cudaStream_t st) {
  const rte_disc_s* d = bt->disc;
  const size_t nb = (size_t)bt->B * d->n_dof;
  double* rho_star = bt->work.p + 2 * nb;   // iteration scratch (the correction source slot)
  int n_groups = 0;
  RTE_TRY(sweep_launch_leak(bt, rho, rho_star, active, st, &n_groups));
  residual_balance_kernel<<<bt->B, kVerifyThreads, 0, st>>>(
      rho, rho_star, bt->leak.p, n_groups, bt->sigma_t.p, bt->sigma_s.p, bt->G0.p, d->mat_id.p,
      d->dim == 1 ? d->mat_r.p : nullptr, d->dim == 1 ? d->dx_dev.p : nullptr,
      std::sqrt(d->hx * d->hy), active, d->n_cells, d->P, d->n_mat, out, cell_balance); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

}  // namespace rte

using namespace rte;

extern "C" int rte_residual(rte_batch_t b, const double* rho, double* out, double* cell_balance,
                            const uint8_t* active, void* stream) {
  if (!b || !rho || !out) return fail(RTE_EINVAL, "rte_residual: null argument");
  RTE_TRY(params_ready(b, "rte_residual"));
  if ((uintptr_t)rho & 15) return fail(RTE_EINVAL, "rte_residual: rho must be 16-byte aligned");
  DeviceGuard g(b->disc->device);
  return residual_launch(b, rho, out, cell_balance, active, (cudaStream_t)stream);
}
