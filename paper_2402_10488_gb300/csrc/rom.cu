// POD reduced order models (paper Sec. 3): offline stage on the GPU, ROMIG and ROMSA online.
//
// Offline (Sec. 3.1.1, 3.2.1): SI-DSA solves of the training instances store the converged
// angular flux f^mu and the first w iterates f^{mu,(l)}; F = [f^mu] and dF = [f^mu - f^{mu,(l)}].
// In X-Y geometry the +-v_z copies of a direction carry identical rows, so snapshots are stored
// once per distinct direction and every row-sum is weighted by the direction's multiplicity;
// this leaves F^T F, the singular values and U unchanged.  The thin SVD: X = Q R by classical
// Gram-Schmidt applied twice per column on the GPU (deterministic tiled FP64 inner products),
// then a one-sided Jacobi SVD R = U_R Sigma V^T on the host, U = Q U_R.  Truncation: a fixed rank,
// or Eq. (pod_truncation) with singular values.  Reduced operators (affine decomposition, cellwise materials m):
//     A_0r = sum_j U_j^T D_j U_j,   A_{a,m} = sum_j U_j^T M_m U_j,
//     A_{s,m} = A_{a,m} - (U^iso)^T M_m U^rho,   A_{mu,r} = A_0r + sum_m sigma_a,m A_{a,m} + sigma_s,m A_{s,m}
// with U^rho = sum_j omega_j U_j and U^iso = sum_j U_j (Eq. (rho_basis)); M_m is the mass matrix
// of material m's share of the cross sections: its indicator, or in 1D with cross sections linear
// across cells the function that is linear on each cell and 1 at the cell ends carrying m.
// Online: ROMIG rho^(0) = U^rho A_{mu,r}^{-1} U^T b_mu, U^T b_mu = (U^iso)^T G + sum over the
// sides of g_side a_side (a_side = U^T of the unit isotropic inflow through that side); ROMSA
// delta rho = dU^rho (dU^T A_mu dU)^{-1} (dU^iso)^T R (Eq. (rom_correction)).  The r x r systems
// are assembled and LU-factored on the device once per parameter set.
#include <cstdio>

#include "common.cuh"

namespace rte {

int run_si(rte_batch_t bt, const rte_solve_opts* o, rte_rom_t rom_c, double* rho,
           rte_solve_report* reports, double* history, cudaStream_t st, double* psi_cur,
           double* psi_win, int window);

// Per-batch online state cached in the ROM handle.
struct RomOnline {
  rte_batch_t batch = nullptr;
  DevBuf<double> lu;    // [B][r][r]
  DevBuf<int> piv;      // [B][r]
  DevBuf<double> proj;  // [B][r]
  DevBuf<uint8_t> tcws; // workspace of the BF16 tensor-core products (first word: status)
};

// ---- kernels ------------------------------------------------------------------------------

// out[part][cls][i][j] = sum over this block's rows of w(row) X[i][row] Y[j][row], rows whose
// class is cls0 + cls (other rows are skipped).  Row index = d * n_dof + e; w = mult[d];
// class = mat[e / P] (or 0).
__global__ void cross_gram_kernel(const double* __restrict__ X, int nx_cols,
                                  const double* __restrict__ Y, int ny_cols, size_t nrow,
                                  int n_dof, int P, const double* __restrict__ wdir,
                                  const int32_t* __restrict__ mat,
                                  const int32_t* __restrict__ matr, int cls0, int n_class,
                                  double* partial) {
  extern __shared__ double sm[];
  const int T = 16;
  double* Xs = sm;                        // [nx_cols][T]
  double* Ys = Xs + (size_t)nx_cols * T;  // [ny_cols][T]
  double* acc = Ys + (size_t)ny_cols * T; // [n_class][nx_cols*ny_cols]
  __shared__ double ws[16], wr[16];
  __shared__ int cs[16], cr[16];
  const int npairs = nx_cols * ny_cols;
  for (int p = threadIdx.x; p < n_class * npairs; p += blockDim.x) acc[p] = 0.0;
  const size_t ntiles = (nrow + T - 1) / T;
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    const size_t r0 = tile * T;
    for (int q = threadIdx.x; q < (nx_cols + ny_cols) * T; q += blockDim.x) {
      const int col = q / T, rr = q % T;
      const size_t row = r0 + rr;
      double v = 0.0;
      if (row < nrow) v = col < nx_cols ? X[(size_t)col * nrow + row] : Y[(size_t)(col - nx_cols) * nrow + row];
      sm[q] = v;
    }
    if (threadIdx.x < T) {
      const size_t row = r0 + threadIdx.x;
      double w = 0.0, w2 = 0.0;
      int c = 0, c2 = 0;
      if (row < nrow) {
        const size_t d = row / n_dof, e = row % n_dof;
        w = wdir ? wdir[d] : 1.0;
        if (matr) {
          w2 = w;
          c2 = matr[e / P] - cls0;
          if (c2 < 0 || c2 >= n_class) w2 = 0.0, c2 = 0;
        }
        c = (mat ? mat[e / P] : 0) - cls0;
        if (c < 0 || c >= n_class) w = 0.0, c = 0;
      }
      ws[threadIdx.x] = w;
      cs[threadIdx.x] = c;
      wr[threadIdx.x] = w2;
      cr[threadIdx.x] = c2;
    }
    __syncthreads();
    if (matr) {
      // 1D, cross sections linear across cells (P = 2; a tile holds whole cells, rows rr and
      // rr ^ 1 are one cell's two moments): material m's share of a cell is 1 at the ends that
      // carry m, so a cell adds x^T [[1/2, -k], [-k, 1/2]] y to its left-end material and
      // x^T [[1/2, k], [k, 1/2]] y to its right-end material, k = 1 / (2 sqrt 3).
      const double k = 0.28867513459481288225;
      for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        const int i = p / ny_cols, j = p % ny_cols;
        for (int rr = 0; rr < T; ++rr) {
          const double x = Xs[i * T + rr];
          const double vd = 0.5 * x * Ys[j * T + rr], vo = k * x * Ys[j * T + (rr ^ 1)];
          acc[cs[rr] * npairs + p] += ws[rr] * (vd - vo);
          acc[cr[rr] * npairs + p] += wr[rr] * (vd + vo);
        }
      }
    } else {
      for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        const int i = p / ny_cols, j = p % ny_cols;
        for (int rr = 0; rr < T; ++rr) {
          const double v = ws[rr] * Xs[i * T + rr] * Ys[j * T + rr];
          acc[cs[rr] * npairs + p] += v;
        }
      }
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < n_class * npairs; p += blockDim.x)
    partial[(size_t)blockIdx.x * n_class * npairs + p] = acc[p];
}

__global__ void sum_partials_kernel(const double* partial, int nparts, int n, double* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double s = 0.0;
  for (int k = 0; k < nparts; ++k) s += partial[(size_t)k * n + p];
  out[p] = s;
}

// U[i][row] = sum_k X[k][row] W[k][i]
// Columns k0 .. k0+nk of the sum (nk <= kBasisChunk); accumulate = add to U instead of storing.
constexpr int kBasisChunk = 128;
__global__ void basis_kernel(const double* __restrict__ X, int k0, int nk,
                             const double* __restrict__ W, int r, size_t nrow, double* U,
                             int accumulate) {
  const size_t row = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrow) return;
  double x[kBasisChunk];
  for (int k = 0; k < nk; ++k) x[k] = X[(size_t)(k0 + k) * nrow + row];
  for (int i = 0; i < r; ++i) {
    double s = accumulate ? U[(size_t)i * nrow + row] : 0.0;
    for (int k = 0; k < nk; ++k) s = fma(x[k], W[(size_t)(k0 + k) * r + i], s);
    U[(size_t)i * nrow + row] = s;
  }
}

// U [r][nrow] = sum_k X[k][row] W[k][i], in chunks of kBasisChunk snapshot columns
static int basis_launch(const double* X, int ncol, const double* W, int r, size_t nrow, double* U,
                        cudaStream_t st) {
  for (int k0 = 0; k0 < ncol; k0 += kBasisChunk) {
    const int nk = std::min(kBasisChunk, ncol - k0);
    basis_kernel<<<(unsigned)((nrow + 127) / 128), 128, 0, st>>>(X, k0, nk, W, r, nrow, U, k0 > 0); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
  }
  return RTE_OK;
}

// column differences: out[col] = F[b] - win[l][b] for the listed (b, l)
__global__ void diff_kernel(const double* F, const double* win, const int* pairs, int ncols,
                            size_t nrow, int B, double* out) {
  const int col = blockIdx.y;
  const int b = pairs[2 * col], l = pairs[2 * col + 1];
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nrow; e += (size_t)gridDim.x * blockDim.x)
    out[(size_t)col * nrow + e] = F[(size_t)b * nrow + e] - win[((size_t)l * B + b) * nrow + e];
}

// U_rho[i][e] = sum_d w_d U[i][d][e],  U_iso[i][e] = sum_d mult_d U[i][d][e]
__global__ void rho_iso_kernel(const double* U, int r, int n_dirs, int n_dof, const double* dirs,
                               double* U_rho, double* U_iso) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)r * n_dof) return;
  const int i = t / n_dof, e = t % n_dof;
  double sr = 0.0, si = 0.0;
  for (int d = 0; d < n_dirs; ++d) {
    const double u = U[((size_t)i * n_dirs + d) * n_dof + e];
    sr = fma(dirs[4 * d + 2], u, sr);
    si = fma(dirs[4 * d + 3], u, si);
  }
  U_rho[t] = sr;
  U_iso[t] = si;
}

// U_iso0[i][c] = U_iso[i][c * P]: the zeroth-moment rows, contiguous for the ROMIG projection
__global__ void iso0_kernel(const double* U_iso, int r, int n_cells, int P, double* U_iso0) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)r * n_cells) return;
  const size_t i = t / n_cells, c = t % n_cells;
  U_iso0[t] = U_iso[i * (size_t)n_cells * P + c * P];
}

// a_side[s][i] = U_i^T e_s: the right-hand side of a unit isotropic inflow through side s (1D: x-,
// x+; 2D: x-, x+, y-, y+), summed over the directions entering through it with their
// multiplicities.  In the orthonormal basis a unit inflow into a boundary cell contributes
// |v_n| * sqrt(h_t / h_n) * (1, -+sqrt3) on the two modes constant along the face (2D; h_n the
// width across the face, h_t along it) and |xi| / sqrt(h) * (1, -+sqrt3) in 1D.  One thread per
// (side, i), fixed summation order.
__global__ void inflow_basis_kernel(const double* U, int r, int n_dirs, int dim, int nx, int ny,
                                    int n_dof, double hx, double hy, const double* dx,
                                    const double* dirs, double* a_side) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * r) return;
  const int side = t / r, i = t % r;
  const double s3 = sqrt(3.0);
  double acc = 0.0;
  if (dim == 1 && side >= 2) {
    a_side[t] = 0.0;
    return;
  }
  for (int d = 0; d < n_dirs; ++d) {
    const double vx = dirs[4 * d], vy = dirs[4 * d + 1], mult = dirs[4 * d + 3];
    const double* u = U + ((size_t)i * n_dirs + d) * n_dof;
    if (dim == 1) {
      const bool in = side == 0 ? vx > 0 : vx < 0;
      if (!in) continue;
      const int c = side == 0 ? 0 : nx - 1;
      const double q = fabs(vx) / sqrt(dx[c]), sg = side == 0 ? -1.0 : 1.0;
      acc += mult * q * (u[2 * c] + sg * s3 * u[2 * c + 1]);
      continue;
    }
    const bool xside = side < 2;
    const double vn = xside ? vx : vy;
    const bool in = (side % 2 == 0) ? vn > 0 : vn < 0;
    if (!in) continue;
    const double q = xside ? fabs(vx) * sqrt(hy / hx) : fabs(vy) * sqrt(hx / hy);
    const double sg = (side % 2 == 0) ? -1.0 : 1.0;
    const int n_face = xside ? ny : nx;
    for (int f = 0; f < n_face; ++f) {
      const int c = xside ? f * nx + (side == 0 ? 0 : nx - 1) : (side == 2 ? 0 : ny - 1) * nx + f;
      // modes constant along the face: k = 0 and k = 1 (x-faces) or k = 2 (y-faces)
      const double m1 = xside ? u[4 * c + 1] : u[4 * c + 2];
      acc += mult * q * (u[4 * c] + sg * s3 * m1);
    }
  }
  a_side[t] = acc;
}

// proj[b][i] += sum_s g[b][s] a_side[s][i]
__global__ void add_inflow_rhs_kernel(double* proj, const double* inflow, const double* a_side, int r,
                                      int B, const uint8_t* mask) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * r) return;
  const int b = t / r, i = t % r;
  if (mask && !mask[b]) return;
  double s = proj[t];
  for (int side = 0; side < 4; ++side) s = fma(inflow[4 * b + side], a_side[(size_t)side * r + i], s);
  proj[t] = s;
}

// Y[i][d] = D_d U[i][d]: the upwind DG transport operator without Sigma_t (2D), with zero inflow.
__global__ void transport_apply2d_kernel(const double* U, int r, int n_dirs, int nx, int ny,
                                         double hx, double hy, const double* dirs, double* Y) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nc = (size_t)nx * ny;
  if (t >= (size_t)r * n_dirs * nc) return;
  const int c = t % nc;
  const int d = (t / nc) % n_dirs;
  const int i = t / (nc * n_dirs);
  const int ci = c % nx, cj = c / nx;
  const double vx = dirs[4 * d], vy = dirs[4 * d + 1];
  const double s3 = sqrt(3.0), sx = vx < 0 ? -1.0 : 1.0, sy = vy < 0 ? -1.0 : 1.0;
  const double ax = fabs(vx) / hx, ay = fabs(vy) / hy;
  const double* u = U + ((size_t)i * n_dirs + d) * nc * 4;
  const double* a = u + (size_t)c * 4;
  double y[4];
  // (ax Kx (x) I + ay I (x) Ky) a,  K = [[1, s sqrt3], [-s sqrt3, 3]], k = a + 2b
  for (int bb = 0; bb < 2; ++bb)
    for (int aa = 0; aa < 2; ++aa) {
      const int k = aa + 2 * bb;
      double v = 0.0;
      for (int a2 = 0; a2 < 2; ++a2) {
        const double K = a2 == aa ? (aa == 0 ? 1.0 : 3.0) : (aa == 0 ? sx * s3 : -sx * s3);
        v += ax * K * a[a2 + 2 * bb];
      }
      for (int b2 = 0; b2 < 2; ++b2) {
        const double K = b2 == bb ? (bb == 0 ? 1.0 : 3.0) : (bb == 0 ? sy * s3 : -sy * s3);
        v += ay * K * a[aa + 2 * b2];
      }
      y[k] = v;
    }
  // upwind x neighbour: its outflow trace t_x[q] = a_{0q} + s_x sqrt3 a_{1q}
  const int iu = ci - (int)sx;
  if (iu >= 0 && iu < nx) {
    const double* an = u + ((size_t)cj * nx + iu) * 4;
    for (int q = 0; q < 2; ++q) {
      const double tq = an[2 * q] + sx * s3 * an[1 + 2 * q];
      y[0 + 2 * q] -= ax * tq;
      y[1 + 2 * q] -= ax * (-sx * s3) * tq;
    }
  }
  const int ju = cj - (int)sy;
  if (ju >= 0 && ju < ny) {
    const double* an = u + ((size_t)ju * nx + ci) * 4;
    for (int q = 0; q < 2; ++q) {
      const double tq = an[q] + sy * s3 * an[q + 2];
      y[q] -= ay * tq;
      y[q + 2] -= ay * (-sy * s3) * tq;
    }
  }
  double* out = Y + ((size_t)i * n_dirs + d) * nc * 4 + (size_t)c * 4;
  for (int k = 0; k < 4; ++k) out[k] = y[k];
}

// 1D: own-cell terms scale with |xi| / h_c; the upwind face couples the upwind cell's outflow
// trace (scaled 1/sqrt h_up) with this cell's inflow trace (scaled 1/sqrt h_c).
__global__ void transport_apply1d_kernel(const double* U, int r, int n_dirs, int nx,
                                         const double* dx, const double* dirs, double* Y) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)r * n_dirs * nx) return;
  const int c = t % nx, d = (t / nx) % n_dirs, i = t / ((size_t)nx * n_dirs);
  const double xi = dirs[4 * d], s3 = sqrt(3.0), sg = xi < 0 ? -1.0 : 1.0, a = fabs(xi) / dx[c];
  const double* u = U + ((size_t)i * n_dirs + d) * nx * 2;
  const double a0 = u[2 * c], a1 = u[2 * c + 1];
  double y0 = a * (a0 + sg * s3 * a1), y1 = a * (-sg * s3 * a0 + 3.0 * a1);
  const int cu = c - (int)sg;
  if (cu >= 0 && cu < nx) {
    const double au = fabs(xi) / sqrt(dx[c] * dx[cu]);
    const double tq = u[2 * cu] + sg * s3 * u[2 * cu + 1];
    y0 -= au * tq;
    y1 -= au * (-sg * s3) * tq;
  }
  double* out = Y + ((size_t)i * n_dirs + d) * nx * 2;
  out[2 * c] = y0;
  out[2 * c + 1] = y1;
}

// A_{mu,r} per instance and its LU factorisation with partial pivoting, one warp per instance: lane l
// assembles the entries e = l, l + 32, ... and owns the rows q = l, l + 32, ... in the elimination.
// Every entry gets the same operations in the same order as a sequential Doolittle elimination, and
// the pivot is the first row of largest magnitude (a warp arg-max with ties to the lower row).
__global__ void rom_assemble_lu_warp_kernel(const double* A0, const double* Aa, const double* As,
                                            int r, int n_mat, const double* sigma_t,
                                            const double* sigma_s, int B, double* LU, int* piv,
                                            const uint8_t* mask) {
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (b >= B) return;                     // uniform over the warp
  if (mask && !mask[b]) return;
  double* A = LU + (size_t)b * r * r;
  for (int e = lane; e < r * r; e += 32) {
    double v = A0[e];
    for (int m = 0; m < n_mat; ++m) {
      const double st = sigma_t[b * n_mat + m], ss = sigma_s[b * n_mat + m];
      v += (st - ss) * Aa[(size_t)m * r * r + e] + ss * As[(size_t)m * r * r + e];
    }
    A[e] = v;
  }
  __syncwarp();
  for (int k = 0; k < r; ++k) {
    double best = -1.0;
    int p = r;
    for (int q = k + lane; q < r; q += 32) {
      const double v = fabs(A[q * r + k]);
      if (v > best) best = v, p = q;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int op = __shfl_xor_sync(0xffffffffu, p, o);
      if (ob > best || (ob == best && op < p)) best = ob, p = op;
    }
    if (lane == 0) piv[b * r + k] = p;
    if (p != k)
      for (int c = lane; c < r; c += 32) {
        const double t = A[k * r + c];
        A[k * r + c] = A[p * r + c];
        A[p * r + c] = t;
      }
    __syncwarp();
    const double inv = 1.0 / A[k * r + k];
    for (int q = k + 1 + lane; q < r; q += 32) {
      const double f = A[q * r + k] * inv;
      A[q * r + k] = f;
      for (int c = k + 1; c < r; ++c) A[q * r + c] -= f * A[k * r + c];
    }
    __syncwarp();
  }
}


// proj[b][i] = sum_e Ut[i][e] v[b][e * stride + off]  (one block per (i, b))
__global__ void project_kernel(const double* Ut, int n, const double* v, int stride, int off,
                               size_t vstride_b, double* proj, int r, const uint8_t* active) {
  const int i = blockIdx.x, b = blockIdx.y;
  if (active && !active[b]) return;
  double s = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x)
    s = fma(Ut[(size_t)i * n + e], v[(size_t)b * vstride_b + (size_t)e * stride + off], s);
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) proj[(size_t)b * r + i] = sh[0];
}

__global__ void lu_solve_kernel(const double* LU, const int* piv, double* x, int r, int B,
                                const uint8_t* active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || (active && !active[b])) return;
  const double* A = LU + (size_t)b * r * r;
  double* y = x + (size_t)b * r;
  for (int k = 0; k < r; ++k) {
    const int p = piv[b * r + k];
    if (p != k) {
      const double t = y[k];
      y[k] = y[p];
      y[p] = t;
    }
  }
  for (int q = 0; q < r; ++q)
    for (int c = 0; c < q; ++c) y[q] -= A[q * r + c] * y[c];
  for (int q = r - 1; q >= 0; --q) {
    for (int c = q + 1; c < r; ++c) y[q] -= A[q * r + c] * y[c];
    y[q] /= A[q * r + q];
  }
}

// out[b][e] = sum_i Ut[i][e] c[b][i]
__global__ void lift_kernel(const double* Ut, int n, const double* c, int r, double* out,
                            const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < r; ++i) s = fma(Ut[(size_t)i * n + e], c[(size_t)b * r + i], s);
    out[(size_t)b * n + e] = s;
  }
}

// ---- host helpers -----------------------------------------------------------------------------

struct GramCtx {
  DevBuf<double> partial, out;
};

// Host: returns sum over rows (weighted/classified) of X_i Y_j -> out[cls][i][j]
// Classes and Y columns are processed in chunks that keep the kernel's shared memory within
// bounds (many classes: e.g. one material per cell).
static int cross_gram(const double* X, int nxc, const double* Y, int nyc, size_t nrow, int n_dof,
                      int P, const double* wdir, const int32_t* mat, int n_class,
                      std::vector<double>& out, cudaStream_t st, const int32_t* matr = nullptr) {
  const int T = 16;
  const size_t budget = 200 * 1024 / sizeof(double);
  auto fits = [&](int nc, int ncl) {
    return (size_t)(nxc + nc) * T + (size_t)ncl * nxc * nc <= budget;
  };
  int ychunk = nyc, cchunk = n_class;
  while (!fits(ychunk, cchunk) && cchunk > 1) cchunk = (cchunk + 1) / 2;
  while (!fits(ychunk, cchunk) && ychunk > 1) ychunk = (ychunk + 1) / 2;
  if (!fits(ychunk, cchunk)) return fail(RTE_EINVAL, "ROM: too many basis vectors for the Gram kernel");
  int nblocks = (int)std::min<size_t>((nrow + T - 1) / T, 1024);
  GramCtx g;
  RTE_TRY(g.partial.alloc((size_t)nblocks * cchunk * nxc * ychunk));
  RTE_TRY(g.out.alloc((size_t)cchunk * nxc * ychunk));
  out.assign((size_t)n_class * nxc * nyc, 0.0);
  std::vector<double> part;
  for (int c0 = 0; c0 < n_class; c0 += cchunk) {
    const int ncl = std::min(cchunk, n_class - c0);
    for (int j0 = 0; j0 < nyc; j0 += ychunk) {
      const int nc = std::min(ychunk, nyc - j0);
      const size_t npairs = (size_t)nxc * nc;
      const size_t smem = ((size_t)(nxc + nc) * T + ncl * npairs) * sizeof(double);
      RTE_CUDA_TRY(cudaFuncSetAttribute(cross_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
      cross_gram_kernel<<<nblocks, 256, smem, st>>>(X, nxc, Y + (size_t)j0 * nrow, nc, nrow, n_dof,
                                                    P, wdir, mat, matr, c0, ncl, g.partial.p); RTE_NOTE_LAUNCH();
      RTE_CUDA_TRY(cudaGetLastError());
      const int n = (int)(ncl * npairs);
      sum_partials_kernel<<<(n + 255) / 256, 256, 0, st>>>(g.partial.p, nblocks, n, g.out.p); RTE_NOTE_LAUNCH();
      part.resize(n);
      RTE_CUDA_TRY(cudaMemcpyAsync(part.data(), g.out.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
      RTE_CUDA_TRY(cudaStreamSynchronize(st));
      for (int c = 0; c < ncl; ++c)
        for (int i = 0; i < nxc; ++i)
          for (int j = 0; j < nc; ++j)
            out[((size_t)(c0 + c) * nxc + i) * nyc + j0 + j] = part[((size_t)c * nxc + i) * nc + j];
    }
  }
  return RTE_OK;
}

// q -= sum_{i<j} h[i] Q_i  (columns contiguous, length nrow)
__global__ void sub_cols_kernel(double* q, const double* Q, int j, const double* h, size_t nrow) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nrow;
       e += (size_t)gridDim.x * blockDim.x) {
    double s = q[e];
    for (int i = 0; i < j; ++i) s = fma(-h[i], Q[(size_t)i * nrow + e], s);
    q[e] = s;
  }
}

__global__ void scale_col_kernel(double* q, double c, size_t nrow) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nrow;
       e += (size_t)gridDim.x * blockDim.x)
    q[e] *= c;
}

// One-sided Jacobi SVD (Hestenes) of a small n x n matrix A (row-major): rotations orthogonalise
// the columns of A; at convergence column k has norm sigma_k and direction u_k.  Returns the
// singular values in descending order and U (row-major, column k = u_k).  Singular values come
// out with an absolute error of a few ulps of ||A|| (no squaring of the matrix).
static void jacobi_svd(std::vector<double> A, int n, std::vector<double>& sv, std::vector<double>& U) {
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double a = 0, b = 0, g = 0;
        for (int k = 0; k < n; ++k) {
          const double x = A[(size_t)k * n + p], y = A[(size_t)k * n + q];
          a += x * x, b += y * y, g += x * y;
        }
        if (g == 0.0 || std::fabs(g) <= 1e-15 * std::sqrt(a * b)) continue;
        rotated = true;
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int k = 0; k < n; ++k) {
          const double x = A[(size_t)k * n + p], y = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * x - s * y;
          A[(size_t)k * n + q] = s * x + c * y;
        }
      }
    if (!rotated) break;
  }
  std::vector<double> nrm(n);
  for (int j = 0; j < n; ++j) {
    double t = 0;
    for (int k = 0; k < n; ++k) t += A[(size_t)k * n + j] * A[(size_t)k * n + j];
    nrm[j] = std::sqrt(t);
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return nrm[x] > nrm[y]; });
  sv.resize(n);
  U.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    const int j = order[i];
    sv[i] = nrm[j];
    for (int k = 0; k < n; ++k) U[(size_t)k * n + i] = nrm[j] > 0 ? A[(size_t)k * n + j] / nrm[j] : 0.0;
  }
}

// One round of the parallel one-sided Jacobi SVD on the device: A is n x n, column-major (column
// j at A + j n); block k rotates the disjoint column pair pairs[2k], pairs[2k+1] (-1: no partner)
// so that the two columns become orthogonal.  rotated is set when some pair was not yet
// orthogonal to the tolerance.  Dot products are reduced in a fixed order (deterministic).
__global__ void jacobi_round_kernel(double* A, size_t n, const int* pairs, int npairs,
                                    int* rotated) {
  const int k = blockIdx.x;
  if (k >= npairs) return;
  const int p = pairs[2 * k], q = pairs[2 * k + 1];
  if (p < 0 || q < 0) return;
  double* ap = A + (size_t)p * n;
  double* aq = A + (size_t)q * n;
  double a = 0, b = 0, g = 0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = ap[i], y = aq[i];
    a = fma(x, x, a), b = fma(y, y, b), g = fma(x, y, g);
  }
  __shared__ double sa[256], sb[256], sg[256];
  sa[threadIdx.x] = a, sb[threadIdx.x] = b, sg[threadIdx.x] = g;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      sa[threadIdx.x] += sa[threadIdx.x + h];
      sb[threadIdx.x] += sb[threadIdx.x + h];
      sg[threadIdx.x] += sg[threadIdx.x + h];
    }
    __syncthreads();
  }
  a = sa[0], b = sb[0], g = sg[0];
  if (g == 0.0 || fabs(g) <= 1e-15 * sqrt(a * b)) return;
  const double zeta = (b - a) / (2.0 * g);
  const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = ap[i], y = aq[i];
    ap[i] = c * x - s * y;
    aq[i] = s * x + c * y;
  }
  if (threadIdx.x == 0) atomicExch(rotated, 1);
}

// Round-robin (circle method) pairing: every two of n columns meet once per sweep, in n' - 1
// rounds of n' / 2 disjoint pairs (n' = n rounded up to even; -1 marks the dummy column).
static std::vector<int> round_robin_pairs(int n) {
  const int m = n + (n & 1);
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i < n ? i : -1;
  std::vector<int> pairs((size_t)(m - 1) * m);
  for (int r = 0; r < m - 1; ++r) {
    for (int k = 0; k < m / 2; ++k) {
      pairs[((size_t)r * (m / 2) + k) * 2] = order[k];
      pairs[((size_t)r * (m / 2) + k) * 2 + 1] = order[m - 1 - k];
    }
    const int last = order[m - 1];
    for (int i = m - 1; i > 1; --i) order[i] = order[i - 1];
    order[1] = last;
  }
  return pairs;
}

// Sweeps of the one-sided Jacobi method on the n columns (length len, contiguous) of A on the
// device until no pair needs a rotation.
static int jacobi_columns_device(double* A, size_t len, int n, cudaStream_t st) {
  if (n < 2) return RTE_OK;
  const int m = n + (n & 1);
  const std::vector<int> pairs = round_robin_pairs(n);
  DevBuf<int> P, flag;
  RTE_TRY(P.alloc(pairs.size()));
  RTE_TRY(flag.alloc(1));
  RTE_CUDA_TRY(cudaMemcpyAsync(P.p, pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice, st));
  for (int sweep = 0; sweep < 80; ++sweep) {
    RTE_CUDA_TRY(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    for (int r = 0; r < m - 1; ++r) {
      jacobi_round_kernel<<<m / 2, 256, 0, st>>>(A, len, P.p + (size_t)r * m, m / 2, flag.p); RTE_NOTE_LAUNCH();
    }
    RTE_CUDA_TRY(cudaGetLastError());
    int h = 0;
    RTE_CUDA_TRY(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    if (!h) break;
  }
  return RTE_OK;
}

// One-sided Jacobi SVD of the n x n row-major matrix R on the device (for large snapshot counts):
// the round-robin (circle) ordering pairs every two columns once per sweep in n - 1 rounds of
// n / 2 disjoint pairs.  Same outputs as jacobi_svd.
static int jacobi_svd_device(const std::vector<double>& R, int n, std::vector<double>& sv,
                             std::vector<double>& U, cudaStream_t st) {
  std::vector<double> Acm((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Acm[(size_t)j * n + i] = R[(size_t)i * n + j];
  DevBuf<double> A;
  RTE_TRY(A.alloc(Acm.size()));
  RTE_CUDA_TRY(cudaMemcpyAsync(A.p, Acm.data(), sizeof(double) * Acm.size(), cudaMemcpyHostToDevice, st));
  RTE_TRY(jacobi_columns_device(A.p, n, n, st));
  RTE_CUDA_TRY(cudaMemcpyAsync(Acm.data(), A.p, sizeof(double) * Acm.size(), cudaMemcpyDeviceToHost, st));
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<double> nrm(n);
  for (int j = 0; j < n; ++j) {
    double t = 0;
    for (int i = 0; i < n; ++i) t += Acm[(size_t)j * n + i] * Acm[(size_t)j * n + i];
    nrm[j] = std::sqrt(t);
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int x, int y) { return nrm[x] > nrm[y]; });
  sv.resize(n);
  U.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    const int j = idx[i];
    sv[i] = nrm[j];
    for (int k = 0; k < n; ++k) U[(size_t)k * n + i] = nrm[j] > 0 ? Acm[(size_t)j * n + k] / nrm[j] : 0.0;
  }
  return RTE_OK;
}

// rows of direction d (row = d * n_dof + e) scaled by w[d]^power (power = +-1/2)
__global__ void scale_rows_kernel(double* A, int ncol, size_t nrow, int n_dof, const double* w,
                                  double power) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)ncol * nrow) return;
  const size_t row = t % nrow;
  if (w) A[t] *= pow(w[row / n_dof], power);
}

// norms[j] = ||A_j|| for the n columns of length len (fixed-order block reduction)
__global__ void col_norms_kernel(const double* A, size_t len, double* norms) {
  const double* a = A + (size_t)blockIdx.x * len;
  double s = 0.0;
  for (size_t i = threadIdx.x; i < len; i += blockDim.x) s = fma(a[i], a[i], s);
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) norms[blockIdx.x] = sqrt(sh[0]);
}

// U[i] = A[idx[i]] / sv[i], rows unweighted by w^-1/2
__global__ void take_cols_kernel(const double* A, const int* idx, const double* sv, int r, size_t nrow,
                                 int n_dof, const double* w, double* U) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)r * nrow) return;
  const int i = t / nrow;
  const size_t row = t % nrow;
  const double sc = w ? 1.0 / sqrt(w[row / n_dof]) : 1.0;
  U[t] = A[(size_t)idx[i] * nrow + row] / sv[i] * sc;
}

// Truncation rank: a fixed rank, or Eq. (pod_truncation) with singular values.
static void pod_rank_of(rte_rom_t rom, int ncol, int rank, double eps_pod) {
  double total = 0.0;
  for (double v : rom->sv) total += v;
  int r = rank;
  if (r <= 0) {  // smallest l with sum_{k<=l} s_k / trace >= 1 - eps
    double acc = 0.0;
    r = ncol;
    for (int i = 0; i < ncol; ++i) {
      acc += rom->sv[i];
      if (acc / total >= 1.0 - eps_pod) {
        r = i + 1;
        break;
      }
    }
  }
  int nz = 0;
  for (int i = 0; i < ncol; ++i) nz += rom->sv[i] > 1e-14 * rom->sv[0];
  r = std::min(r, std::max(nz, 1));
  r = std::min(r, ncol);
  rom->r = r;
  rom->n_snap = ncol;
  double kept = 0.0;
  for (int i = 0; i < r; ++i) kept += rom->sv[i];
  rom->eps_equiv = total > 0 ? 1.0 - kept / total : 0.0;
}

// POD of a snapshot matrix of moderate size by the one-sided Jacobi method applied to the
// (row-weighted) snapshots themselves on the device: the columns are rotated until mutually
// orthogonal; their norms are the singular values and their directions the left singular vectors.
// No orthogonalisation of nearly dependent snapshots is involved, so large snapshot sets with many
// tiny singular values keep their accuracy.
static int pod_direct(rte_rom_t rom, const double* X, int ncol, size_t nrow, int rank,
                      double eps_pod, const double* wdir, cudaStream_t st) {
  const rte_disc_s* d = rom->disc;
  DevBuf<double> A, nrmd, svd;
  DevBuf<int> idxd;
  RTE_TRY(A.alloc((size_t)ncol * nrow));
  RTE_TRY(nrmd.alloc(ncol));
  RTE_CUDA_TRY(cudaMemcpyAsync(A.p, X, sizeof(double) * ncol * nrow, cudaMemcpyDeviceToDevice, st));
  const size_t tot = (size_t)ncol * nrow;
  scale_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(A.p, ncol, nrow, d->n_dof, wdir, 0.5); RTE_NOTE_LAUNCH();
  RTE_TRY(jacobi_columns_device(A.p, nrow, ncol, st));
  col_norms_kernel<<<ncol, 256, 0, st>>>(A.p, nrow, nrmd.p); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  std::vector<double> nrm(ncol);
  RTE_CUDA_TRY(cudaMemcpyAsync(nrm.data(), nrmd.p, sizeof(double) * ncol, cudaMemcpyDeviceToHost, st));
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int> idx(ncol);
  for (int i = 0; i < ncol; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int x, int y) { return nrm[x] > nrm[y]; });
  rom->sv.resize(ncol);
  for (int i = 0; i < ncol; ++i) rom->sv[i] = nrm[idx[i]];
  pod_rank_of(rom, ncol, rank, eps_pod);
  const int r = rom->r;
  RTE_TRY(idxd.alloc(r));
  RTE_TRY(svd.alloc(r));
  RTE_CUDA_TRY(cudaMemcpyAsync(idxd.p, idx.data(), sizeof(int) * r, cudaMemcpyHostToDevice, st));
  RTE_CUDA_TRY(cudaMemcpyAsync(svd.p, rom->sv.data(), sizeof(double) * r, cudaMemcpyHostToDevice, st));
  RTE_TRY(rom->U.alloc((size_t)r * nrow));
  take_cols_kernel<<<(unsigned)(((size_t)r * nrow + 255) / 256), 256, 0, st>>>(
      A.p, idxd.p, svd.p, r, nrow, d->n_dof, wdir, rom->U.p); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  return RTE_OK;
}

// POD of X [ncol][nrow] (columns contiguous): fills rom->U [r][nrow], sv, r, eps_equiv.
// Thin SVD X = Q R = (Q U_R) Sigma V^T: Q from classical Gram-Schmidt applied twice per column on
// the GPU (inner products weighted by direction multiplicity), then a one-sided Jacobi SVD of the
// small R.  Unlike an eigen-decomposition of X^T X this resolves singular values down to a few
// ulps of sigma_1, which truncation tolerances like eps_POD = 1e-9 need.  Snapshot sets with more
// than 256 columns and at most 4e8 entries go through pod_direct instead: orthogonalising many
// nearly dependent snapshots one by one loses the small singular values.
static int pod(rte_rom_t rom, const double* X, int ncol, size_t nrow, int rank, double eps_pod,
               const double* wdir, cudaStream_t st) {
  const rte_disc_s* d = rom->disc;
  if (ncol < 1) return fail(RTE_EINVAL, "ROM: no snapshots");
  if (ncol > 4096) return fail(RTE_EINVAL, "ROM: at most 4096 snapshots per basis");
  if (ncol > 256 && (double)ncol * nrow <= 4e8) return pod_direct(rom, X, ncol, nrow, rank, eps_pod, wdir, st);
  DevBuf<double> Q, hdev;
  RTE_TRY(Q.alloc((size_t)ncol * nrow));
  RTE_TRY(hdev.alloc(ncol));
  RTE_CUDA_TRY(cudaMemcpyAsync(Q.p, X, sizeof(double) * ncol * nrow, cudaMemcpyDeviceToDevice, st));
  std::vector<double> R((size_t)ncol * ncol, 0.0), h, nn;
  const unsigned grid = (unsigned)std::min<size_t>((nrow + 255) / 256, 4096);
  for (int j = 0; j < ncol; ++j) {
    double* qj = Q.p + (size_t)j * nrow;
    RTE_TRY(cross_gram(qj, 1, qj, 1, nrow, d->n_dof, d->P, wdir, nullptr, 1, nn, st));
    const double xnorm = std::sqrt(std::max(nn[0], 0.0));
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      RTE_TRY(cross_gram(qj, 1, Q.p, j, nrow, d->n_dof, d->P, wdir, nullptr, 1, h, st));
      for (int i = 0; i < j; ++i) R[(size_t)i * ncol + j] += h[i];
      RTE_CUDA_TRY(cudaMemcpyAsync(hdev.p, h.data(), sizeof(double) * j, cudaMemcpyHostToDevice, st));
      sub_cols_kernel<<<grid, 256, 0, st>>>(qj, Q.p, j, hdev.p, nrow); RTE_NOTE_LAUNCH();
      RTE_CUDA_TRY(cudaGetLastError());
    }
    RTE_TRY(cross_gram(qj, 1, qj, 1, nrow, d->n_dof, d->P, wdir, nullptr, 1, nn, st));
    const double nrm = std::sqrt(std::max(nn[0], 0.0));
    // a column already in the span of the previous ones (to rounding) contributes nothing new
    const bool dependent = !(nrm > 1e-14 * xnorm) || nrm == 0.0;
    R[(size_t)j * ncol + j] = dependent ? 0.0 : nrm;
    scale_col_kernel<<<grid, 256, 0, st>>>(qj, dependent ? 0.0 : 1.0 / nrm, nrow); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
  }
  std::vector<double> UR;
  if (ncol <= 256) jacobi_svd(R, ncol, rom->sv, UR);
  else RTE_TRY(jacobi_svd_device(R, ncol, rom->sv, UR, st));
  pod_rank_of(rom, ncol, rank, eps_pod);
  const int r = rom->r;
  // U = Q U_R[:, :r]
  std::vector<double> W((size_t)ncol * r);
  for (int k = 0; k < ncol; ++k)
    for (int i = 0; i < r; ++i) W[(size_t)k * r + i] = UR[(size_t)k * ncol + i];
  DevBuf<double> Wd;
  RTE_TRY(Wd.alloc(W.size()));
  RTE_CUDA_TRY(cudaMemcpyAsync(Wd.p, W.data(), sizeof(double) * W.size(), cudaMemcpyHostToDevice, st));
  RTE_TRY(rom->U.alloc((size_t)r * nrow));
  RTE_TRY(basis_launch(Q.p, ncol, Wd.p, r, nrow, rom->U.p, st));
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  return RTE_OK;
}

// U^rho, U^iso and the affine reduced operators for a basis already in rom->U.
static int reduce_operators(rte_rom_t rom, cudaStream_t st) {
  const rte_disc_s* d = rom->disc;
  const int r = rom->r, n = d->n_dof;
  const size_t nrow = (size_t)d->n_dirs * n;
  RTE_TRY(rom->U_rho.alloc((size_t)r * n));
  RTE_TRY(rom->U_iso.alloc((size_t)r * n));
  rho_iso_kernel<<<(unsigned)(((size_t)r * n + 255) / 256), 256, 0, st>>>(
      rom->U.p, r, d->n_dirs, n, d->dir_dev.p, rom->U_rho.p, rom->U_iso.p); RTE_NOTE_LAUNCH();
  RTE_TRY(rom->U_iso0.alloc((size_t)r * d->n_cells));
  iso0_kernel<<<(unsigned)(((size_t)r * d->n_cells + 255) / 256), 256, 0, st>>>(
      rom->U_iso.p, r, d->n_cells, d->P, rom->U_iso0.p); RTE_NOTE_LAUNCH();
  RTE_TRY(rom->a_side.alloc((size_t)4 * r));
  inflow_basis_kernel<<<(4 * r + 127) / 128, 128, 0, st>>>(
      rom->U.p, r, d->n_dirs, d->dim, d->nx, d->ny, d->n_dof, d->hx, d->hy,
      d->dim == 1 ? d->dx_dev.p : nullptr, d->dir_dev.p, rom->a_side.p); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  // multiplicity per direction as the row weight
  std::vector<double> mult(d->n_dirs);
  for (int k = 0; k < d->n_dirs; ++k) mult[k] = d->dirs[k].mult;
  DevBuf<double> multd, Y;
  RTE_TRY(multd.alloc(d->n_dirs));
  RTE_CUDA_TRY(cudaMemcpyAsync(multd.p, mult.data(), sizeof(double) * d->n_dirs, cudaMemcpyHostToDevice, st));
  RTE_TRY(Y.alloc((size_t)r * nrow));
  if (d->dim == 2) {
    const size_t tot = (size_t)r * d->n_dirs * d->n_cells;
    transport_apply2d_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
        rom->U.p, r, d->n_dirs, d->nx, d->ny, d->hx, d->hy, d->dir_dev.p, Y.p); RTE_NOTE_LAUNCH();
  } else {
    const size_t tot = (size_t)r * d->n_dirs * d->nx;
    transport_apply1d_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
        rom->U.p, r, d->n_dirs, d->nx, d->dx_dev.p, d->dir_dev.p, Y.p); RTE_NOTE_LAUNCH();
  }
  RTE_CUDA_TRY(cudaGetLastError());
  std::vector<double> A0, Aa, C;
  // A_0r[i][j] = sum_rows mult U_i (D U_j)
  RTE_TRY(cross_gram(rom->U.p, r, Y.p, r, nrow, n, d->P, multd.p, nullptr, 1, A0, st));
  RTE_TRY(cross_gram(rom->U.p, r, rom->U.p, r, nrow, n, d->P, multd.p, d->mat_id.p, d->n_mat, Aa, st,
                     d->mat_r.p));
  RTE_TRY(cross_gram(rom->U_iso.p, r, rom->U_rho.p, r, n, n, d->P, nullptr, d->mat_id.p, d->n_mat, C,
                     st, d->mat_r.p));
  rom->A0 = A0;
  rom->Aa = Aa;
  rom->As.resize(Aa.size());
  for (size_t k = 0; k < Aa.size(); ++k) rom->As[k] = Aa[k] - C[k];
  RTE_TRY(rom->A0_dev.alloc(A0.size()));
  RTE_TRY(rom->Aa_dev.alloc(Aa.size()));
  RTE_TRY(rom->As_dev.alloc(Aa.size()));
  RTE_CUDA_TRY(cudaMemcpyAsync(rom->A0_dev.p, A0.data(), 8 * A0.size(), cudaMemcpyHostToDevice, st));
  RTE_CUDA_TRY(cudaMemcpyAsync(rom->Aa_dev.p, Aa.data(), 8 * Aa.size(), cudaMemcpyHostToDevice, st));
  RTE_CUDA_TRY(cudaMemcpyAsync(rom->As_dev.p, rom->As.data(), 8 * Aa.size(), cudaMemcpyHostToDevice, st));
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  rom->U.release();  // the online stage needs U^rho, U^iso and the reduced operators only
  return RTE_OK;
}

// Assemble and factor A_{mu,r} for the instances of `bt` in `mask` (all when null); the factors
// are cached in the ROM handle for that batch.
int rom_prepare(rte_rom_t rom, rte_batch_t bt, cudaStream_t st, const uint8_t* mask) {
  if (!rom->online) rom->online = new RomOnline();
  RomOnline* o = rom->online;
  const int r = rom->r, B = bt->B;
  if (o->lu.n != (size_t)B * r * r) {
    RTE_TRY(o->lu.alloc((size_t)B * r * r));
    RTE_TRY(o->piv.alloc((size_t)B * r));
    RTE_TRY(o->proj.alloc((size_t)B * r));
  }
  rom_assemble_lu_warp_kernel<<<(B + 3) / 4, 128, 0, st>>>(rom->A0_dev.p, rom->Aa_dev.p, rom->As_dev.p,
                                                           r, bt->disc->n_mat, bt->sigma_t.p,
                                                           bt->sigma_s.p, B, o->lu.p, o->piv.p,
                                                           mask); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  o->batch = bt;
  return RTE_OK;
}

// ROMIG (Sec. 3.1.2): U^T b = (U^iso)^T G + sum_s g_s a_side[s]; G has only its zeroth moment per
// cell, so its projection reads the k = 0 rows of U^iso, kept contiguous as U_iso0 [r][n_cells].
int rom_guess_launch(rte_rom_t rom, rte_batch_t b, double* rho0, const uint8_t* mask,
                     cudaStream_t st) {
  RTE_TRY(rom_prepare(rom, b, st, mask));
  const int r = rom->r, n = b->disc->n_dof, B = b->B, nc = b->disc->n_cells;
  RomOnline* o = rom->online;
  project_kernel<<<dim3(r, B), 256, 0, st>>>(rom->U_iso0.p, nc, b->G0.p, 1, 0, (size_t)nc,
                                             o->proj.p, r, mask); RTE_NOTE_LAUNCH();
  add_inflow_rhs_kernel<<<(B * r + 127) / 128, 128, 0, st>>>(o->proj.p, b->inflow.p, rom->a_side.p, r,
                                                             B, mask); RTE_NOTE_LAUNCH();
  lu_solve_kernel<<<(B + 63) / 64, 64, 0, st>>>(o->lu.p, o->piv.p, o->proj.p, r, B, mask); RTE_NOTE_LAUNCH();
  lift_kernel<<<dim3(std::min((n + 255) / 256, 1024), B), 256, 0, st>>>(rom->U_rho.p, n, o->proj.p, r,
                                                                        rho0, mask); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

int rom_tc_status(rte_rom_t rom, int* status) {
  *status = 0;
  if (!rom->online || !rom->online->tcws.p) return RTE_OK;
  RTE_CUDA_TRY(cudaMemcpy(status, rom->online->tcws.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (*status) RTE_CUDA_TRY(cudaMemset(rom->online->tcws.p, 0, sizeof(int)));  // reported once
  return RTE_OK;
}

int rom_correction(rte_rom_t rom, rte_batch_t bt, const double* R, double* drho,
                   const uint8_t* active, cudaStream_t st, bool bf16) {
  RomOnline* o = rom->online;
  if (!o || o->batch != bt) RTE_TRY(rom_prepare(rom, bt, st));
  o = rom->online;
  const int r = rom->r, n = bt->disc->n_dof, B = bt->B;
  if (bf16 && r <= 32) {
    const size_t need = pod_project_ws_bytes(n, B, bt->n_sm);
    if (o->tcws.n < need) {
      RTE_TRY(o->tcws.alloc(need));
      RTE_CUDA_TRY(cudaMemsetAsync(o->tcws.p, 0, 256, st));
    }
    RTE_TRY(pod_project_bf16(rom->U_iso.p, r, n, R, B, active, o->proj.p, o->tcws.p, bt->n_sm, st));
    lu_solve_kernel<<<(B + 63) / 64, 64, 0, st>>>(o->lu.p, o->piv.p, o->proj.p, r, B, active); RTE_NOTE_LAUNCH();
    RTE_TRY(pod_lift_bf16(rom->U_rho.p, r, n, o->proj.p, B, active, drho,
                          reinterpret_cast<int*>(o->tcws.p), st));
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
  }
  project_kernel<<<dim3(r, B), 256, 0, st>>>(rom->U_iso.p, n, R, 1, 0, (size_t)n, o->proj.p, r, active); RTE_NOTE_LAUNCH();
  lu_solve_kernel<<<(B + 63) / 64, 64, 0, st>>>(o->lu.p, o->piv.p, o->proj.p, r, B, active); RTE_NOTE_LAUNCH();
  lift_kernel<<<dim3(std::min((n + 255) / 256, 1024), B), 256, 0, st>>>(rom->U_rho.p, n, o->proj.p, r,
                                                                        drho, active); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

}  // namespace rte

rte_rom_s::~rte_rom_s() { delete online; }

using namespace rte;

extern "C" int rte_rom_build(rte_batch_t train, const rte_rom_opts* opts, rte_rom_t* rom_p,
                             rte_rom_t* rom_c, void* stream) {
  if (!train || !opts) return fail(RTE_EINVAL, "rte_rom_build: null argument");
  RTE_TRY(params_ready(train, "rte_rom_build"));
  if (opts->window < 1 || opts->max_iter < 1 || !(opts->eps_train > 0) ||
      (opts->correction_start != 0 && opts->correction_start != 1))
    return fail(RTE_EINVAL, "rte_rom_build: bad options");
  if ((opts->rank_p <= 0 || opts->rank_c <= 0) && !(opts->eps_pod > 0 && opts->eps_pod < 1))
    return fail(RTE_EINVAL, "rte_rom_build: need a rank or 0 < eps_pod < 1");
  const bool romig_start = opts->correction_start == 1 && rom_c != nullptr;
  if (rom_p) *rom_p = nullptr;
  if (rom_c) *rom_c = nullptr;
  rte_disc_s* d = train->disc;
  DeviceGuard g(d->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int B = train->B, w = opts->window;
  const size_t nrow = (size_t)d->n_dirs * d->n_dof;
  DevBuf<double> psi_cur, psi_win, rho;
  RTE_TRY(psi_cur.alloc((size_t)B * nrow));
  RTE_TRY(psi_win.alloc((size_t)w * B * nrow));
  RTE_TRY(rho.alloc((size_t)B * d->n_dof));
  RTE_CUDA_TRY(cudaMemsetAsync(rho.p, 0, sizeof(double) * B * d->n_dof, st));
  rte_solve_opts so{opts->eps_train, 0, opts->max_iter, RTE_SA_DSA, 0, 0.0,
                    opts->dsa_rtol > 0 ? opts->dsa_rtol : 1e-12, 2000, nullptr, 0.0, 0.0, 0, 0, 0};
  std::vector<rte_solve_report> rep(B);
  int s = run_si(train, &so, nullptr, rho.p, rep.data(), nullptr, st, psi_cur.p, psi_win.p, w);
  if (s != RTE_OK) return s == RTE_ENOCONV ? fail(RTE_ENOCONV, "training solve did not converge") : s;
  std::vector<double> mult(d->n_dirs);
  for (int k = 0; k < d->n_dirs; ++k) mult[k] = d->dirs[k].mult;
  DevBuf<double> multd;
  RTE_TRY(multd.alloc(d->n_dirs));
  RTE_CUDA_TRY(cudaMemcpyAsync(multd.p, mult.data(), 8 * mult.size(), cudaMemcpyHostToDevice, st));
  // parametric ROM from F = [f^mu] (needed first when the correction runs start from ROMIG)
  rte_rom_s* rp = nullptr;
  if (rom_p || romig_start) {
    rp = new rte_rom_s();
    rp->disc = d;
    int e = pod(rp, psi_cur.p, B, nrow, opts->rank_p, opts->eps_pod, multd.p, st);
    if (e == RTE_OK) e = reduce_operators(rp, st);
    if (e != RTE_OK) {
      delete rp;
      return e;
    }
  }
  if (romig_start) {
    // remark after Alg. 2: the same training solves again, from the ROMIG guess
    int e = rom_guess_launch(rp, train, rho.p, nullptr, st);
    if (e == RTE_OK) e = run_si(train, &so, nullptr, rho.p, rep.data(), nullptr, st, psi_cur.p, psi_win.p, w);
    if (e != RTE_OK) {
      delete rp;
      return e == RTE_ENOCONV ? fail(RTE_ENOCONV, "training solve did not converge") : e;
    }
  }
  // correction snapshots: (b, l) for l < min(n_conv, w)
  std::vector<int> pairs;
  for (int b = 0; b < B; ++b)
    for (int l = 0; l < std::min(rep[b].n_sweep, w); ++l) pairs.push_back(b), pairs.push_back(l);
  const int ndc = (int)pairs.size() / 2;
  if (rom_c) {
    DevBuf<double> dF;
    DevBuf<int> pairs_d;
    int e = dF.alloc((size_t)ndc * nrow);
    if (e == RTE_OK) e = pairs_d.alloc(pairs.size());
    if (e == RTE_OK && cudaMemcpyAsync(pairs_d.p, pairs.data(), sizeof(int) * pairs.size(),
                                       cudaMemcpyHostToDevice, st) != cudaSuccess)
      e = fail(RTE_ECUDA, "rte_rom_build: upload");
    if (e == RTE_OK) {
      diff_kernel<<<dim3(1024, ndc), 256, 0, st>>>(psi_cur.p, psi_win.p, pairs_d.p, ndc, nrow, B, dF.p); RTE_NOTE_LAUNCH();
      if (cudaGetLastError() != cudaSuccess) e = fail(RTE_ECUDA, "rte_rom_build: diff kernel");
    }
    auto* rc = new rte_rom_s();
    rc->disc = d;
    if (e == RTE_OK) e = pod(rc, dF.p, ndc, nrow, opts->rank_c, opts->eps_pod, multd.p, st);
    if (e == RTE_OK) e = reduce_operators(rc, st);
    if (e != RTE_OK) {
      delete rc;
      delete rp;
      return e;
    }
    *rom_c = rc;
  }
  if (rom_p) *rom_p = rp;
  else delete rp;
  return RTE_OK;
}

extern "C" int rte_rom_destroy(rte_rom_t rom) {
  if (!rom) return RTE_OK;
  DeviceGuard g(rom->disc->device);
  delete rom;
  return RTE_OK;
}

extern "C" int rte_rom_info(rte_rom_t rom, double* info, double* sv) {
  if (!rom || !info) return fail(RTE_EINVAL, "rte_rom_info: null argument");
  double tot = 0.0;
  for (double v : rom->sv) tot += v;
  info[0] = rom->r;
  info[1] = rom->n_snap;
  info[2] = rom->eps_equiv;
  info[3] = rom->disc->n_dirs;
  info[4] = rom->disc->n_dof;
  info[5] = tot;
  if (sv) std::memcpy(sv, rom->sv.data(), sizeof(double) * rom->sv.size());
  return RTE_OK;
}

extern "C" int rte_rom_initial_guess(rte_rom_t rom, rte_batch_t b, double* rho0,
                                     const uint8_t* active, void* stream) {
  if (!rom || !b || !rho0) return fail(RTE_EINVAL, "rte_rom_initial_guess: null argument");
  RTE_TRY(params_ready(b, "rte_rom_initial_guess"));
  if (rom->disc != b->disc) return fail(RTE_EINVAL, "ROM built on another discretisation");
  DeviceGuard g(b->disc->device);
  cudaStream_t st = (cudaStream_t)stream;
  PhaseScope ps(b, 2, st);
  RTE_TRY(rom_guess_launch(rom, b, rho0, active, st));
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  return RTE_OK;
}

extern "C" int rte_romsa_correction(rte_rom_t rom, rte_batch_t b, const double* R, double* drho,
                                    const uint8_t* active, void* stream) {
  if (!rom || !b || !R || !drho) return fail(RTE_EINVAL, "rte_romsa_correction: null argument");
  RTE_TRY(params_ready(b, "rte_romsa_correction"));
  if (rom->disc != b->disc) return fail(RTE_EINVAL, "ROM built on another discretisation");
  DeviceGuard g(b->disc->device);
  cudaStream_t st = (cudaStream_t)stream;
  RTE_TRY(rom_prepare(rom, b, st));
  return rom_correction(rom, b, R, drho, active, st);
}

// ---- persistence of the online part of a ROM ------------------------------------------------
// File layout (little-endian): magic "RTEROM03", int32 header {dim, nx, ny, n_phi, n_vz, n_mat,
// r, n_snap, n_cells, P}, double {x0, x1, y0, y1, eps_equiv}, int32 mat_id[n_cells],
// 1D only: double dx[nx] and int32 mat_id_right[nx] (mat_id again when the cross sections are
// cellwise constant), then double sv[n_snap], A0[r][r], Aa[n_mat][r][r], As[n_mat][r][r],
// a_side[4][r], U_rho[r][n_dof], U_iso[r][n_dof].
namespace {
const char kRomMagic[8] = {'R', 'T', 'E', 'R', 'O', 'M', '0', '3'};

struct FileCloser {
  FILE* f;
  ~FileCloser() {
    if (f) fclose(f);
  }
};
}  // namespace

extern "C" int rte_rom_save(rte_rom_t rom, const char* path) {
  if (!rom || !path) return fail(RTE_EINVAL, "rte_rom_save: null argument");
  const rte_disc_s* d = rom->disc;
  DeviceGuard g(d->device);
  const int r = rom->r;
  const size_t n = (size_t)r * d->n_dof;
  std::vector<double> urho(n), uiso(n), aside((size_t)4 * r);
  RTE_CUDA_TRY(cudaMemcpy(urho.data(), rom->U_rho.p, 8 * n, cudaMemcpyDeviceToHost));
  RTE_CUDA_TRY(cudaMemcpy(uiso.data(), rom->U_iso.p, 8 * n, cudaMemcpyDeviceToHost));
  RTE_CUDA_TRY(cudaMemcpy(aside.data(), rom->a_side.p, 8 * aside.size(), cudaMemcpyDeviceToHost));
  FileCloser fc{fopen(path, "wb")};
  if (!fc.f) return fail(RTE_EINVAL, std::string("rte_rom_save: cannot open ") + path);
  const int32_t hdr[10] = {d->dim, d->nx, d->ny, d->n_phi, d->n_vz, d->n_mat, r, rom->n_snap,
                           d->n_cells, d->P};
  const double geo[5] = {d->x0, d->x1, d->y0, d->y1, rom->eps_equiv};
  bool ok = fwrite(kRomMagic, 1, 8, fc.f) == 8 && fwrite(hdr, 4, 10, fc.f) == 10 &&
            fwrite(geo, 8, 5, fc.f) == 5 &&
            fwrite(d->mat_host.data(), 4, d->n_cells, fc.f) == (size_t)d->n_cells &&
            (d->dim != 1 || fwrite(d->dx.data(), 8, d->dx.size(), fc.f) == d->dx.size()) &&
            (d->dim != 1 ||
             fwrite(d->matr_host.data(), 4, d->matr_host.size(), fc.f) == d->matr_host.size()) &&
            fwrite(rom->sv.data(), 8, rom->sv.size(), fc.f) == rom->sv.size() &&
            fwrite(rom->A0.data(), 8, rom->A0.size(), fc.f) == rom->A0.size() &&
            fwrite(rom->Aa.data(), 8, rom->Aa.size(), fc.f) == rom->Aa.size() &&
            fwrite(rom->As.data(), 8, rom->As.size(), fc.f) == rom->As.size() &&
            fwrite(aside.data(), 8, aside.size(), fc.f) == aside.size() &&
            fwrite(urho.data(), 8, n, fc.f) == n && fwrite(uiso.data(), 8, n, fc.f) == n;
  if (!ok) return fail(RTE_EINVAL, std::string("rte_rom_save: write failed: ") + path);
  return RTE_OK;
}

extern "C" int rte_rom_load(rte_disc_t disc, const char* path, rte_rom_t* out) {
  if (!disc || !path || !out) return fail(RTE_EINVAL, "rte_rom_load: null argument");
  *out = nullptr;
  FileCloser fc{fopen(path, "rb")};
  if (!fc.f) return fail(RTE_EINVAL, std::string("rte_rom_load: cannot open ") + path);
  char magic[8];
  int32_t hdr[10];
  double geo[5];
  if (fread(magic, 1, 8, fc.f) != 8 || std::memcmp(magic, kRomMagic, 8) != 0 ||
      fread(hdr, 4, 10, fc.f) != 10 || fread(geo, 8, 5, fc.f) != 5)
    return fail(RTE_EINVAL, "rte_rom_load: not a ROM file");
  const rte_disc_s* d = disc;
  if (hdr[0] != d->dim || hdr[1] != d->nx || hdr[2] != d->ny || hdr[3] != d->n_phi ||
      hdr[4] != d->n_vz || hdr[5] != d->n_mat || hdr[8] != d->n_cells || hdr[9] != d->P ||
      geo[0] != d->x0 || geo[1] != d->x1 || geo[2] != d->y0 || geo[3] != d->y1)
    return fail(RTE_EINVAL, "rte_rom_load: the file was built on another discretisation");
  const int r = hdr[6], n_snap = hdr[7];
  if (r < 1 || n_snap < r || r > 4096 || n_snap > (1 << 20))
    return fail(RTE_EINVAL, "rte_rom_load: bad ROM sizes");
  std::vector<int32_t> mat(d->n_cells);
  if (fread(mat.data(), 4, mat.size(), fc.f) != mat.size() || mat != d->mat_host)
    return fail(RTE_EINVAL, "rte_rom_load: the file was built on another material map");
  if (d->dim == 1) {
    std::vector<double> dxf(d->nx);
    if (fread(dxf.data(), 8, dxf.size(), fc.f) != dxf.size() || dxf != d->dx)
      return fail(RTE_EINVAL, "rte_rom_load: the file was built on another mesh");
    std::vector<int32_t> matr(d->nx);
    if (fread(matr.data(), 4, matr.size(), fc.f) != matr.size() || matr != d->matr_host)
      return fail(RTE_EINVAL, "rte_rom_load: the file was built on another material map");
  }
  auto* rom = new rte_rom_s();
  rom->disc = disc;
  rom->r = r;
  rom->n_snap = n_snap;
  rom->eps_equiv = geo[4];
  rom->sv.resize(n_snap);
  rom->A0.resize((size_t)r * r);
  rom->Aa.resize((size_t)d->n_mat * r * r);
  rom->As.resize((size_t)d->n_mat * r * r);
  const size_t n = (size_t)r * d->n_dof;
  std::vector<double> urho(n), uiso(n), aside((size_t)4 * r);
  bool ok = fread(rom->sv.data(), 8, rom->sv.size(), fc.f) == rom->sv.size() &&
            fread(rom->A0.data(), 8, rom->A0.size(), fc.f) == rom->A0.size() &&
            fread(rom->Aa.data(), 8, rom->Aa.size(), fc.f) == rom->Aa.size() &&
            fread(rom->As.data(), 8, rom->As.size(), fc.f) == rom->As.size() &&
            fread(aside.data(), 8, aside.size(), fc.f) == aside.size() &&
            fread(urho.data(), 8, n, fc.f) == n && fread(uiso.data(), 8, n, fc.f) == n;
  if (!ok) {
    delete rom;
    return fail(RTE_EINVAL, "rte_rom_load: truncated file");
  }
  DeviceGuard g(d->device);
  int e = RTE_OK;
  auto up = [&](DevBuf<double>& buf, const std::vector<double>& h) {
    if (e != RTE_OK) return;
    e = buf.alloc(h.size());
    if (e == RTE_OK && cudaMemcpy(buf.p, h.data(), 8 * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      e = fail(RTE_ECUDA, "rte_rom_load: upload failed");
  };
  up(rom->U_rho, urho);
  up(rom->U_iso, uiso);
  up(rom->A0_dev, rom->A0);
  up(rom->Aa_dev, rom->Aa);
  up(rom->As_dev, rom->As);
  up(rom->a_side, aside);
  if (e == RTE_OK) e = rom->U_iso0.alloc((size_t)r * d->n_cells);
  if (e == RTE_OK) {
    iso0_kernel<<<(unsigned)(((size_t)r * d->n_cells + 255) / 256), 256>>>(rom->U_iso.p, r, d->n_cells,
                                                                          d->P, rom->U_iso0.p); RTE_NOTE_LAUNCH();
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
      e = fail(RTE_ECUDA, "rte_rom_load: set-up kernel failed");
  }
  if (e != RTE_OK) {
    delete rom;
    return e;
  }
  *out = rom;
  return RTE_OK;
}
