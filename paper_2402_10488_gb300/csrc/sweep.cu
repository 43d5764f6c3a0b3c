// Transport sweep fused with the scalar-flux reduction (paper Alg. 1, Eq. (transport_sweep)).
//
// 2D: upwind DG-Q^1 on a uniform Cartesian mesh.  In every cell and direction the local system
//     M a = s + E_x t_x + E_y t_y,   M = sigma_t I + a_x (K_x (x) I) + a_y (I (x) K_y)
// is solved with a per-(material, direction) table M^-1 computed once per parameter set, where
// a_x = |v_x|/h_x, K_x = [[1, s_x sqrt3], [-s_x sqrt3, 3]] (s_x the sign of v_x), s = Sigma_s rho
// + G are the cell's source moments and t_x, t_y the upwind traces
//     t_x[b] = a_{0b} + s_x sqrt3 a_{1b}   (x-outflow face, expanded along y),
//     t_y[a] = a_{a0} + s_y sqrt3 a_{a1}   (y-outflow face, expanded along x).
// On an inflow boundary t = g sqrt(h_x h_y) (isotropic inflow g, zeroth moment only).  The inflow
// couplings have two distinct entries per direction, E_x t_x = (a_x t_x0, b_x t_x0, a_x t_x1,
// b_x t_x1) and E_y t_y = (a_y t_y0, a_y t_y1, b_y t_y0, b_y t_y1) with b = -s sqrt3 a, so the
// right-hand side is formed first (8 FMA) and M^-1 applied to it (16): 32 FMA per cell and
// direction with the traces and the scalar-flux accumulation, against 40 with M^-1 E_x, M^-1 E_y
// tabulated.
//
// Parallel layout (GB300): one warp per (instance, quadrant, group of <= DPW directions).  The
// warp sweeps the mesh in blocks of H = min(32, n_x) rows; lane l owns row l of the block and
// processes column t at step s = (block)*n_x + t + l, so each step is one wavefront diagonal.
// The y-inflow comes from lane l-1 of the previous step by a register shuffle; lane 0 of the
// next row block reads the previous block's last row from a shared-memory line buffer; the
// x-inflow stays in registers.  No block-wide barrier is needed.  Each warp writes its
// omega-weighted partial scalar flux per cell; a second kernel sums the partials in a fixed
// order (deterministic) and fuses the stop-test norms.
#include "common.cuh"

namespace rte {

__device__ __forceinline__ void inv4(double m[16]) {
  // Gauss-Jordan with partial pivoting on a 4x4 row-major matrix, in place.
  double a[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 8; ++c) a[r][c] = c < 4 ? m[4 * r + c] : (c - 4 == r ? 1.0 : 0.0);
  for (int k = 0; k < 4; ++k) {
    int p = k;
    for (int r = k + 1; r < 4; ++r)
      if (fabs(a[r][k]) > fabs(a[p][k])) p = r;
    if (p != k)
      for (int c = 0; c < 8; ++c) {
        double tmp = a[k][c];
        a[k][c] = a[p][c];
        a[p][c] = tmp;
      }
    double piv = 1.0 / a[k][k];
    for (int c = 0; c < 8; ++c) a[k][c] *= piv;
    for (int r = 0; r < 4; ++r)
      if (r != k) {
        double f = a[r][k];
        for (int c = 0; c < 8; ++c) a[r][c] -= f * a[k][c];
      }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) m[4 * r + c] = a[r][c + 4];
}

// Position of instance b among the instances a launch runs (b itself without a mask).  Launches
// index their per-instance partial sums by it, so a launch needs partial-sum space only for the
// instances it runs; a batch with few running instances can then use finer direction groups.
// Called by all 32 lanes of a warp.
__device__ __forceinline__ int active_rank(const uint8_t* active, int b) {
  if (!active) return b;
  int c = 0;
  for (int i = threadIdx.x & 31; i < b; i += 32) c += active[i] != 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  return c;
}

// One thread per (instance, material, direction): the cell tables.
__global__ void tables2d_kernel(double* tables, const double* sigma_t, const double* dirs,
                                int B, int n_mat, int n_dirs, double hx, double hy,
                                const uint8_t* mask) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * n_mat * n_dirs) return;
  const int d = idx % n_dirs;
  const int m = (idx / n_dirs) % n_mat;
  const int b = idx / (n_dirs * n_mat);
  if (mask && !mask[b]) return;
  const double st = sigma_t[b * n_mat + m];
  const double vx = dirs[4 * d], vy = dirs[4 * d + 1];
  const double s3 = sqrt(3.0);
  const double sx = vx < 0 ? -1.0 : 1.0, sy = vy < 0 ? -1.0 : 1.0;
  const double ax = fabs(vx) / hx, ay = fabs(vy) / hy;
  const double K[2][2][2] = {{{1.0, sx * s3}, {-sx * s3, 3.0}}, {{1.0, sy * s3}, {-sy * s3, 3.0}}};
  double M[16];
  for (int bb = 0; bb < 2; ++bb)
    for (int aa = 0; aa < 2; ++aa)
      for (int b2 = 0; b2 < 2; ++b2)
        for (int a2 = 0; a2 < 2; ++a2) {
          double v = 0.0;
          if (aa == a2 && bb == b2) v += st;
          if (bb == b2) v += ax * K[0][aa][a2];
          if (aa == a2) v += ay * K[1][bb][b2];
          M[4 * (aa + 2 * bb) + (a2 + 2 * b2)] = v;
        }
  inv4(M);
  double* T = tables + (size_t)idx * kTab2D;
  for (int k = 0; k < 16; ++k) T[k] = M[k];
}

// Per-direction inflow couplings of the 2D cell solve (see the file header): a = |v|/h and
// b = -s sqrt3 a along x and y.
struct InflowCoef {
  double ax, bx, ay, by;
};
__device__ __forceinline__ InflowCoef inflow_coef(const double* dirs, int d, double ihx, double ihy) {
  const double s3 = 1.7320508075688772;
  const double vx = dirs[4 * d], vy = dirs[4 * d + 1];
  InflowCoef c;
  c.ax = fabs(vx) * ihx;
  c.ay = fabs(vy) * ihy;
  c.bx = (vx < 0 ? s3 : -s3) * c.ax;
  c.by = (vy < 0 ? s3 : -s3) * c.ay;
  return c;
}

// One cell of one direction: a = M^-1 (s + E_x t_x + E_y t_y), T the direction's M^-1 (row-major).
__device__ __forceinline__ void cell_solve(const double* T, const InflowCoef& e, double s0, double s1,
                                           double s2, double s3v, const double tx[2],
                                           const double ty[2], double a[4]) {
  const double r0 = fma(e.ay, ty[0], fma(e.ax, tx[0], s0));
  const double r1 = fma(e.ay, ty[1], fma(e.bx, tx[0], s1));
  const double r2 = fma(e.by, ty[0], fma(e.ax, tx[1], s2));
  const double r3 = fma(e.by, ty[1], fma(e.bx, tx[1], s3v));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 m01 = reinterpret_cast<const double2*>(T + 4 * k)[0];
    const double2 m23 = reinterpret_cast<const double2*>(T + 4 * k)[1];
    a[k] = fma(m23.y, r3, fma(m23.x, r2, fma(m01.y, r1, m01.x * r0)));
  }
}

// One thread per (instance, cell, direction), 1D: M = Sigma_t + (|xi|/h) [[1, s sqrt3],
// [-s sqrt3, 3]] (s the sign of xi, h the cell's width; Sigma_t = sigma_t I, or the 2x2 of
// linear_sigma when the cross sections are linear across cells) and the inflow coupling: a unit
// face value u entering the cell contributes |xi| u phi_k(inflow face) = (|xi| / sqrt h)
// (1, -s sqrt3) to the right-hand side.  T = {M^-1 (2x2), M^-1 (|xi| / sqrt h)(1, -s sqrt3),
// 1 / sqrt h}.
__global__ void tables1d_kernel(double* tables, const double* sigma_t, const double* dirs, int B,
                                int n_mat, int n_cells, int n_dirs, const int32_t* mat,
                                const int32_t* matr, const double* dx, const uint8_t* mask) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * n_cells * n_dirs) return;
  const int d = idx % n_dirs;
  const int c = (idx / n_dirs) % n_cells;
  const int b = idx / (n_dirs * n_cells);
  if (mask && !mask[b]) return;
  double st = sigma_t[b * n_mat + mat[c]], to = 0.0;
  if (matr) linear_sigma(st, sigma_t[b * n_mat + matr[c]], st, to);
  const double xi = dirs[4 * d], h = dx[c];
  const double s3 = sqrt(3.0), sg = xi < 0 ? -1.0 : 1.0, a = fabs(xi) / h;
  const double m00 = st + a, m01 = to + a * sg * s3, m10 = to - a * sg * s3, m11 = st + 3.0 * a;
  const double det = m00 * m11 - m01 * m10;
  const double i00 = m11 / det, i01 = -m01 / det, i10 = -m10 / det, i11 = m00 / det;
  const double q = 1.0 / sqrt(h), e0 = fabs(xi) * q, e1 = -sg * s3 * fabs(xi) * q;
  double* T = tables + (size_t)idx * kTab1D;
  T[0] = i00, T[1] = i01, T[2] = i10, T[3] = i11;
  T[4] = i00 * e0 + i01 * e1;
  T[5] = i10 * e0 + i11 * e1;
  T[6] = q;
  T[7] = 0.0;
}


// With LEAK the kernel also records, per cell, sum over its directions of
//     omega_j ( |v_x| int_{x-outflow face} f - |v_x| int_{x-inflow face} f + the same along y ),
// the net upwind outflow that enters the cell's particle balance (the DG equation tested with the
// cell's indicator function): with t the face traces above, int_face f = t[0] sqrt(h_face / h_n),
// h_n the cell's extent normal to the face.
// One warp sweeps direction group g of instance b (the body of sweep2d_kernel and of the
// work-queue sweep over several batches, sweep2d_multi_kernel).
template <int DPW, bool SMEM_TAB, bool PRESRC, bool LEAK>
__device__ __forceinline__ void sweep2d_warp(const Sweep2DArgs& A, int g, int b) {
  const int lane = threadIdx.x & 31;
  if (A.active && !A.active[b]) return;
  const SweepGroup grp = A.groups[g];
  const bool xneg = grp.quad & 1, yneg = (grp.quad & 2) != 0;
  extern __shared__ double smem[];
  double* ybuf = smem;                                   // [nx][DPW][2]
  double* tab_s = smem + (size_t)A.nx * DPW * 2;         // [n_mat][DPW][32]
  double* sig_s = tab_s + (SMEM_TAB ? A.n_mat * DPW * kTab2D : 0);
  const double* __restrict__ tabg = A.tables + (size_t)b * A.n_mat * A.n_dirs * kTab2D;
  if (SMEM_TAB) {
    for (int e = lane; e < A.n_mat * DPW * kTab2D; e += 32) {
      const int m = e / (DPW * kTab2D), r = e % (DPW * kTab2D), dd = r / kTab2D, k = r % kTab2D;
      tab_s[e] = dd < grp.nd ? tabg[((size_t)m * A.n_dirs + grp.d0 + dd) * kTab2D + k] : 0.0;
    }
  }
  for (int m = lane; m < A.n_mat; m += 32) sig_s[m] = A.sigma_s[(size_t)b * A.n_mat + m];
  __syncwarp();

  double w[DPW];
  InflowCoef ec[DPW];
#pragma unroll
  for (int dd = 0; dd < DPW; ++dd) {
    w[dd] = dd < grp.nd ? A.dirs[4 * (grp.d0 + dd) + 2] : 0.0;
    ec[dd] = inflow_coef(A.dirs, grp.d0 + (dd < grp.nd ? dd : 0), A.ihx, A.ihy);
  }
  const double s3 = sqrt(3.0);
  const double c3x = xneg ? -s3 : s3, c3y = yneg ? -s3 : s3;
  const double gxb = A.with_source ? A.inflow[4 * b + (xneg ? 1 : 0)] * A.sq_area : 0.0;
  const double gyb = A.with_source ? A.inflow[4 * b + (yneg ? 3 : 2)] * A.sq_area : 0.0;
  const int H = A.nx < 32 ? A.nx : 32;
  const int nrb = (A.ny + H - 1) / H;
  const int total = nrb * A.nx;
  const double* __restrict__ rin = A.rho_in + (size_t)b * A.n_dof;
  const double* __restrict__ G0 = A.G0 + (size_t)b * A.n_cells;
  double* part = A.partial + ((size_t)active_rank(A.active, b) * A.n_groups + g) * A.n_dof;
  double* psi = A.psi_out ? A.psi_out + ((size_t)b * A.n_dirs + grp.d0) * A.n_dof : nullptr;

  double tx[DPW][2], typ[DPW][2];
#pragma unroll
  for (int dd = 0; dd < DPW; ++dd) tx[dd][0] = tx[dd][1] = typ[dd][0] = typ[dd][1] = 0.0;
  double lkx[DPW], lky[DPW];
  double* lkp = nullptr;
  if (LEAK) {
#pragma unroll
    for (int dd = 0; dd < DPW; ++dd) {
      lkx[dd] = dd < grp.nd ? w[dd] * fabs(A.dirs[4 * (grp.d0 + dd)]) * A.lx : 0.0;
      lky[dd] = dd < grp.nd ? w[dd] * fabs(A.dirs[4 * (grp.d0 + dd) + 1]) * A.ly : 0.0;
    }
    lkp = A.leak + ((size_t)active_rank(A.active, b) * A.n_groups + g) * A.n_cells;
  }

  for (int s = 0; s < total + H - 1; ++s) {
    const int u = s - lane;
    const bool inrange = lane < H && u >= 0 && u < total;
    const int rb = inrange ? u / A.nx : 0;
    const int t = inrange ? u - rb * A.nx : 0;
    const int r = rb * H + lane;
    const bool act = inrange && r < A.ny;
    double ty[DPW][2];
#pragma unroll
    for (int dd = 0; dd < DPW; ++dd) {
      ty[dd][0] = __shfl_up_sync(0xffffffffu, typ[dd][0], 1);
      ty[dd][1] = __shfl_up_sync(0xffffffffu, typ[dd][1], 1);
    }
    if (act) {
      if (r == 0) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) ty[dd][0] = gyb, ty[dd][1] = 0.0;
      } else if (lane == 0) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) {
          ty[dd][0] = ybuf[(t * DPW + dd) * 2];
          ty[dd][1] = ybuf[(t * DPW + dd) * 2 + 1];
        }
      }
      if (t == 0) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) tx[dd][0] = gxb, tx[dd][1] = 0.0;
      }
      const int i = xneg ? A.nx - 1 - t : t;
      const int j = yneg ? A.ny - 1 - r : r;
      const int c = j * A.nx + i;
      const int m = A.mat[c];
      const double2 r01 = reinterpret_cast<const double2*>(rin + 4 * (size_t)c)[0];
      const double2 r23 = reinterpret_cast<const double2*>(rin + 4 * (size_t)c)[1];
      double s0, s1, s2, s3v;
      if (PRESRC) {  // sources formed once per sweep by cell_source_kernel
        s0 = r01.x, s1 = r01.y, s2 = r23.x, s3v = r23.y;
      } else {
        const double ss = sig_s[m];
        s0 = fma(ss, r01.x, A.with_source ? G0[c] : 0.0);
        s1 = ss * r01.y, s2 = ss * r23.x, s3v = ss * r23.y;
      }
      double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0, lk = 0.0;
#pragma unroll
      for (int dd = 0; dd < DPW; ++dd) {
        if (dd < grp.nd) {
          const double* T = SMEM_TAB ? tab_s + (m * DPW + dd) * kTab2D
                                     : tabg + ((size_t)m * A.n_dirs + grp.d0 + dd) * kTab2D;
          double a[4];
          cell_solve(T, ec[dd], s0, s1, s2, s3v, tx[dd], ty[dd], a);
          const double txin = tx[dd][0];
          tx[dd][0] = fma(c3x, a[1], a[0]);
          tx[dd][1] = fma(c3x, a[3], a[2]);
          typ[dd][0] = fma(c3y, a[2], a[0]);
          typ[dd][1] = fma(c3y, a[3], a[1]);
          if (LEAK) lk = fma(lkx[dd], tx[dd][0] - txin, fma(lky[dd], typ[dd][0] - ty[dd][0], lk));
          acc0 = fma(w[dd], a[0], acc0);
          acc1 = fma(w[dd], a[1], acc1);
          acc2 = fma(w[dd], a[2], acc2);
          acc3 = fma(w[dd], a[3], acc3);
          if (psi) {
            double2* p = reinterpret_cast<double2*>(psi + (size_t)dd * A.n_dof + 4 * (size_t)c);
            p[0] = make_double2(a[0], a[1]);
            p[1] = make_double2(a[2], a[3]);
          }
        }
      }
      double2* po = reinterpret_cast<double2*>(part + 4 * (size_t)c);
      po[0] = make_double2(acc0, acc1);
      po[1] = make_double2(acc2, acc3);
      if (LEAK) lkp[c] = lk;
      if (lane == H - 1 && rb + 1 < nrb) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) {
          ybuf[(t * DPW + dd) * 2] = typ[dd][0];
          ybuf[(t * DPW + dd) * 2 + 1] = typ[dd][1];
        }
      }
    }
    __syncwarp();
  }
}

template <int DPW, bool SMEM_TAB, bool PRESRC = false, bool LEAK = false>
__global__ void __launch_bounds__(32) sweep2d_kernel(const Sweep2DArgs A) {
  sweep2d_warp<DPW, SMEM_TAB, PRESRC, LEAK>(A, blockIdx.x, blockIdx.y);
}

// One sweep of several batches (different meshes and quadratures) in one launch: a persistent grid
// of one-warp blocks takes work items (batch, instance, direction group) from a shared counter in
// the order of the list -- longest sweeps first, so that the launch's tail is short -- and sweeps
// each with the batch's own arguments.  Every item writes only its own partial sums, so the result
// does not depend on which warp took which item.  The shared memory is sized for the largest batch.

template <int DPW>
__global__ void __launch_bounds__(32) sweep2d_multi_kernel(const Sweep2DArgs* __restrict__ descs,
                                                           const SweepItem* __restrict__ items,
                                                           int n_items, int* counter) {
  const int lane = threadIdx.x;
  for (;;) {
    int i = 0;
    if (lane == 0) i = atomicAdd(counter, 1);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= n_items) return;
    const SweepItem it = items[i];
    const Sweep2DArgs A = descs[it.batch];
    sweep2d_warp<DPW, true, true, false>(A, it.group, it.inst);
    __syncwarp();   // the next item restages the shared memory
  }
}

// Multi-warp variant for launches with too few (instance, group) pairs to give every SM
// sub-partition a warp (the last iterations of a batch, a lone large request): NW warps of one CTA
// share the row blocks of one direction group, warp w taking blocks w, w + NW, ...  Block rb starts
// D steps after block rb - 1 (KBA-style pipelining); lane 0 of block rb reads the last row of
// block rb - 1, written by another warp at least kKbaChunk + 1 steps earlier, and every warp passes
// a block barrier every kKbaChunk steps, so that row is visible when read (no flags, no waits other
// than the barriers, which every thread reaches the same number of times).  Blocks alternate
// between two line buffers.  D >= H + kKbaChunk, and NW * D >= nx + H - 1 so that a warp has
// finished a block before its next one starts.  Sources are the precomputed cell sources.
constexpr int kKbaChunk = 8;

template <int DPW, bool SMEM_TAB>
__global__ void __launch_bounds__(256) sweep2d_kba_kernel(const Sweep2DArgs A, int D) {
  const int g = blockIdx.x, b = blockIdx.y;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, NW = blockDim.x >> 5;
  if (A.active && !A.active[b]) return;  // uniform over the CTA, before any barrier
  const SweepGroup grp = A.groups[g];
  const bool xneg = grp.quad & 1, yneg = (grp.quad & 2) != 0;
  extern __shared__ double smem[];
  double* ybuf = smem;                                       // [2][nx][DPW][2]
  double* tab_s = smem + 2 * (size_t)A.nx * DPW * 2;         // [n_mat][DPW][32]
  const double* __restrict__ tabg = A.tables + (size_t)b * A.n_mat * A.n_dirs * kTab2D;
  if (SMEM_TAB) {
    for (int e = threadIdx.x; e < A.n_mat * DPW * kTab2D; e += blockDim.x) {
      const int m = e / (DPW * kTab2D), r = e % (DPW * kTab2D), dd = r / kTab2D, k = r % kTab2D;
      tab_s[e] = dd < grp.nd ? tabg[((size_t)m * A.n_dirs + grp.d0 + dd) * kTab2D + k] : 0.0;
    }
  }
  __syncthreads();
  double w[DPW];
  InflowCoef ec[DPW];
#pragma unroll
  for (int dd = 0; dd < DPW; ++dd) {
    w[dd] = dd < grp.nd ? A.dirs[4 * (grp.d0 + dd) + 2] : 0.0;
    ec[dd] = inflow_coef(A.dirs, grp.d0 + (dd < grp.nd ? dd : 0), A.ihx, A.ihy);
  }
  const double s3 = sqrt(3.0);
  const double c3x = xneg ? -s3 : s3, c3y = yneg ? -s3 : s3;
  const double gxb = A.with_source ? A.inflow[4 * b + (xneg ? 1 : 0)] * A.sq_area : 0.0;
  const double gyb = A.with_source ? A.inflow[4 * b + (yneg ? 3 : 2)] * A.sq_area : 0.0;
  const int H = A.nx < 32 ? A.nx : 32;
  const int nrb = (A.ny + H - 1) / H;
  const int steps = (nrb - 1) * D + A.nx + H - 1;
  const int padded = (steps + kKbaChunk - 1) / kKbaChunk * kKbaChunk;
  const double* __restrict__ S = A.rho_in + (size_t)b * A.n_dof;
  double* part = A.partial + ((size_t)active_rank(A.active, b) * A.n_groups + g) * A.n_dof;
  double* psi = A.psi_out ? A.psi_out + ((size_t)b * A.n_dirs + grp.d0) * A.n_dof : nullptr;
  double tx[DPW][2], typ[DPW][2];
#pragma unroll
  for (int dd = 0; dd < DPW; ++dd) tx[dd][0] = tx[dd][1] = typ[dd][0] = typ[dd][1] = 0.0;
  for (int s = 0; s < padded; ++s) {
    int rb = -1, u = -1;
    if (s >= wid * D) {
      rb = wid + NW * ((s - wid * D) / (NW * D));
      u = s - rb * D - lane;
    }
    const bool inrange = lane < H && rb >= 0 && rb < nrb && u >= 0 && u < A.nx;
    const int t = inrange ? u : 0;
    const int r = rb * H + lane;
    const bool act = inrange && r < A.ny;
    double ty[DPW][2];
#pragma unroll
    for (int dd = 0; dd < DPW; ++dd) {
      ty[dd][0] = __shfl_up_sync(0xffffffffu, typ[dd][0], 1);
      ty[dd][1] = __shfl_up_sync(0xffffffffu, typ[dd][1], 1);
    }
    if (act) {
      if (r == 0) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) ty[dd][0] = gyb, ty[dd][1] = 0.0;
      } else if (lane == 0) {
        const double* yb = ybuf + (size_t)((rb - 1) & 1) * A.nx * DPW * 2;
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) {
          ty[dd][0] = yb[(t * DPW + dd) * 2];
          ty[dd][1] = yb[(t * DPW + dd) * 2 + 1];
        }
      }
      if (t == 0) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) tx[dd][0] = gxb, tx[dd][1] = 0.0;
      }
      const int i = xneg ? A.nx - 1 - t : t;
      const int j = yneg ? A.ny - 1 - r : r;
      const int c = j * A.nx + i;
      const int m = A.mat[c];
      const double2 r01 = reinterpret_cast<const double2*>(S + 4 * (size_t)c)[0];
      const double2 r23 = reinterpret_cast<const double2*>(S + 4 * (size_t)c)[1];
      const double s0 = r01.x, s1 = r01.y, s2 = r23.x, s3v = r23.y;
      double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
#pragma unroll
      for (int dd = 0; dd < DPW; ++dd) {
        if (dd < grp.nd) {
          const double* T = SMEM_TAB ? tab_s + (m * DPW + dd) * kTab2D
                                     : tabg + ((size_t)m * A.n_dirs + grp.d0 + dd) * kTab2D;
          double a[4];
          cell_solve(T, ec[dd], s0, s1, s2, s3v, tx[dd], ty[dd], a);
          tx[dd][0] = fma(c3x, a[1], a[0]);
          tx[dd][1] = fma(c3x, a[3], a[2]);
          typ[dd][0] = fma(c3y, a[2], a[0]);
          typ[dd][1] = fma(c3y, a[3], a[1]);
          acc0 = fma(w[dd], a[0], acc0);
          acc1 = fma(w[dd], a[1], acc1);
          acc2 = fma(w[dd], a[2], acc2);
          acc3 = fma(w[dd], a[3], acc3);
          if (psi) {
            double2* p = reinterpret_cast<double2*>(psi + (size_t)dd * A.n_dof + 4 * (size_t)c);
            p[0] = make_double2(a[0], a[1]);
            p[1] = make_double2(a[2], a[3]);
          }
        }
      }
      double2* po = reinterpret_cast<double2*>(part + 4 * (size_t)c);
      po[0] = make_double2(acc0, acc1);
      po[1] = make_double2(acc2, acc3);
      if (lane == H - 1 && rb + 1 < nrb) {
        double* yb = ybuf + (size_t)(rb & 1) * A.nx * DPW * 2;
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) {
          yb[(t * DPW + dd) * 2] = typ[dd][0];
          yb[(t * DPW + dd) * 2 + 1] = typ[dd][1];
        }
      }
    }
    __syncwarp();
    if ((s + 1) % kKbaChunk == 0) __syncthreads();
  }
}

// S = Sigma_s rho + G (zeroth moment only; G omitted without source): the right-hand side shared
// by all directions of a sweep, formed once per cell instead of once per direction warp.
__global__ void cell_source_kernel(const double* __restrict__ rho, double* S,
                                   const double* __restrict__ sigma_s, const double* __restrict__ G0,
                                   const int32_t* __restrict__ mat, const uint8_t* active,
                                   int n_cells, int n_mat, int with_source) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const double ss = sigma_s[(size_t)b * n_mat + mat[c]];
  const double2* r = reinterpret_cast<const double2*>(rho + ((size_t)b * n_cells + c) * 4);
  const double2 a = r[0], e = r[1];
  double2* o = reinterpret_cast<double2*>(S + ((size_t)b * n_cells + c) * 4);
  o[0] = make_double2(fma(ss, a.x, with_source ? G0[(size_t)b * n_cells + c] : 0.0), ss * a.y);
  o[1] = make_double2(ss * e.x, ss * e.y);
}

struct Sweep1DArgs {
  const double* rho_in;
  double* partial;
  double* psi_out;
  const uint8_t* active;
  const double* tables;
  const double* sigma_s;
  const double* G0;
  const double* inflow;
  const int32_t* mat;
  const int32_t* matr;      // material at each cell's right end (linear cross sections) or null
  const double* dirs;
  int B, nx, n_dof, n_mat, n_dirs, with_source;
  double* leak = nullptr;   // or [rank][n_dirs][nx]: omega |xi| (u_out - u_in) per cell (balance)
};

// 1D slab: one thread per (instance, direction), sequential in upwind order (2x2 cell solves).
// The carried quantity is the angular flux's value u at the face between two cells (the inflow
// value g at the boundary); per-cell tables hold the cell width's effect.
__global__ void sweep1d_kernel(const Sweep1DArgs A) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= A.B * A.n_dirs) return;
  const int b = idx / A.n_dirs, d = idx % A.n_dirs;
  if (A.active && !A.active[b]) return;
  const double xi = A.dirs[4 * d], w = A.dirs[4 * d + 2];
  const bool neg = xi < 0;
  const double c3 = neg ? -sqrt(3.0) : sqrt(3.0);
  double u = A.with_source ? A.inflow[4 * b + (neg ? 1 : 0)] : 0.0;
  const double* rin = A.rho_in + (size_t)b * A.n_dof;
  int rank = b;
  if (A.active) {
    rank = 0;
    for (int i = 0; i < b; ++i) rank += A.active[i] != 0;
  }
  double* part = A.partial + ((size_t)rank * A.n_dirs + d) * A.n_dof;
  double* psi = A.psi_out ? A.psi_out + ((size_t)b * A.n_dirs + d) * A.n_dof : nullptr;
  const double* tab = A.tables + (size_t)b * A.nx * A.n_dirs * kTab1D;
  for (int step = 0; step < A.nx; ++step) {
    const int c = neg ? A.nx - 1 - step : step;
    const int m = A.mat[c];
    const double* T = tab + ((size_t)c * A.n_dirs + d) * kTab1D;
    const double ss = A.sigma_s[(size_t)b * A.n_mat + m];
    const double g0 = A.with_source ? A.G0[(size_t)b * A.nx + c] : 0.0;
    double s0, s1;
    if (A.matr) {   // Sigma_s = [[sb, so], [so, sb]]
      double sb, so;
      linear_sigma(ss, A.sigma_s[(size_t)b * A.n_mat + A.matr[c]], sb, so);
      s0 = fma(sb, rin[2 * c], fma(so, rin[2 * c + 1], g0));
      s1 = fma(so, rin[2 * c], sb * rin[2 * c + 1]);
    } else {
      s0 = fma(ss, rin[2 * c], g0);
      s1 = ss * rin[2 * c + 1];
    }
    const double a0 = fma(T[4], u, fma(T[1], s1, T[0] * s0));
    const double a1 = fma(T[5], u, fma(T[3], s1, T[2] * s0));
    const double uin = u;
    u = fma(c3, a1, a0) * T[6];
    part[2 * c] = w * a0;
    part[2 * c + 1] = w * a1;
    if (psi) psi[2 * c] = a0, psi[2 * c + 1] = a1;
    if (A.leak) A.leak[((size_t)rank * A.n_dirs + d) * A.nx + c] = w * fabs(xi) * (u - uin);
  }
}

// rho_out = sum of the group partials (fixed order); optional stop-test norms per instance.
// |x| as the bit pattern of a non-negative double: such patterns order like the values, so the
// stop-test maxima are taken with integer max on the ALU instead of FP64 min/max instructions (a
// NaN orders above +inf and so shows up in the norm).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

// Block-wide maxima of (dmax, rmax) as bit patterns, folded into norms[2b], norms[2b + 1].
__device__ __forceinline__ void block_norms(unsigned long long dmax, unsigned long long rmax,
                                            unsigned long long* norms, int b) {
  for (int o = 16; o > 0; o >>= 1) {
    dmax = umax64(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    rmax = umax64(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  }
  __shared__ unsigned long long sd[32], sr[32];
  const int wid = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (ln == 0) sd[wid] = dmax, sr[wid] = rmax;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    dmax = ln < nw ? sd[ln] : 0ull;
    rmax = ln < nw ? sr[ln] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      dmax = umax64(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      rmax = umax64(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    }
    if (ln == 0) {
      atomicMax(norms + 2 * b, dmax);
      atomicMax(norms + 2 * b + 1, rmax);
    }
  }
}

// With R (2D, P = 4 moments per cell) the same pass also forms the correction source
// R = sigma_s (rho_out - rho_in) of every swept instance, as correction_source_kernel does.
__global__ void reduce_partials_kernel(const double* __restrict__ partial,
                                       const double* __restrict__ rho_in, double* rho_out,
                                       unsigned long long* norms, const uint8_t* active,
                                       int n_groups, int n_dof, double* R = nullptr,
                                       const double* __restrict__ sigma_s = nullptr,
                                       const int32_t* __restrict__ mat = nullptr, int n_mat = 0) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int rank = active_rank(active, b);
  const int e = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  unsigned long long dmax = 0ull, rmax = 0ull;
  if (e < n_dof) {
    const double* p = partial + (size_t)rank * n_groups * n_dof + e;
    double2 acc = reinterpret_cast<const double2*>(p)[0];
    for (int g = 1; g < n_groups; ++g) {
      const double2 v = reinterpret_cast<const double2*>(p + (size_t)g * n_dof)[0];
      acc.x += v.x;
      acc.y += v.y;
    }
    reinterpret_cast<double2*>(rho_out + (size_t)b * n_dof + e)[0] = acc;
    if (norms || R) {
      const double2 ri = reinterpret_cast<const double2*>(rho_in + (size_t)b * n_dof + e)[0];
      if (norms) {
        dmax = umax64(abs_bits(acc.x - ri.x), abs_bits(acc.y - ri.y));
        rmax = umax64(abs_bits(acc.x), abs_bits(acc.y));
      }
      if (R) {
        const double ss = sigma_s[(size_t)b * n_mat + mat[e / 4]];
        reinterpret_cast<double2*>(R + (size_t)b * n_dof + e)[0] =
            make_double2(ss * (acc.x - ri.x), ss * (acc.y - ri.y));
      }
    }
  }
  if (!norms) return;
  block_norms(dmax, rmax, norms, b);
}

__global__ void change_norm_kernel(const double* __restrict__ rs, const double* __restrict__ rp,
                                   unsigned long long* norms, int n_dof) {
  const int b = blockIdx.y;
  double dmax = 0.0, rmax = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_dof; e += gridDim.x * blockDim.x) {
    const double a = rs[(size_t)b * n_dof + e], c = rp[(size_t)b * n_dof + e];
    dmax = fmax(dmax, fabs(a - c));
    rmax = fmax(rmax, fabs(a));
  }
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(norms + 2 * b, (unsigned long long)__double_as_longlong(dmax));
    atomicMax(norms + 2 * b + 1, (unsigned long long)__double_as_longlong(rmax));
  }
}

__global__ void bits_to_double_kernel(const unsigned long long* bits, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __longlong_as_double((long long)bits[i]);
}

// R = Sigma_s (rho_star - rho_prev), cellwise-constant sigma_s (orthonormal basis).
__global__ void correction_source_kernel(const double* rs, const double* rp, double* R,
                                         const double* sigma_s, const int32_t* mat,
                                         const uint8_t* active, int n_dof, int P, int n_mat) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_dof; e += gridDim.x * blockDim.x) {
    const size_t o = (size_t)b * n_dof + e;
    R[o] = sigma_s[(size_t)b * n_mat + mat[e / P]] * (rs[o] - rp[o]);
  }
}

// The same in 1D with sigma_s linear across cells: one thread per cell applies the 2x2 of
// linear_sigma (both moments read before either is written, so R may alias rs or rp).
__global__ void correction_source1d_linear_kernel(const double* rs, const double* rp, double* R,
                                                  const double* sigma_s, const int32_t* mat,
                                                  const int32_t* matr, const uint8_t* active,
                                                  int nx, int n_mat) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nx; c += gridDim.x * blockDim.x) {
    const size_t o = (size_t)b * 2 * nx + 2 * c;
    double sb, so;
    linear_sigma(sigma_s[(size_t)b * n_mat + mat[c]], sigma_s[(size_t)b * n_mat + matr[c]], sb, so);
    const double d0 = rs[o] - rp[o], d1 = rs[o + 1] - rp[o + 1];
    R[o] = fma(sb, d0, so * d1);
    R[o + 1] = fma(so, d0, sb * d1);
  }
}

__global__ void add_kernel(const double* x, const double* y, double* out, const uint8_t* active,
                           int n_dof) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_dof; e += gridDim.x * blockDim.x) {
    const size_t o = (size_t)b * n_dof + e;
    out[o] = y ? x[o] + y[o] : x[o];
  }
}

// ---- host side ----------------------------------------------------------------------------

int setup_tables(rte_batch_t bt, cudaStream_t st, const uint8_t* mask) {
  const rte_disc_s* d = bt->disc;
  const int n = bt->B * d->n_mat * d->n_dirs;
  const int th = 128, bl = (n + th - 1) / th;
  if (d->dim == 2) {
    tables2d_kernel<<<bl, th, 0, st>>>(bt->tables.p, bt->sigma_t.p, d->dir_dev.p, bt->B, d->n_mat,
                                       d->n_dirs, d->hx, d->hy, mask); RTE_NOTE_LAUNCH();
  } else {
    const int n1 = bt->B * d->n_cells * d->n_dirs;
    tables1d_kernel<<<(n1 + th - 1) / th, th, 0, st>>>(bt->tables.p, bt->sigma_t.p, d->dir_dev.p,
                                                       bt->B, d->n_mat, d->n_cells, d->n_dirs,
                                                       d->mat_id.p, d->mat_r.p, d->dx_dev.p,
                                                       mask); RTE_NOTE_LAUNCH();
  }
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

template <int DPW, bool PRESRC = false, bool LEAK = false>
static int launch2d(const Sweep2DArgs& A, int B, int n_groups, cudaStream_t st) {
  const size_t ybytes = (size_t)A.nx * DPW * 2 * sizeof(double);
  const size_t tbytes = (size_t)A.n_mat * DPW * kTab2D * sizeof(double);
  const size_t sbytes = (size_t)A.n_mat * sizeof(double);
  dim3 grid(n_groups, B);
  if (ybytes + tbytes + sbytes <= 48 * 1024) {
    sweep2d_kernel<DPW, true, PRESRC, LEAK><<<grid, 32, ybytes + tbytes + sbytes, st>>>(A); RTE_NOTE_LAUNCH();
  } else {
    const size_t bytes = ybytes + sbytes;
    if (bytes > 200 * 1024) return fail(RTE_EINVAL, "sweep: mesh row too long for shared memory");
    if (bytes > 48 * 1024) {
      RTE_CUDA_TRY(cudaFuncSetAttribute(sweep2d_kernel<DPW, false, PRESRC, LEAK>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    }
    sweep2d_kernel<DPW, false, PRESRC, LEAK><<<grid, 32, bytes, st>>>(A); RTE_NOTE_LAUNCH();
  }
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

template <int DPW>
static int launch2d_kba(const Sweep2DArgs& A, int B, int n_groups, int NW, int D, cudaStream_t st) {
  const size_t ybytes = 2 * (size_t)A.nx * DPW * 2 * sizeof(double);
  const size_t tbytes = (size_t)A.n_mat * DPW * kTab2D * sizeof(double);
  dim3 grid(n_groups, B);
  if (ybytes + tbytes <= 48 * 1024) {
    sweep2d_kba_kernel<DPW, true><<<grid, 32 * NW, ybytes + tbytes, st>>>(A, D); RTE_NOTE_LAUNCH();
  } else {
    if (ybytes > 200 * 1024) return fail(RTE_EINVAL, "sweep: mesh row too long for shared memory");
    if (ybytes > 48 * 1024)
      RTE_CUDA_TRY(cudaFuncSetAttribute(sweep2d_kba_kernel<DPW, false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ybytes));
    sweep2d_kba_kernel<DPW, false><<<grid, 32 * NW, ybytes, st>>>(A, D); RTE_NOTE_LAUNCH();
  }
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

// Steps of the pipelined sweep with NW warps per direction group (D as in sweep_launch).
static int kba_steps(int nx, int ny, int NW) {
  const int H = nx < 32 ? nx : 32;
  const int nrb = (ny + H - 1) / H;
  const int D = std::max(H + kKbaChunk, (nx + H - 1 + NW - 1) / NW);
  return (nrb - 1) * D + nx + H - 1;
}

// Warps per direction group for a launch (one CTA per group).  Cost model: the launch takes the
// pipelined sweep's steps times the warps sharing the busiest SM sub-partition's FP64 unit, with
// the CTAs spread evenly over the SMs (ceil(ctas / n_sm) on the busiest) and each SM's warps over
// its four sub-partitions.  More than one warp only when that cost is at least 10% below one warp
// walking all row blocks, and no more warps than row blocks.
static int kba_warps(const rte_disc_s* d, int n_sm, long long ctas) {
  const int H = d->nx < 32 ? d->nx : 32;
  const int nrb = (d->ny + H - 1) / H;
  if (nrb < 2 || ctas <= 0) return 1;
  const long long per_sm = (ctas + n_sm - 1) / n_sm;
  const long long single = (long long)(nrb * d->nx + H - 1) * ((per_sm + 3) / 4);
  int best = 1;
  long long best_cost = single;
  for (int nw = 2; nw <= std::min(nrb, 8); ++nw) {
    const long long cost = (long long)kba_steps(d->nx, d->ny, nw) * ((per_sm * nw + 3) / 4);
    if (cost < best_cost) best = nw, best_cost = cost;
  }
  return best_cost < 0.9 * single ? best : 1;
}

// Records bt->started_ev (when set) on the sweep's stream and clears it (see rte_batch_s).
static int note_started(rte_batch_t bt, cudaStream_t st) {
  if (!bt->started_ev) return RTE_OK;
  RTE_CUDA_TRY(cudaEventRecord(bt->started_ev, st));
  bt->started_ev = nullptr;
  return RTE_OK;
}

int sweep_launch(rte_batch_t bt, const double* rho_in, double* rho_out, double* psi_out,
                 int with_source, const uint8_t* active, cudaStream_t st, bool fuse_norms,
                 int n_active, bool zero_norms) {
  if (n_active < 0) n_active = bt->B;
  const rte_disc_s* d = bt->disc;
  int dpw = bt->dpw, n_groups = 0;
  const SweepGroup* gdev = nullptr;
  pick_groups(bt, n_active, &dpw, &n_groups, &gdev);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (bt->timing) {
    RTE_CUDA_TRY(cudaEventCreate(&ev0));
    RTE_CUDA_TRY(cudaEventCreate(&ev1));
    RTE_CUDA_TRY(cudaEventRecord(ev0, st));
  }
  if (d->dim == 2) {
    cell_source_kernel<<<dim3((d->n_cells + 127) / 128, bt->B), 128, 0, st>>>(
        rho_in, bt->S.p, bt->sigma_s.p, bt->G0.p, d->mat_id.p, active, d->n_cells, d->n_mat,
        with_source); RTE_NOTE_LAUNCH();
    RTE_TRY(note_started(bt, st));
    Sweep2DArgs A{bt->S.p,      bt->partial.p, psi_out,        active,      bt->tables.p,
                  bt->sigma_s.p, bt->G0.p,     bt->inflow.p,   d->mat_id.p, d->dir_dev.p,
                  gdev,         d->nx,         d->ny,          d->n_cells,  d->n_dof,
                  d->n_mat,     d->n_dirs,     n_groups,       with_source, std::sqrt(d->hx * d->hy),
                  1.0 / d->hx,  1.0 / d->hy};
    const int H0 = d->nx < 32 ? d->nx : 32;
    const int nrb = (d->ny + H0 - 1) / H0;
    int NW = 1;
    if (bt->force_nw > 0) {
      NW = bt->force_nw;
    } else if (!bt->tuned_nw.empty() && bt->tuned_nw.size() == bt->tuned.size() && !bt->force_dpw) {
      NW = bt->tuned_nw.back();   // the measured choice for this running count
      for (size_t e = 0; e < bt->tuned.size(); ++e)
        if (n_active <= bt->tuned[e].first) {
          NW = bt->tuned_nw[e];
          break;
        }
    } else if (bt->kba) {
      NW = kba_warps(d, bt->n_sm, (long long)n_active * n_groups);
    }
    NW = std::max(1, std::min(NW, std::min(nrb, 8)));
    if (NW >= 2) {
      const int H = d->nx < 32 ? d->nx : 32;
      const int D = std::max(H + kKbaChunk, (d->nx + H - 1 + NW - 1) / NW);  // as in kba_steps
      switch (dpw) {
        case 1: RTE_TRY(launch2d_kba<1>(A, bt->B, n_groups, NW, D, st)); break;
        case 2: RTE_TRY(launch2d_kba<2>(A, bt->B, n_groups, NW, D, st)); break;
        case 4: RTE_TRY(launch2d_kba<4>(A, bt->B, n_groups, NW, D, st)); break;
        case 8: RTE_TRY(launch2d_kba<8>(A, bt->B, n_groups, NW, D, st)); break;
        default: return fail(RTE_EINVAL, "unsupported directions-per-warp");
      }
    } else {
      switch (dpw) {
        case 1: RTE_TRY((launch2d<1, true>(A, bt->B, n_groups, st))); break;
        case 2: RTE_TRY((launch2d<2, true>(A, bt->B, n_groups, st))); break;
        case 4: RTE_TRY((launch2d<4, true>(A, bt->B, n_groups, st))); break;
        case 8: RTE_TRY((launch2d<8, true>(A, bt->B, n_groups, st))); break;
        default: return fail(RTE_EINVAL, "unsupported directions-per-warp");
      }
    }
  } else {
    Sweep1DArgs A{rho_in,      bt->partial.p, psi_out,  active, bt->tables.p, bt->sigma_s.p,
                  bt->G0.p,    bt->inflow.p,  d->mat_id.p, d->mat_r.p, d->dir_dev.p, bt->B, d->nx,
                  d->n_dof,    d->n_mat,      d->n_dirs, with_source};
    const int n = bt->B * d->n_dirs;
    RTE_TRY(note_started(bt, st));
    sweep1d_kernel<<<(n + 63) / 64, 64, 0, st>>>(A); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
  }
  if (bt->timing) {
    RTE_CUDA_TRY(cudaEventRecord(ev1, st));
    bt->sweep_ev.emplace_back(ev0, ev1);
    bt->sweep_launches += 1;
    bt->sweep_units += (double)n_active * d->n_cells * d->n_dirs;
  }
  if (fuse_norms && zero_norms)
    RTE_CUDA_TRY(cudaMemsetAsync(bt->norms.p, 0, sizeof(unsigned long long) * 2 * bt->B, st));
  const int th = 256;
  dim3 grid((d->n_dof / 2 + th - 1) / th, bt->B);
  double* fuse_R = d->dim == 2 ? bt->fuse_R : nullptr;
  reduce_partials_kernel<<<grid, th, 0, st>>>(bt->partial.p, rho_in, rho_out,
                                             fuse_norms ? bt->norms.p : nullptr, active, n_groups,
                                             d->n_dof, fuse_R, bt->sigma_s.p, d->mat_id.p,
                                             d->n_mat); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

// One FP64 sweep with source of the running instances of several 2D batches, in one launch of
// sweep2d_multi_kernel (see there), each batch's cell sources and partial-sum reduction (with the
// stop-test norms) launched per batch around it, all on `st`.  host_act[k]: batch k's running
// instances (host copy of its device mask act[k]).  Every batch sweeps DPW directions per warp,
// DPW = 4 or, when a batch's partial sums need wider groups, 8.  `ws` is scratch the call owns:
// descriptors, work list and counter.
int sweep_launch_multi(const std::vector<rte_batch_t>& bts, const std::vector<const double*>& rho_in,
                       const std::vector<double*>& rho_out, const std::vector<const uint8_t*>& act,
                       const std::vector<const uint8_t*>& host_act, MultiSweepScratch& ws,
                       cudaStream_t st) {
  const int n = (int)bts.size();
  int dpw = 4;
  for (rte_batch_t bt : bts) dpw = std::max(dpw, bt->min_dpw);
  const int k = dpw == 4 ? 2 : 3;
  std::vector<Sweep2DArgs> descs(n);
  std::vector<std::pair<long long, SweepItem>> work;
  size_t smem = 0;
  for (int q = 0; q < n; ++q) {
    rte_batch_t bt = bts[q];
    const rte_disc_s* d = bt->disc;
    if (d->dim != 2) return fail(RTE_EINVAL, "multi-batch sweep: 2D batches only");
    int n_act = 0;
    for (int b = 0; b < bt->B; ++b) n_act += host_act[q][b] != 0;
    if ((size_t)n_act * bt->gcount[k] * d->n_dof > bt->partial.n)
      return fail(RTE_EINVAL, "multi-batch sweep: partial sums do not fit");
    cell_source_kernel<<<dim3((d->n_cells + 127) / 128, bt->B), 128, 0, st>>>(
        rho_in[q], bt->S.p, bt->sigma_s.p, bt->G0.p, d->mat_id.p, act[q], d->n_cells, d->n_mat, 1); RTE_NOTE_LAUNCH();
    descs[q] = Sweep2DArgs{bt->S.p,      bt->partial.p, nullptr,      act[q],      bt->tables.p,
                           bt->sigma_s.p, bt->G0.p,     bt->inflow.p, d->mat_id.p, d->dir_dev.p,
                           bt->groups_all_dev.p + bt->goff[k], d->nx, d->ny, d->n_cells, d->n_dof,
                           d->n_mat,     d->n_dirs,     bt->gcount[k], 1,       std::sqrt(d->hx * d->hy),
                           1.0 / d->hx,  1.0 / d->hy};
    const int H = d->nx < 32 ? d->nx : 32;
    const long long steps = (long long)((d->ny + H - 1) / H) * d->nx + H - 1;
    for (int b = 0; b < bt->B; ++b)
      if (host_act[q][b])
        for (int g = 0; g < bt->gcount[k]; ++g) work.push_back({steps, SweepItem{q, g, b, 0}});
    smem = std::max(smem, ((size_t)d->nx * dpw * 2 + (size_t)d->n_mat * dpw * kTab2D + d->n_mat) *
                              sizeof(double));
    if (bt->timing) bt->sweep_units += (double)n_act * d->n_cells * d->n_dirs;
  }
  RTE_CUDA_TRY(cudaGetLastError());
  // longest sweeps first; ties keep the batch / instance / group order
  std::stable_sort(work.begin(), work.end(),
                   [](const auto& a, const auto& b) { return a.first > b.first; });
  const int n_items = (int)work.size();
  if (n_items > 0) {
    if (ws.descs.n < (size_t)n) RTE_TRY(ws.descs.alloc(n));
    if (ws.items.n < (size_t)n_items) RTE_TRY(ws.items.alloc(n_items));
    if (!ws.counter.p) RTE_TRY(ws.counter.alloc(1));
    ws.h_items.resize(n_items);
    for (int i = 0; i < n_items; ++i) ws.h_items[i] = work[i].second;
    ws.h_descs = descs;
    RTE_CUDA_TRY(cudaMemcpyAsync(ws.descs.p, ws.h_descs.data(), sizeof(Sweep2DArgs) * n,
                                 cudaMemcpyHostToDevice, st));
    RTE_CUDA_TRY(cudaMemcpyAsync(ws.items.p, ws.h_items.data(), sizeof(SweepItem) * n_items,
                                 cudaMemcpyHostToDevice, st));
    RTE_CUDA_TRY(cudaMemsetAsync(ws.counter.p, 0, sizeof(int), st));
    if (smem > 200 * 1024) return fail(RTE_EINVAL, "multi-batch sweep: shared memory exceeded");
    int n_sm = 0, dev = 0;
    RTE_CUDA_TRY(cudaGetDevice(&dev));
    RTE_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::min(n_items, 16 * n_sm);   // a persistent grid: warps take items in turn
    if (dpw == 4) {
      if (smem > 48 * 1024)
        RTE_CUDA_TRY(cudaFuncSetAttribute(sweep2d_multi_kernel<4>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      sweep2d_multi_kernel<4><<<grid, 32, smem, st>>>(ws.descs.p, ws.items.p, n_items, ws.counter.p); RTE_NOTE_LAUNCH();
    } else {
      if (smem > 48 * 1024)
        RTE_CUDA_TRY(cudaFuncSetAttribute(sweep2d_multi_kernel<8>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      sweep2d_multi_kernel<8><<<grid, 32, smem, st>>>(ws.descs.p, ws.items.p, n_items, ws.counter.p); RTE_NOTE_LAUNCH();
    }
    RTE_CUDA_TRY(cudaGetLastError());
  }
  const int th = 256;
  for (int q = 0; q < n; ++q) {
    rte_batch_t bt = bts[q];
    const rte_disc_s* d = bt->disc;
    RTE_CUDA_TRY(cudaMemsetAsync(bt->norms.p, 0, sizeof(unsigned long long) * 2 * bt->B, st));
    dim3 grid((d->n_dof / 2 + th - 1) / th, bt->B);
    reduce_partials_kernel<<<grid, th, 0, st>>>(bt->partial.p, rho_in[q], rho_out[q], bt->norms.p,
                                               act[q], bt->gcount[k], d->n_dof); RTE_NOTE_LAUNCH();
  }
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

int norms_to_host(rte_batch_t bt, double* host, cudaStream_t st) {
  std::vector<unsigned long long> bits(2 * bt->B);
  RTE_CUDA_TRY(cudaMemcpyAsync(bits.data(), bt->norms.p, sizeof(unsigned long long) * bits.size(),
                               cudaMemcpyDeviceToHost, st));
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  for (size_t k = 0; k < bits.size(); ++k) {
    long long v = (long long)bits[k];
    double x;
    std::memcpy(&x, &v, sizeof(double));
    host[k] = x;
  }
  return RTE_OK;
}

int correction_source_launch(rte_batch_t bt, const double* rs, const double* rp, double* R,
                             const uint8_t* active, cudaStream_t st) {
  const rte_disc_s* d = bt->disc;
  if (d->linear) {
    dim3 grid1(std::min((d->nx + 255) / 256, 1024), bt->B);
    correction_source1d_linear_kernel<<<grid1, 256, 0, st>>>(rs, rp, R, bt->sigma_s.p, d->mat_id.p,
                                                             d->mat_r.p, active, d->nx, d->n_mat); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
  }
  dim3 grid(std::min((d->n_dof + 255) / 256, 1024), bt->B);
  correction_source_kernel<<<grid, 256, 0, st>>>(rs, rp, R, bt->sigma_s.p, d->mat_id.p, active,
                                                 d->n_dof, d->P, d->n_mat); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

int axpy_launch(rte_batch_t bt, const double* x, const double* y, double* out,
                const uint8_t* active, cudaStream_t st) {
  const rte_disc_s* d = bt->disc;
  dim3 grid(std::min((d->n_dof + 255) / 256, 1024), bt->B);
  add_kernel<<<grid, 256, 0, st>>>(x, y, out, active, d->n_dof); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

}  // namespace rte

using namespace rte;

extern "C" int rte_sweep(rte_batch_t b, const double* rho_in, double* rho_out, double* psi_out,
                         int with_source, const uint8_t* active, void* stream) {
  if (!b || !rho_in || !rho_out) return fail(RTE_EINVAL, "rte_sweep: null argument");
  RTE_TRY(params_ready(b, "rte_sweep"));
  if (rho_in == rho_out) return fail(RTE_EINVAL, "rte_sweep: rho_out aliases rho_in");
  if (((uintptr_t)rho_in | (uintptr_t)rho_out | (uintptr_t)psi_out) & 15)
    return fail(RTE_EINVAL, "rte_sweep: arrays must be 16-byte aligned");
  DeviceGuard g(b->disc->device);
  return sweep_launch(b, rho_in, rho_out, psi_out, with_source, active, (cudaStream_t)stream,
                      false, -1);
}

extern "C" int rte_change_norm(rte_batch_t b, const double* rho_star, const double* rho_prev,
                               double* norms, void* stream) {
  if (!b || !rho_star || !rho_prev || !norms) return fail(RTE_EINVAL, "rte_change_norm: null");
  DeviceGuard g(b->disc->device);
  cudaStream_t st = (cudaStream_t)stream;
  RTE_CUDA_TRY(cudaMemsetAsync(b->norms.p, 0, sizeof(unsigned long long) * 2 * b->B, st));
  dim3 grid(std::min((b->disc->n_dof + 255) / 256, 256), b->B);
  change_norm_kernel<<<grid, 256, 0, st>>>(rho_star, rho_prev, b->norms.p, b->disc->n_dof); RTE_NOTE_LAUNCH();
  bits_to_double_kernel<<<(2 * b->B + 127) / 128, 128, 0, st>>>(b->norms.p, norms, 2 * b->B); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

extern "C" int rte_correction_source(rte_batch_t b, const double* rho_star, const double* rho_prev,
                                     double* R, void* stream) {
  if (!b || !rho_star || !rho_prev || !R) return fail(RTE_EINVAL, "rte_correction_source: null");
  RTE_TRY(params_ready(b, "rte_correction_source"));
  DeviceGuard g(b->disc->device);
  return correction_source_launch(b, rho_star, rho_prev, R, nullptr, (cudaStream_t)stream);
}

namespace rte {

// Same launches as sweep_launch (sweep kernel, then the fixed-order partial-sum reduction) with
// the partial sums placed in caller-provided device memory; no timing and no norms.  Used by the
// allocation-free entry point in noalloc.cu.
int sweep_launch_with_scratch(rte_batch_t bt, const double* rho_in, double* rho_out,
                              int with_source, cudaStream_t st, double* partial) {
  const rte_disc_s* d = bt->disc;
  const int n_groups = (int)bt->groups.size();
  if (d->dim == 2) {
    Sweep2DArgs A{rho_in,       partial,       nullptr,        nullptr,     bt->tables.p,
                  bt->sigma_s.p, bt->G0.p,     bt->inflow.p,   d->mat_id.p, d->dir_dev.p,
                  bt->groups_dev.p, d->nx,     d->ny,          d->n_cells,  d->n_dof,
                  d->n_mat,     d->n_dirs,     n_groups,       with_source, std::sqrt(d->hx * d->hy),
                  1.0 / d->hx,  1.0 / d->hy};
    switch (bt->dpw) {
      case 1: RTE_TRY(launch2d<1>(A, bt->B, n_groups, st)); break;
      case 2: RTE_TRY(launch2d<2>(A, bt->B, n_groups, st)); break;
      case 4: RTE_TRY(launch2d<4>(A, bt->B, n_groups, st)); break;
      case 8: RTE_TRY(launch2d<8>(A, bt->B, n_groups, st)); break;
      default: return fail(RTE_EINVAL, "unsupported directions-per-warp");
    }
  } else {
    Sweep1DArgs A{rho_in,      partial,       nullptr,  nullptr, bt->tables.p, bt->sigma_s.p,
                  bt->G0.p,    bt->inflow.p,  d->mat_id.p, d->mat_r.p, d->dir_dev.p, bt->B, d->nx,
                  d->n_dof,    d->n_mat,      d->n_dirs, with_source};
    const int n = bt->B * d->n_dirs;
    sweep1d_kernel<<<(n + 63) / 64, 64, 0, st>>>(A); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
  }
  const int th = 256;
  dim3 grid((d->n_dof / 2 + th - 1) / th, bt->B);
  reduce_partials_kernel<<<grid, th, 0, st>>>(partial, rho_in, rho_out, nullptr, nullptr, n_groups,
                                             d->n_dof); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

// One FP64 sweep with source of the instances in `active` (every instance when null) that also
// records each cell's net face outflow per work group in bt->leak (allocated here on first use:
// B x groups x n_cells doubles).  2D sweeps use the widest direction groups (8 per warp), which
// need the fewest leak partials and fit every batch's partial-sum buffer.  *n_groups receives the
// number of groups whose leak partials the caller sums.
int sweep_launch_leak(rte_batch_t bt, const double* rho_in, double* rho_out, const uint8_t* active,
                      cudaStream_t st, int* n_groups_out) {
  const rte_disc_s* d = bt->disc;
  int n_groups = 0;
  const SweepGroup* gdev = nullptr;
  if (d->dim == 2) {
    n_groups = bt->gcount[3];
    gdev = bt->groups_all_dev.p + bt->goff[3];
  } else {
    n_groups = d->n_dirs;
  }
  const size_t need = (size_t)bt->B * n_groups * d->n_cells;
  if (bt->leak.n < need) RTE_TRY(bt->leak.alloc(need));
  if (d->dim == 2) {
    cell_source_kernel<<<dim3((d->n_cells + 127) / 128, bt->B), 128, 0, st>>>(
        rho_in, bt->S.p, bt->sigma_s.p, bt->G0.p, d->mat_id.p, active, d->n_cells, d->n_mat, 1); RTE_NOTE_LAUNCH();
    Sweep2DArgs A{bt->S.p,      bt->partial.p, nullptr,        active,      bt->tables.p,
                  bt->sigma_s.p, bt->G0.p,     bt->inflow.p,   d->mat_id.p, d->dir_dev.p,
                  gdev,         d->nx,         d->ny,          d->n_cells,  d->n_dof,
                  d->n_mat,     d->n_dirs,     n_groups,       1,           std::sqrt(d->hx * d->hy),
                  1.0 / d->hx,  1.0 / d->hy,   bt->leak.p,     std::sqrt(d->hy / d->hx),
                  std::sqrt(d->hx / d->hy)};
    RTE_TRY((launch2d<8, true, true>(A, bt->B, n_groups, st)));
  } else {
    Sweep1DArgs A{rho_in,      bt->partial.p, nullptr,  active, bt->tables.p, bt->sigma_s.p,
                  bt->G0.p,    bt->inflow.p,  d->mat_id.p, d->mat_r.p, d->dir_dev.p, bt->B, d->nx,
                  d->n_dof,    d->n_mat,      d->n_dirs, 1,      bt->leak.p};
    const int n = bt->B * d->n_dirs;
    sweep1d_kernel<<<(n + 63) / 64, 64, 0, st>>>(A); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
  }
  const int th = 256;
  dim3 grid((d->n_dof / 2 + th - 1) / th, bt->B);
  reduce_partials_kernel<<<grid, th, 0, st>>>(bt->partial.p, rho_in, rho_out, nullptr, active,
                                             n_groups, d->n_dof); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  *n_groups_out = n_groups;
  return RTE_OK;
}

}  // namespace rte

// ---- FP32 sweep (precision variant) --------------------------------------------------------------
//
// Same wavefront layout and cell algebra as sweep2d_kernel, in single precision: FP32 tables,
// FP32 sources formed once per sweep, FP32 partial sums.  The FP32 units of GB300 run at about 59x
// the FP64 rate, so these sweeps are cheap; rte_solve uses them for the early iterations of an
// instance and switches it to the FP64 sweep for the final ones (rte_solve_opts.fp32_switch).
//
// Correction sweeps of the FP64 outer residual-correction loop (rte_solve_opts.refine_kappa): for
// the instances flagged in `inner`, the sweep applies L to the error e = rho - x0 of the outer
// point x0 alone -- cell sources Sigma_s (rho - x0), no volume source, no inflow -- and the FP64
// reduction adds y0 = L x0 + b (the FP64 sweep of x0), so rho_out = y0 + L (rho - x0) = L rho + b
// with FP32 rounding confined to the small e.
namespace rte {

// FP32 copy of the sweep tables, M^-1 of each (instance, material, direction) in pair-major order:
// the column entries of rows (0, 1) side by side, then those of rows (2, 3) --
// (m00, m10, m01, m11, m02, m12, m03, m13, m20, m30, m21, m31, m22, m32, m23, m33) -- so that one
// packed FMA applies a column to two rows (f32_cell).
__global__ void tables_to_f32_kernel(const double* t64, float* t32, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = (int)(i % kTab2D), row = k / 4, col = k % 4, pr = row / 2;
  t32[i - k + 8 * pr + 2 * col + (row - 2 * pr)] = (float)t64[i];
}

// Packed single-precision pairs (PTX fma.rn.f32x2 / mul.rn.f32x2, sm_100 and later): one
// instruction for two FP32 operations, each rounded exactly as the scalar fmaf / multiply.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// floats of the FP32 sweep's y-inflow line buffer, rounded up so that the tables behind it start
// on a 16-byte boundary
__host__ __device__ __forceinline__ int ybuf32_floats(int nx, int dpw) {
  return (nx * dpw * 2 + 3) & ~3;
}

__global__ void cell_source32_kernel(const double* __restrict__ rho, float* S,
                                     const double* __restrict__ sigma_s,
                                     const double* __restrict__ G0, const int32_t* __restrict__ mat,
                                     const uint8_t* active, int n_cells, int n_mat, int with_source,
                                     const uint8_t* inner, const double* __restrict__ x0) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const double ss = sigma_s[(size_t)b * n_mat + mat[c]];
  const size_t o = ((size_t)b * n_cells + c) * 4;
  const double* r = rho + o;
  double v0 = r[0], v1 = r[1], v2 = r[2], v3 = r[3];
  bool src = with_source;
  if (inner && inner[b]) {
    const double* x = x0 + o;
    v0 -= x[0], v1 -= x[1], v2 -= x[2], v3 -= x[3];
    src = false;
  }
  const double s0 = fma(ss, v0, src ? G0[(size_t)b * n_cells + c] : 0.0);
  reinterpret_cast<float4*>(S)[(size_t)b * n_cells + c] =
      make_float4((float)s0, (float)(ss * v1), (float)(ss * v2), (float)(ss * v3));
}

struct Sweep2D32Args {
  const float* S;
  float* partial;
  const uint8_t* active;
  const uint8_t* inner;   // correction sweeps: no inflow
  const float* tables;
  const double* inflow;
  const int32_t* mat;
  const double* dirs;
  const SweepGroup* groups;
  int nx, ny, n_cells, n_dof, n_mat, n_dirs, n_groups, with_source;
  double sq_area;
  double ihx, ihy;          // 1 / h_x, 1 / h_y
};

// Per-material stride of the FP32 kernel's shared-memory tables: a group's DPW tables of 16 floats,
// padded by 4 floats so that rows of consecutive materials fall into different banks (a warp's
// lanes on either side of a material interface then read their rows without a bank conflict).
__host__ __device__ __forceinline__ int tab32_stride(int dpw) { return dpw * kTab2D + 4; }

template <int DPW>
__global__ void __launch_bounds__(32) sweep2d_f32_kernel(const Sweep2D32Args A) {
  const int g = blockIdx.x, b = blockIdx.y, lane = threadIdx.x;
  if (A.active && !A.active[b]) return;
  const SweepGroup grp = A.groups[g];
  const bool xneg = grp.quad & 1, yneg = (grp.quad & 2) != 0;
  extern __shared__ float smf[];
  float* ybuf = smf;                                 // [nx][DPW][2]
  float* tab_s = smf + ybuf32_floats(A.nx, DPW);     // [n_mat][tab32_stride], 16-byte aligned
  const int mstride = tab32_stride(DPW);
  const float* __restrict__ tabg = A.tables + (size_t)b * A.n_mat * A.n_dirs * kTab2D;
  for (int e = lane; e < A.n_mat * DPW * kTab2D; e += 32) {
    const int m = e / (DPW * kTab2D), r = e % (DPW * kTab2D), dd = r / kTab2D, k = r % kTab2D;
    tab_s[m * mstride + r] = dd < grp.nd ? tabg[((size_t)m * A.n_dirs + grp.d0 + dd) * kTab2D + k] : 0.f;
  }
  __syncwarp();
  float w[DPW], ax[DPW], bx[DPW], ay[DPW], by[DPW];
#pragma unroll
  for (int dd = 0; dd < DPW; ++dd) {
    const bool in = dd < grp.nd;
    w[dd] = in ? (float)A.dirs[4 * (grp.d0 + dd) + 2] : 0.f;
    const double vx = in ? A.dirs[4 * (grp.d0 + dd)] : 0.0, vy = in ? A.dirs[4 * (grp.d0 + dd) + 1] : 0.0;
    const double axd = fabs(vx) * A.ihx, ayd = fabs(vy) * A.ihy;
    ax[dd] = (float)axd, ay[dd] = (float)ayd;
    bx[dd] = (float)((vx < 0 ? 1.7320508075688772 : -1.7320508075688772) * axd);
    by[dd] = (float)((vy < 0 ? 1.7320508075688772 : -1.7320508075688772) * ayd);
  }
  const float s3 = 1.7320508075688772f;
  const float c3x = xneg ? -s3 : s3, c3y = yneg ? -s3 : s3;
  const bool src = A.with_source && !(A.inner && A.inner[b]);
  const float gxb = src ? (float)(A.inflow[4 * b + (xneg ? 1 : 0)] * A.sq_area) : 0.f;
  const float gyb = src ? (float)(A.inflow[4 * b + (yneg ? 3 : 2)] * A.sq_area) : 0.f;
  const int H = A.nx < 32 ? A.nx : 32;
  const int nrb = (A.ny + H - 1) / H;
  const int total = nrb * A.nx;
  const float4* __restrict__ Sb = reinterpret_cast<const float4*>(A.S) + (size_t)b * A.n_cells;
  float4* part = reinterpret_cast<float4*>(A.partial + ((size_t)active_rank(A.active, b) * A.n_groups + g) * A.n_dof);
  float tx[DPW][2], typ[DPW][2];
#pragma unroll
  for (int dd = 0; dd < DPW; ++dd) tx[dd][0] = tx[dd][1] = typ[dd][0] = typ[dd][1] = 0.f;
  // A lane handles u = s - lane, u = 0, 1, ..., total - 1, at column t = u mod nx of row block
  // rb = u / nx; both are kept as counters (tn, rbn: the position of u + 1) instead of being
  // divided out at every step.  Its cell is c = j nx + i with i, j the mirrored t and rb H + lane.
  auto cell_of = [&](int t_, int rb_) {
    const int r_ = rb_ * H + lane;
    return (yneg ? A.ny - 1 - r_ : r_) * A.nx + (xneg ? A.nx - 1 - t_ : t_);
  };
  int tn = 0, rbn = 0;
  // the next step's material and cell source are loaded while this step computes, so the
  // global-memory latency is off the wavefront's critical path
  int m_next = 0;
  float4 sv_next = make_float4(0.f, 0.f, 0.f, 0.f);
  if (lane == 0 && H > 0 && A.ny > 0) {   // lane 0's first cell (u = 0 at step 0)
    const int c0 = cell_of(0, 0);
    m_next = A.mat[c0], sv_next = Sb[c0];
  }
  for (int s = 0; s < total + H - 1; ++s) {
    const int u = s - lane;
    int t = 0, rb = 0;
    if (u >= 0) {   // this step's position; advance the next one
      t = tn, rb = rbn;
      if (++tn == A.nx) tn = 0, ++rbn;
    }
    const bool inrange = lane < H && u >= 0 && u < total;
    const int r = rb * H + lane;
    const bool act = inrange && r < A.ny;
    const int m = m_next;
    const float4 sv = sv_next;
    // u + 1 sits at (tn, rbn)
    if (lane < H && u + 1 >= 0 && u + 1 < total && rbn * H + lane < A.ny) {
      const int c1 = cell_of(tn, rbn);
      m_next = A.mat[c1], sv_next = Sb[c1];
    }
    float ty[DPW][2];
#pragma unroll
    for (int dd = 0; dd < DPW; ++dd) {
      ty[dd][0] = __shfl_up_sync(0xffffffffu, typ[dd][0], 1);
      ty[dd][1] = __shfl_up_sync(0xffffffffu, typ[dd][1], 1);
    }
    if (act) {
      if (r == 0) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) ty[dd][0] = gyb, ty[dd][1] = 0.f;
      } else if (lane == 0) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) {
          ty[dd][0] = ybuf[(t * DPW + dd) * 2];
          ty[dd][1] = ybuf[(t * DPW + dd) * 2 + 1];
        }
      }
      if (t == 0) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) tx[dd][0] = gxb, tx[dd][1] = 0.f;
      }
      const int c = cell_of(t, rb);
      float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
      // every slot of the group is computed without a branch, so the DPW directions' FMA chains
      // can be interleaved: a slot beyond the group's directions has zero tables and weight and
      // adds nothing
      const float4* Tm = reinterpret_cast<const float4*>(tab_s + m * mstride);
      float2 acc01 = make_float2(acc0, acc1), acc23 = make_float2(acc2, acc3);
#pragma unroll
      for (int dd = 0; dd < DPW; ++dd) {
        const float4* T = Tm + dd * (kTab2D / 4);
        // right-hand side s + E_x t_x + E_y t_y as the pairs (r0, r1), (r2, r3), then M^-1 applied
        // column by column to the row pairs (a0, a1), (a2, a3) (pair-major tables): the same
        // roundings in the same order as one fmaf per entry
        const float2 exb = make_float2(ax[dd], bx[dd]);
        const float2 tyv = make_float2(ty[dd][0], ty[dd][1]);
        const float2 r01 = fma2(make_float2(ay[dd], ay[dd]), tyv,
                                fma2(exb, make_float2(tx[dd][0], tx[dd][0]), make_float2(sv.x, sv.y)));
        const float2 r23 = fma2(make_float2(by[dd], by[dd]), tyv,
                                fma2(exb, make_float2(tx[dd][1], tx[dd][1]), make_float2(sv.z, sv.w)));
        const float4 q0 = T[0], q1 = T[1], q2 = T[2], q3 = T[3];
        const float2 rr0 = make_float2(r01.x, r01.x), rr1 = make_float2(r01.y, r01.y);
        const float2 rr2 = make_float2(r23.x, r23.x), rr3 = make_float2(r23.y, r23.y);
        float2 a01 = mul2(make_float2(q0.x, q0.y), rr0);
        a01 = fma2(make_float2(q0.z, q0.w), rr1, a01);
        a01 = fma2(make_float2(q1.x, q1.y), rr2, a01);
        a01 = fma2(make_float2(q1.z, q1.w), rr3, a01);
        float2 a23 = mul2(make_float2(q2.x, q2.y), rr0);
        a23 = fma2(make_float2(q2.z, q2.w), rr1, a23);
        a23 = fma2(make_float2(q3.x, q3.y), rr2, a23);
        a23 = fma2(make_float2(q3.z, q3.w), rr3, a23);
        tx[dd][0] = fmaf(c3x, a01.y, a01.x);
        tx[dd][1] = fmaf(c3x, a23.y, a23.x);
        const float2 tyo = fma2(make_float2(c3y, c3y), a23, a01);
        typ[dd][0] = tyo.x, typ[dd][1] = tyo.y;
        const float2 ww = make_float2(w[dd], w[dd]);
        acc01 = fma2(ww, a01, acc01);
        acc23 = fma2(ww, a23, acc23);
      }
      part[c] = make_float4(acc01.x, acc01.y, acc23.x, acc23.y);
      if (lane == H - 1 && rb + 1 < nrb) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) {
          ybuf[(t * DPW + dd) * 2] = typ[dd][0];
          ybuf[(t * DPW + dd) * 2 + 1] = typ[dd][1];
        }
      }
    }
    __syncwarp();
  }
}

// rho_out (FP64) = sum of the FP32 group partials (fixed order, summed in FP32: the partials carry
// FP32 rounding already, and FP64 additions would bind on GB300's FP64 pipe), plus y0 in FP64 for
// the instances flagged in `inner`; fused norms (the change itself is formed in FP64).
__global__ void reduce_partials32_kernel(const float* __restrict__ partial,
                                         const double* __restrict__ rho_in, double* rho_out,
                                         unsigned long long* norms, const uint8_t* active,
                                         int n_groups, int n_dof, const uint8_t* inner,
                                         const double* __restrict__ y0, double* R,
                                         const double* __restrict__ sigma_s,
                                         const int32_t* __restrict__ mat, int n_mat) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int rank = active_rank(active, b);
  const int e = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  unsigned long long dmax = 0ull, rmax = 0ull;
  if (e < n_dof) {
    const float* p = partial + (size_t)rank * n_groups * n_dof + e;
    float4 s = *reinterpret_cast<const float4*>(p);
    for (int g = 1; g < n_groups; ++g) {
      const float4 v = *reinterpret_cast<const float4*>(p + (size_t)g * n_dof);
      s.x += v.x, s.y += v.y, s.z += v.z, s.w += v.w;
    }
    double a0 = s.x, a1 = s.y, a2 = s.z, a3 = s.w;
    if (inner && inner[b]) {
      const double* y = y0 + (size_t)b * n_dof + e;
      a0 += y[0], a1 += y[1], a2 += y[2], a3 += y[3];
    }
    double* o = rho_out + (size_t)b * n_dof + e;
    o[0] = a0, o[1] = a1, o[2] = a2, o[3] = a3;
    if (norms || R) {
      const double* ri = rho_in + (size_t)b * n_dof + e;
      if (norms) {
        dmax = umax64(umax64(abs_bits(a0 - ri[0]), abs_bits(a1 - ri[1])),
                      umax64(abs_bits(a2 - ri[2]), abs_bits(a3 - ri[3])));
        rmax = umax64(umax64(abs_bits(a0), abs_bits(a1)), umax64(abs_bits(a2), abs_bits(a3)));
      }
      if (R) {   // the correction source, as correction_source_kernel forms it
        const double ss = sigma_s[(size_t)b * n_mat + mat[e / 4]];
        double* r = R + (size_t)b * n_dof + e;
        r[0] = ss * (a0 - ri[0]), r[1] = ss * (a1 - ri[1]), r[2] = ss * (a2 - ri[2]), r[3] = ss * (a3 - ri[3]);
      }
    }
  }
  if (!norms) return;
  block_norms(dmax, rmax, norms, b);
}

template <int DPW>
static int launch2d_f32(const Sweep2D32Args& A, int B, int n_groups, cudaStream_t st) {
  const size_t bytes =
      ((size_t)ybuf32_floats(A.nx, DPW) + (size_t)A.n_mat * tab32_stride(DPW)) * sizeof(float);
  if (bytes > 200 * 1024) return fail(RTE_EINVAL, "FP32 sweep: shared memory exceeded");
  if (bytes > 48 * 1024) {
    RTE_CUDA_TRY(cudaFuncSetAttribute(sweep2d_f32_kernel<DPW>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  }
  sweep2d_f32_kernel<DPW><<<dim3(n_groups, B), 32, bytes, st>>>(A); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

// One FP32 sweep of the active instances of a 2D batch, partial sums reduced in FP64 into
// rho_out with the stop-test norms fused (as sweep_launch with fuse_norms).
int sweep_launch_f32(rte_batch_t bt, const double* rho_in, double* rho_out, const uint8_t* active,
                     cudaStream_t st, int n_active, bool zero_norms, const uint8_t* inner,
                     const double* x0, const double* y0) {
  if (inner && (!x0 || !y0)) return fail(RTE_EINVAL, "FP32 correction sweep without x0, y0");
  const rte_disc_s* d = bt->disc;
  if (d->dim != 2) return fail(RTE_EINVAL, "FP32 sweep: 2D only");
  if (!bt->tables32.p) {
    const size_t n = bt->tables.n;
    RTE_TRY(bt->tables32.alloc(n));
    RTE_TRY(bt->S32.alloc((size_t)bt->B * d->n_dof));
    bt->tables32_stale = true;
  }
  int dpw = bt->dpw, n_groups = 0;
  const SweepGroup* gdev = nullptr;
  pick_groups(bt, n_active, &dpw, &n_groups, &gdev, true);
  const size_t need32 = bt->partial.n;  // the same group-slice capacity as the FP64 partial sums
  if (bt->partial32.n < need32) RTE_TRY(bt->partial32.alloc(need32));
  if (bt->tables32_stale) {
    const size_t n = bt->tables.n;
    tables_to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(bt->tables.p, bt->tables32.p, n); RTE_NOTE_LAUNCH();
    bt->tables32_stale = false;
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (bt->timing) {
    RTE_CUDA_TRY(cudaEventCreate(&ev0));
    RTE_CUDA_TRY(cudaEventCreate(&ev1));
    RTE_CUDA_TRY(cudaEventRecord(ev0, st));
  }
  cell_source32_kernel<<<dim3((d->n_cells + 127) / 128, bt->B), 128, 0, st>>>(
      rho_in, bt->S32.p, bt->sigma_s.p, bt->G0.p, d->mat_id.p, active, d->n_cells, d->n_mat, 1,
      inner, x0); RTE_NOTE_LAUNCH();
  RTE_TRY(note_started(bt, st));
  Sweep2D32Args A{bt->S32.p,  bt->partial32.p, active,   inner,    bt->tables32.p, bt->inflow.p,
                  d->mat_id.p, d->dir_dev.p,   gdev,     d->nx,          d->ny,
                  d->n_cells, d->n_dof,        d->n_mat, d->n_dirs,      n_groups,
                  1,          std::sqrt(d->hx * d->hy), 1.0 / d->hx, 1.0 / d->hy};
  switch (dpw) {
    case 1: RTE_TRY(launch2d_f32<1>(A, bt->B, n_groups, st)); break;
    case 2: RTE_TRY(launch2d_f32<2>(A, bt->B, n_groups, st)); break;
    case 4: RTE_TRY(launch2d_f32<4>(A, bt->B, n_groups, st)); break;
    case 8: RTE_TRY(launch2d_f32<8>(A, bt->B, n_groups, st)); break;
    default: return fail(RTE_EINVAL, "unsupported directions-per-warp");
  }
  if (bt->timing) {
    RTE_CUDA_TRY(cudaEventRecord(ev1, st));
    bt->phase_ev.push_back({0, ev0, ev1});
    bt->phase_calls[0] += 1;
    bt->sweep32_units += (double)n_active * d->n_cells * d->n_dirs;
  }
  if (zero_norms)
    RTE_CUDA_TRY(cudaMemsetAsync(bt->norms.p, 0, sizeof(unsigned long long) * 2 * bt->B, st));
  const int th = 256;
  reduce_partials32_kernel<<<dim3((d->n_dof / 4 + th - 1) / th, bt->B), th, 0, st>>>(
      bt->partial32.p, rho_in, rho_out, bt->norms.p, active, n_groups, d->n_dof, inner, y0,
      bt->fuse_R, bt->sigma_s.p, d->mat_id.p, d->n_mat); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

}  // namespace rte

extern "C" int rte_sweep_f32(rte_batch_t b, const double* rho_in, double* rho_out,
                             const uint8_t* active, void* stream) {
  if (!b || !rho_in || !rho_out) return fail(RTE_EINVAL, "rte_sweep_f32: null argument");
  RTE_TRY(params_ready(b, "rte_sweep_f32"));
  if (b->disc->dim != 2) return fail(RTE_EINVAL, "rte_sweep_f32: 2D batches only");
  if (rho_in == rho_out) return fail(RTE_EINVAL, "rte_sweep_f32: rho_out aliases rho_in");
  DeviceGuard g(b->disc->device);
  // the group choice is sized for every instance running (the mask is device memory)
  return sweep_launch_f32(b, rho_in, rho_out, active, (cudaStream_t)stream, b->B);
}

namespace rte {
// Empirical choice of the sweep decomposition: for running-instance counts B, B/2, B/4, ..., 1
// (the first instances of the batch) every directions-per-warp value the partial-sum buffer
// allows is timed with CUDA events on `st`, and the fastest is kept per count -- separately for
// the FP64 sweep and for the FP32 sweep of the precision variant (which is bound by the latency of
// its wavefront rather than by the FP64 pipe, so it may want more, narrower warps).
static int autotune(rte_batch_t bt, cudaStream_t st, int* n_entries, int* table) {
  const rte_disc_s* d = bt->disc;
  const int B = bt->B;
  const size_t nb = (size_t)B * d->n_dof;
  std::vector<int> bands;
  for (int n = B; n >= 1; n = n == 1 ? 0 : (n + 1) / 2) bands.push_back(n);
  std::reverse(bands.begin(), bands.end());
  DevBuf<uint8_t> mask;
  RTE_TRY(mask.alloc(B));
  std::vector<uint8_t> h(B);
  cudaEvent_t e0, e1;
  RTE_CUDA_TRY(cudaEventCreate(&e0));
  RTE_CUDA_TRY(cudaEventCreate(&e1));
  const bool timing = bt->timing;
  bt->timing = false;
  bt->tuned.clear();
  bt->tuned32.clear();
  bt->tuned_nw.clear();
  int status = RTE_OK;
  RTE_CUDA_TRY(cudaMemsetAsync(bt->work.p, 0, sizeof(double) * nb, st));
  for (int n : bands) {
    for (int b = 0; b < B; ++b) h[b] = b < n;
    if (cudaMemcpyAsync(mask.p, h.data(), B, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      status = fail(RTE_ECUDA, "autotune: mask upload");
      break;
    }
    for (int prec = 0; prec < (d->dim == 2 ? 2 : 1) && status == RTE_OK; ++prec) {
      float best_ms = 0.f;
      int best = 0;
      auto launch = [&]() {
        return prec == 0 ? sweep_launch(bt, bt->work.p, bt->work.p + nb, nullptr, 1, mask.p, st, true, n)
                         : sweep_launch_f32(bt, bt->work.p, bt->work.p + nb, mask.p, st, n);
      };
      int best_nw = 1;
      // FP64: also the pipelined sweep with 2, 4 or 8 warps per direction group (row blocks
      // permitting); the FP32 sweep has one form
      const int H0 = d->nx < 32 ? d->nx : 32;
      const int nw_max = prec == 0 ? std::min(8, (d->ny + H0 - 1) / H0) : 1;
      for (int dpw = 1; dpw <= kMaxDirsPerWarp && status == RTE_OK; dpw *= 2) {
        const int k = dpw == 1 ? 0 : dpw == 2 ? 1 : dpw == 4 ? 2 : 3;
        if ((size_t)n * bt->gcount[k] * d->n_dof > bt->partial.n) continue;  // no partial-sum space
        for (int nw = 1; nw <= nw_max && status == RTE_OK; nw *= 2) {
          bt->force_dpw = dpw;
          bt->force_nw = prec == 0 ? nw : 0;
          float ms = 0.f;
          status = launch();
          if (status == RTE_OK && cudaEventRecord(e0, st) != cudaSuccess) status = fail(RTE_ECUDA, "autotune: event");
          for (int rep = 0; rep < 2 && status == RTE_OK; ++rep) status = launch();
          if (status == RTE_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                                   cudaEventSynchronize(e1) != cudaSuccess ||
                                   cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            status = fail(RTE_ECUDA, "autotune: timing");
          if (status == RTE_OK && (best == 0 || ms < best_ms)) best_ms = ms, best = dpw, best_nw = nw;
        }
      }
      if (status != RTE_OK) break;
      (prec == 0 ? bt->tuned : bt->tuned32).emplace_back(n, best);
      if (prec == 0) bt->tuned_nw.push_back(best_nw);
    }
    if (status != RTE_OK) break;
  }
  bt->force_dpw = 0;
  bt->force_nw = 0;
  bt->timing = timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != RTE_OK) {
    bt->tuned.clear();
    bt->tuned32.clear();
    bt->tuned_nw.clear();
    return status;
  }
  bt->dpw_dynamic = true;
  if (n_entries) *n_entries = (int)bt->tuned.size();
  if (table)
    for (size_t k = 0; k < bt->tuned.size(); ++k) {
      table[2 * k] = bt->tuned[k].first;
      table[2 * k + 1] = bt->tuned[k].second;
    }
  return RTE_OK;
}
}  // namespace rte

extern "C" int rte_batch_tuned(rte_batch_t b, int* n_entries, int* table) {
  if (!b || !n_entries) return fail(RTE_EINVAL, "rte_batch_tuned: null argument");
  const bool ok = b->tuned_nw.size() == b->tuned.size();
  *n_entries = ok ? (int)b->tuned.size() : 0;
  if (table && ok)
    for (size_t k = 0; k < b->tuned.size(); ++k) {
      table[3 * k] = b->tuned[k].first;
      table[3 * k + 1] = b->tuned[k].second;
      table[3 * k + 2] = b->tuned_nw[k];
    }
  return RTE_OK;
}

extern "C" int rte_batch_autotune(rte_batch_t b, void* stream, int* n_entries, int* table) {
  if (!b) return fail(RTE_EINVAL, "rte_batch_autotune: null argument");
  RTE_TRY(params_ready(b, "rte_batch_autotune"));
  if (n_entries) *n_entries = 0;
  if (b->disc->dim != 2) return RTE_OK;
  DeviceGuard g(b->disc->device);
  return autotune(b, (cudaStream_t)stream, n_entries, table);
}

// ---- float-float sweep (the precision variant's outer sweeps) ------------------------------------
//
// The sweep and scalar-flux reduction of sweep2d_kernel in float-float arithmetic: every value is
// an unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi) / 2), about 48 significant
// bits.  A sum uses Knuth's TwoSum (s + e = a + b exactly, six additions); a product uses the FMA
// form of Dekker's exact product (fma(a, b, -p) is the rounding error of p = a * b); an FMA of two
// such numbers is one exact product, the two cross terms, one TwoSum and a renormalisation, 15
// FP32 operations.  On GB300 the FP32 pipe is about 60 times as wide as the FP64 pipe, so the 32
// FMAs of a cell-direction solve take several times fewer pipe cycles this way than in FP64.  The
// cell sources come from FP64 (rho and sigma_s in FP64, split once per cell), the per-group
// partial sums go back to FP64 and are reduced by the FP64 sweep's kernel (with the stop-test
// norms and the correction source), so only the sweep itself carries the float-float rounding
// (~1e-14 relative per FMA): far below what the outer residual of the precision variant needs,
// which is why its outer sweeps may run this way (rte_solve_opts.outer_ff).
namespace rte {

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
// both signs flipped by one integer XOR (exact, and not on the FP32 pipe)
__device__ __forceinline__ float2 neg2(float2 a) {
  float2 d;
  asm("{\n\t.reg .b64 ra;\n\tmov.b64 ra, {%2, %3};\n\txor.b64 ra, ra, 0x8000000080000000;\n\t"
      "mov.b64 {%0, %1}, ra;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y));
  return d;
}

// Two float-float numbers side by side, (hi.x + lo.x, hi.y + lo.y), so that every step is one
// packed instruction for both.  The asm statements are opaque to the compiler, so no addition is
// contracted into an FMA or reassociated, which the error-free transformations rely on.
struct FF2 {
  float2 hi, lo;
};

// a * b + c
__device__ __forceinline__ FF2 ff_fma2(const FF2& a, const FF2& b, const FF2& c) {
  const float2 p = mul2(a.hi, b.hi);
  float2 pe = fma2(a.hi, b.hi, neg2(p));   // exactly a.hi * b.hi - p
  pe = fma2(a.hi, b.lo, pe);
  pe = fma2(a.lo, b.hi, pe);
  const float2 s = add2(p, c.hi);          // TwoSum: s + e = p + c.hi exactly
  const float2 bv = sub2(s, p);
  float2 e = add2(sub2(p, sub2(s, bv)), sub2(c.hi, bv));
  e = add2(e, add2(pe, c.lo));
  FF2 r;                                   // renormalised: |r.lo| <= ulp(r.hi) / 2
  r.hi = add2(s, e);
  r.lo = sub2(e, sub2(r.hi, s));
  return r;
}

// a * b
__device__ __forceinline__ FF2 ff_mul2(const FF2& a, const FF2& b) {
  const float2 p = mul2(a.hi, b.hi);
  float2 pe = fma2(a.hi, b.hi, neg2(p));
  pe = fma2(a.hi, b.lo, pe);
  pe = fma2(a.lo, b.hi, pe);
  FF2 r;
  r.hi = add2(p, pe);
  r.lo = sub2(pe, sub2(r.hi, p));
  return r;
}

__device__ __forceinline__ FF2 ff_pair(float h0, float h1, float l0, float l1) {
  FF2 r;
  r.hi = make_float2(h0, h1);
  r.lo = make_float2(l0, l1);
  return r;
}

// v = hi + lo with hi = v rounded to FP32 and lo the rest rounded to FP32
__device__ __forceinline__ void ff_split(double v, float& hi, float& lo) {
  hi = __double2float_rn(v);
  lo = __double2float_rn(v - (double)hi);
}

// Float-float sweep tables: per (instance, material, direction) 32 floats, the 16 hi parts of
// M^-1 in the pair-major order of tables_to_f32_kernel, then the 16 lo parts in the same order.
__global__ void tables_to_ff_kernel(const double* t64, float* tff, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = (int)(i % kTab2D), row = k / 4, col = k % 4, pr = row / 2;
  const int q = 8 * pr + 2 * col + (row - 2 * pr);
  const size_t base = (i - k) * 2;
  float h, l;
  ff_split(t64[i], h, l);
  tff[base + q] = h;
  tff[base + kTab2D + q] = l;
}

// Cell sources S = Sigma_s rho + G in FP64 (as cell_source_kernel), stored split: per cell the 4
// hi parts, then the 4 lo parts.
__global__ void cell_source_ff_kernel(const double* __restrict__ rho, float* S,
                                      const double* __restrict__ sigma_s,
                                      const double* __restrict__ G0, const int32_t* __restrict__ mat,
                                      const uint8_t* active, int n_cells, int n_mat) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const double ss = sigma_s[(size_t)b * n_mat + mat[c]];
  const double2* r = reinterpret_cast<const double2*>(rho + ((size_t)b * n_cells + c) * 4);
  const double2 a = r[0], e = r[1];
  const double v[4] = {fma(ss, a.x, G0[(size_t)b * n_cells + c]), ss * a.y, ss * e.x, ss * e.y};
  float h[4], l[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) ff_split(v[k], h[k], l[k]);
  float4* o = reinterpret_cast<float4*>(S) + ((size_t)b * n_cells + c) * 2;
  o[0] = make_float4(h[0], h[1], h[2], h[3]);
  o[1] = make_float4(l[0], l[1], l[2], l[3]);
}

struct Sweep2DFFArgs {
  const float* S;           // [B][n_cells][8] split cell sources
  double* partial;          // [running rank][n_groups][n_dof], as the FP64 sweep's
  const uint8_t* active;
  const float* tables;      // [B][n_mat][n_dirs][32] split sweep tables
  const double* inflow;
  const int32_t* mat;
  const double* dirs;
  const SweepGroup* groups;
  int nx, ny, n_cells, n_dof, n_mat, n_dirs, n_groups;
  double sq_area;
  double ihx, ihy;          // 1 / h_x, 1 / h_y
};

// floats of the y-inflow line buffer ([nx][DPW][2 traces][hi, lo]) and of one material's tables
// in shared memory (DPW directions of 32 floats, padded by 4 like tab32_stride)
__host__ __device__ __forceinline__ int ybuf_ff_floats(int nx, int dpw) { return nx * dpw * 4; }
__host__ __device__ __forceinline__ int tab_ff_stride(int dpw) { return dpw * 2 * kTab2D + 4; }

// The wavefront of sweep2d_f32_kernel (lane = row of a block of 32 rows, one step per column,
// the next step's material and sources loaded ahead), with the cell algebra of cell_solve in
// float-float: right-hand side s + E_x t_x + E_y t_y, M^-1 applied column by column to the row
// pairs (a0, a1), (a2, a3), the outflow traces and the weighted partial sums, each operation in
// the order of the FP64 kernel.
template <int DPW>
__global__ void __launch_bounds__(32) sweep2d_ff_kernel(const Sweep2DFFArgs A) {
  const int g = blockIdx.x, b = blockIdx.y, lane = threadIdx.x;
  if (A.active && !A.active[b]) return;
  const SweepGroup grp = A.groups[g];
  const bool xneg = grp.quad & 1, yneg = (grp.quad & 2) != 0;
  extern __shared__ float smf[];
  float* ybuf = smf;
  float* tab_s = smf + ybuf_ff_floats(A.nx, DPW);     // 16-byte aligned: nx * DPW * 4 floats
  const int mstride = tab_ff_stride(DPW);
  const int per_dir = 2 * kTab2D;
  const float* __restrict__ tabg = A.tables + (size_t)b * A.n_mat * A.n_dirs * per_dir;
  for (int e = lane; e < A.n_mat * DPW * per_dir; e += 32) {
    const int m = e / (DPW * per_dir), r = e % (DPW * per_dir), dd = r / per_dir, k = r % per_dir;
    tab_s[m * mstride + r] = dd < grp.nd ? tabg[((size_t)m * A.n_dirs + grp.d0 + dd) * per_dir + k] : 0.f;
  }
  __syncwarp();
  // per direction: weight and inflow couplings (a = |v| / h, b = -s sqrt3 a), split
  float wh[DPW], wl[DPW], axh[DPW], axl[DPW], bxh[DPW], bxl[DPW], ayh[DPW], ayl[DPW], byh[DPW],
      byl[DPW];
#pragma unroll
  for (int dd = 0; dd < DPW; ++dd) {
    const bool in = dd < grp.nd;
    const double vx = in ? A.dirs[4 * (grp.d0 + dd)] : 0.0, vy = in ? A.dirs[4 * (grp.d0 + dd) + 1] : 0.0;
    const double axd = fabs(vx) * A.ihx, ayd = fabs(vy) * A.ihy;
    ff_split(in ? A.dirs[4 * (grp.d0 + dd) + 2] : 0.0, wh[dd], wl[dd]);
    ff_split(axd, axh[dd], axl[dd]);
    ff_split(ayd, ayh[dd], ayl[dd]);
    ff_split((vx < 0 ? 1.7320508075688772 : -1.7320508075688772) * axd, bxh[dd], bxl[dd]);
    ff_split((vy < 0 ? 1.7320508075688772 : -1.7320508075688772) * ayd, byh[dd], byl[dd]);
  }
  float s3h, s3l;
  ff_split(1.7320508075688772, s3h, s3l);
  const FF2 C3X = xneg ? ff_pair(-s3h, -s3h, -s3l, -s3l) : ff_pair(s3h, s3h, s3l, s3l);
  const FF2 C3Y = yneg ? ff_pair(-s3h, -s3h, -s3l, -s3l) : ff_pair(s3h, s3h, s3l, s3l);
  float gxh, gxl, gyh, gyl;
  ff_split(A.inflow[4 * b + (xneg ? 1 : 0)] * A.sq_area, gxh, gxl);
  ff_split(A.inflow[4 * b + (yneg ? 3 : 2)] * A.sq_area, gyh, gyl);
  const int H = A.nx < 32 ? A.nx : 32;
  const int nrb = (A.ny + H - 1) / H;
  const int total = nrb * A.nx;
  const float4* __restrict__ Sb = reinterpret_cast<const float4*>(A.S) + (size_t)b * A.n_cells * 2;
  double* part = A.partial + ((size_t)active_rank(A.active, b) * A.n_groups + g) * A.n_dof;
  // traces entering the next cell, per direction: x (from the left) and y (to the row below)
  FF2 tx[DPW], typ[DPW];
#pragma unroll
  for (int dd = 0; dd < DPW; ++dd) tx[dd] = typ[dd] = ff_pair(0.f, 0.f, 0.f, 0.f);
  auto cell_of = [&](int t_, int rb_) {
    const int r_ = rb_ * H + lane;
    return (yneg ? A.ny - 1 - r_ : r_) * A.nx + (xneg ? A.nx - 1 - t_ : t_);
  };
  int tn = 0, rbn = 0;
  int m_next = 0;
  float4 svh_next = make_float4(0.f, 0.f, 0.f, 0.f), svl_next = svh_next;
  if (lane == 0 && H > 0 && A.ny > 0) {
    const int c0 = cell_of(0, 0);
    m_next = A.mat[c0], svh_next = Sb[2 * (size_t)c0], svl_next = Sb[2 * (size_t)c0 + 1];
  }
  for (int s = 0; s < total + H - 1; ++s) {
    const int u = s - lane;
    int t = 0, rb = 0;
    if (u >= 0) {
      t = tn, rb = rbn;
      if (++tn == A.nx) tn = 0, ++rbn;
    }
    const bool inrange = lane < H && u >= 0 && u < total;
    const int r = rb * H + lane;
    const bool act = inrange && r < A.ny;
    const int m = m_next;
    const float4 svh = svh_next, svl = svl_next;
    if (lane < H && u + 1 >= 0 && u + 1 < total && rbn * H + lane < A.ny) {
      const int c1 = cell_of(tn, rbn);
      m_next = A.mat[c1], svh_next = Sb[2 * (size_t)c1], svl_next = Sb[2 * (size_t)c1 + 1];
    }
    FF2 ty[DPW];
#pragma unroll
    for (int dd = 0; dd < DPW; ++dd) {
      ty[dd].hi.x = __shfl_up_sync(0xffffffffu, typ[dd].hi.x, 1);
      ty[dd].hi.y = __shfl_up_sync(0xffffffffu, typ[dd].hi.y, 1);
      ty[dd].lo.x = __shfl_up_sync(0xffffffffu, typ[dd].lo.x, 1);
      ty[dd].lo.y = __shfl_up_sync(0xffffffffu, typ[dd].lo.y, 1);
    }
    if (act) {
      if (r == 0) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) ty[dd] = ff_pair(gyh, 0.f, gyl, 0.f);
      } else if (lane == 0) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) {
          const float4 v = *reinterpret_cast<const float4*>(ybuf + (t * DPW + dd) * 4);
          ty[dd] = ff_pair(v.x, v.y, v.z, v.w);
        }
      }
      if (t == 0) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd) tx[dd] = ff_pair(gxh, 0.f, gxl, 0.f);
      }
      const int c = cell_of(t, rb);
      const FF2 S01 = ff_pair(svh.x, svh.y, svl.x, svl.y);
      const FF2 S23 = ff_pair(svh.z, svh.w, svl.z, svl.w);
      FF2 acc01 = ff_pair(0.f, 0.f, 0.f, 0.f), acc23 = acc01;
      const float4* Tm = reinterpret_cast<const float4*>(tab_s + m * mstride);
#pragma unroll
      for (int dd = 0; dd < DPW; ++dd) {
        // every slot is computed; a slot beyond the group's directions has zero tables and
        // weight and adds nothing
        const float4* Th = Tm + dd * (per_dir / 4);
        const float4* Tl = Th + kTab2D / 4;
        // r0 = s0 + a_x t_x0 + a_y t_y0, r1 = s1 + b_x t_x0 + a_y t_y1 (and r2, r3 with t_x1, b_y)
        const FF2 EX = ff_pair(axh[dd], bxh[dd], axl[dd], bxl[dd]);
        const FF2 AY = ff_pair(ayh[dd], ayh[dd], ayl[dd], ayl[dd]);
        const FF2 BY = ff_pair(byh[dd], byh[dd], byl[dd], byl[dd]);
        const FF2 TX0 = ff_pair(tx[dd].hi.x, tx[dd].hi.x, tx[dd].lo.x, tx[dd].lo.x);
        const FF2 TX1 = ff_pair(tx[dd].hi.y, tx[dd].hi.y, tx[dd].lo.y, tx[dd].lo.y);
        const FF2 r01 = ff_fma2(AY, ty[dd], ff_fma2(EX, TX0, S01));
        const FF2 r23 = ff_fma2(BY, ty[dd], ff_fma2(EX, TX1, S23));
        const FF2 R0 = ff_pair(r01.hi.x, r01.hi.x, r01.lo.x, r01.lo.x);
        const FF2 R1 = ff_pair(r01.hi.y, r01.hi.y, r01.lo.y, r01.lo.y);
        const FF2 R2 = ff_pair(r23.hi.x, r23.hi.x, r23.lo.x, r23.lo.x);
        const FF2 R3 = ff_pair(r23.hi.y, r23.hi.y, r23.lo.y, r23.lo.y);
        const float4 h0 = Th[0], h1 = Th[1], h2 = Th[2], h3 = Th[3];
        const float4 l0 = Tl[0], l1 = Tl[1], l2 = Tl[2], l3 = Tl[3];
        FF2 a01 = ff_mul2(ff_pair(h0.x, h0.y, l0.x, l0.y), R0);
        a01 = ff_fma2(ff_pair(h0.z, h0.w, l0.z, l0.w), R1, a01);
        a01 = ff_fma2(ff_pair(h1.x, h1.y, l1.x, l1.y), R2, a01);
        a01 = ff_fma2(ff_pair(h1.z, h1.w, l1.z, l1.w), R3, a01);
        FF2 a23 = ff_mul2(ff_pair(h2.x, h2.y, l2.x, l2.y), R0);
        a23 = ff_fma2(ff_pair(h2.z, h2.w, l2.z, l2.w), R1, a23);
        a23 = ff_fma2(ff_pair(h3.x, h3.y, l3.x, l3.y), R2, a23);
        a23 = ff_fma2(ff_pair(h3.z, h3.w, l3.z, l3.w), R3, a23);
        // outflow traces: t_x = (a0 + c3x a1, a2 + c3x a3), t_y = (a0 + c3y a2, a1 + c3y a3)
        tx[dd] = ff_fma2(C3X, ff_pair(a01.hi.y, a23.hi.y, a01.lo.y, a23.lo.y),
                         ff_pair(a01.hi.x, a23.hi.x, a01.lo.x, a23.lo.x));
        typ[dd] = ff_fma2(C3Y, a23, a01);
        const FF2 W = ff_pair(wh[dd], wh[dd], wl[dd], wl[dd]);
        acc01 = ff_fma2(W, a01, acc01);
        acc23 = ff_fma2(W, a23, acc23);
      }
      double2* po = reinterpret_cast<double2*>(part + 4 * (size_t)c);
      po[0] = make_double2((double)acc01.hi.x + (double)acc01.lo.x,
                           (double)acc01.hi.y + (double)acc01.lo.y);
      po[1] = make_double2((double)acc23.hi.x + (double)acc23.lo.x,
                           (double)acc23.hi.y + (double)acc23.lo.y);
      if (lane == H - 1 && rb + 1 < nrb) {
#pragma unroll
        for (int dd = 0; dd < DPW; ++dd)
          *reinterpret_cast<float4*>(ybuf + (t * DPW + dd) * 4) =
              make_float4(typ[dd].hi.x, typ[dd].hi.y, typ[dd].lo.x, typ[dd].lo.y);
      }
    }
    __syncwarp();
  }
}

template <int DPW>
static int launch2d_ff(const Sweep2DFFArgs& A, int B, int n_groups, cudaStream_t st) {
  const size_t bytes =
      ((size_t)ybuf_ff_floats(A.nx, DPW) + (size_t)A.n_mat * tab_ff_stride(DPW)) * sizeof(float);
  if (bytes > 200 * 1024) return fail(RTE_EINVAL, "float-float sweep: shared memory exceeded");
  if (bytes > 48 * 1024) {
    RTE_CUDA_TRY(cudaFuncSetAttribute(sweep2d_ff_kernel<DPW>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  }
  sweep2d_ff_kernel<DPW><<<dim3(n_groups, B), 32, bytes, st>>>(A); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

// One float-float sweep with source of the active instances of a 2D batch, its partial sums
// reduced in FP64 into rho_out by reduce_partials_kernel (with the stop-test norms when
// fuse_norms, and the correction source when bt->fuse_R is set), as sweep_launch.  Directions
// per warp: the FP64 sweep's choice for this running count, at most 4 (the float-float state of
// 8 directions does not fit the registers of one thread); when the batch's partial-sum buffer
// holds only the groups of 8 directions per warp, the FP64 sweep runs instead.
int sweep_launch_ff(rte_batch_t bt, const double* rho_in, double* rho_out, const uint8_t* active,
                    cudaStream_t st, int n_active, bool fuse_norms, bool zero_norms) {
  const rte_disc_s* d = bt->disc;
  if (d->dim != 2) return fail(RTE_EINVAL, "float-float sweep: 2D only");
  if (n_active < 0) n_active = bt->B;
  int dpw = bt->dpw, n_groups = 0;
  const SweepGroup* gdev = nullptr;
  pick_groups(bt, n_active, &dpw, &n_groups, &gdev);
  if (dpw > 4) {
    if (!bt->groups_all_dev.p ||
        (size_t)std::max(n_active, 1) * bt->gcount[2] * d->n_dof > bt->partial.n)
      return sweep_launch(bt, rho_in, rho_out, nullptr, 1, active, st, fuse_norms, n_active,
                          zero_norms);
    dpw = 4;
    n_groups = bt->gcount[2];
    gdev = bt->groups_all_dev.p + bt->goff[2];
  }
  if (!bt->tablesff.p) {
    RTE_TRY(bt->tablesff.alloc(2 * bt->tables.n));
    RTE_TRY(bt->Sff.alloc(2 * (size_t)bt->B * d->n_dof));
    bt->tablesff_stale = true;
  }
  if (bt->tablesff_stale) {
    const size_t n = bt->tables.n;
    tables_to_ff_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(bt->tables.p, bt->tablesff.p, n); RTE_NOTE_LAUNCH();
    bt->tablesff_stale = false;
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (bt->timing) {
    RTE_CUDA_TRY(cudaEventCreate(&ev0));
    RTE_CUDA_TRY(cudaEventCreate(&ev1));
    RTE_CUDA_TRY(cudaEventRecord(ev0, st));
  }
  cell_source_ff_kernel<<<dim3((d->n_cells + 127) / 128, bt->B), 128, 0, st>>>(
      rho_in, bt->Sff.p, bt->sigma_s.p, bt->G0.p, d->mat_id.p, active, d->n_cells, d->n_mat); RTE_NOTE_LAUNCH();
  RTE_TRY(note_started(bt, st));
  Sweep2DFFArgs A{bt->Sff.p,   bt->partial.p, active,    bt->tablesff.p, bt->inflow.p,
                  d->mat_id.p, d->dir_dev.p,  gdev,      d->nx,          d->ny,
                  d->n_cells,  d->n_dof,      d->n_mat,  d->n_dirs,      n_groups,
                  std::sqrt(d->hx * d->hy),   1.0 / d->hx, 1.0 / d->hy};
  switch (dpw) {
    case 1: RTE_TRY(launch2d_ff<1>(A, bt->B, n_groups, st)); break;
    case 2: RTE_TRY(launch2d_ff<2>(A, bt->B, n_groups, st)); break;
    case 4: RTE_TRY(launch2d_ff<4>(A, bt->B, n_groups, st)); break;
    default: return fail(RTE_EINVAL, "unsupported directions-per-warp");
  }
  if (bt->timing) {
    RTE_CUDA_TRY(cudaEventRecord(ev1, st));
    bt->phase_ev.push_back({4, ev0, ev1});
    bt->phase_calls[4] += 1;
    bt->sweepff_units += (double)n_active * d->n_cells * d->n_dirs;
  }
  if (fuse_norms && zero_norms)
    RTE_CUDA_TRY(cudaMemsetAsync(bt->norms.p, 0, sizeof(unsigned long long) * 2 * bt->B, st));
  const int th = 256;
  dim3 grid((d->n_dof / 2 + th - 1) / th, bt->B);
  reduce_partials_kernel<<<grid, th, 0, st>>>(bt->partial.p, rho_in, rho_out,
                                             fuse_norms ? bt->norms.p : nullptr, active, n_groups,
                                             d->n_dof, bt->fuse_R, bt->sigma_s.p, d->mat_id.p,
                                             d->n_mat); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

}  // namespace rte

extern "C" int rte_sweep_ff(rte_batch_t b, const double* rho_in, double* rho_out,
                            const uint8_t* active, void* stream) {
  if (!b || !rho_in || !rho_out) return fail(RTE_EINVAL, "rte_sweep_ff: null argument");
  RTE_TRY(params_ready(b, "rte_sweep_ff"));
  if (b->disc->dim != 2) return fail(RTE_EINVAL, "rte_sweep_ff: 2D batches only");
  if (rho_in == rho_out) return fail(RTE_EINVAL, "rte_sweep_ff: rho_out aliases rho_in");
  if (((uintptr_t)rho_in | (uintptr_t)rho_out) & 15)
    return fail(RTE_EINVAL, "rte_sweep_ff: arrays must be 16-byte aligned");
  DeviceGuard g(b->disc->device);
  // the group choice is sized for every instance running (the mask is device memory)
  return sweep_launch_ff(b, rho_in, rho_out, active, (cudaStream_t)stream, b->B, false, false);
}
