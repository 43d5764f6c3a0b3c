"""Transport sweep, the operator L, the coupled system and the residual (paper Sec. 2.2-2.3.1).

One ``Transport`` object holds one parametric instance.  The sweep is Eq. (transport_sweep):
for every direction j solve (D_j + Sigma_t) f_j = Sigma_s rho + G + g^bc_j, then
rho* = sum_j omega_j f_j.  (D_j + Sigma_t) is block lower triangular in the upwind ordering of
the cells (Sec. 2.3); the oracle does not rely on that structure -- it factors each matrix with
a sparse LU and solves, which gives the same f_j up to rounding.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .dg import make_dg
from .quadrature import rule_for


class Transport:
    def __init__(self, problem, b: int = 0):
        problem.validate()
        self.problem = problem
        self.dim = problem.dim
        self.dg = make_dg(problem)
        self.v, self.w = rule_for(problem)
        self.n_angles = self.w.size
        mat = problem.mat_id
        self.sigma_t_mat = problem.sigma_t[b].copy()      # per-material table of this instance
        self.sigma_s_mat = problem.sigma_s[b].copy()
        self.sigma_t_cell = problem.sigma_t[b][mat]
        self.sigma_s_cell = problem.sigma_s[b][mat]
        self.sigma_a_cell = self.sigma_t_cell - self.sigma_s_cell
        # 1D cross sections linear across each cell: the values at the cells' right ends
        self.linear = problem.mat_id_right is not None
        if self.linear:
            mr = problem.mat_id_right
            self.sigma_t_right = problem.sigma_t[b][mr]
            self.sigma_s_right = problem.sigma_s[b][mr]
            self.sigma_a_right = self.sigma_t_right - self.sigma_s_right
            self.St = self.dg.mass_matrix(self.sigma_t_cell, self.sigma_t_right)
            self.Ss = self.dg.mass_matrix(self.sigma_s_cell, self.sigma_s_right)
            self.Sa = self.dg.mass_matrix(self.sigma_a_cell, self.sigma_a_right)
        else:
            self.St = self.dg.mass_matrix(self.sigma_t_cell)
            self.Ss = self.dg.mass_matrix(self.sigma_s_cell)
            self.Sa = self.dg.mass_matrix(self.sigma_a_cell)
        self.G = self.dg.source_vector(problem.source[b])
        self.inflow = problem.inflow[b]
        self.n_dof = self.dg.n_dof
        self._D = [None] * self.n_angles
        self._lu = [None] * self.n_angles
        self._gbc = [None] * self.n_angles

    # ---- per-direction pieces ------------------------------------------------------------
    def D(self, j):
        if self._D[j] is None:
            self._D[j] = self.dg.transport_matrix(self.v[j])
        return self._D[j]

    def gbc(self, j):
        if self._gbc[j] is None:
            self._gbc[j] = self.dg.inflow_vector(self.v[j], self.inflow)
        return self._gbc[j]

    def lu(self, j):
        if self._lu[j] is None:
            self._lu[j] = spla.splu((self.D(j) + self.St).tocsc())
        return self._lu[j]

    # ---- the sweep -------------------------------------------------------------------------
    def sweep(self, rho, with_source=True, store_f=False, extra_rhs=None):
        """One source iteration (Alg. 1 / Eq. (transport_sweep)):
            f_j = (D_j + Sigma_t)^{-1} (Sigma_s rho + G + g^bc_j),   rho* = sum_j omega_j f_j.
        with_source=False drops G and g^bc (the operator L of Eq. (rho_matrix_vec_def));
        extra_rhs[j] (optional) is added to direction j's right-hand side.
        Returns rho* (and f [N_v, N_DOF] when store_f)."""
        s = self.Ss @ rho
        if with_source:
            s = s + self.G
        rho_star = np.zeros(self.n_dof)
        f = np.zeros((self.n_angles, self.n_dof)) if store_f else None
        for j in range(self.n_angles):
            rhs = s + self.gbc(j) if with_source else s.copy()
            if extra_rhs is not None:
                rhs = rhs + extra_rhs[j]
            fj = self.lu(j).solve(rhs)
            rho_star += self.w[j] * fj
            if store_f:
                f[j] = fj
        return (rho_star, f) if store_f else rho_star

    def L(self, rho):
        """L rho = sum_j omega_j (D_j + Sigma_t)^{-1} Sigma_s rho (Eq. (rho_matrix_vec_def))."""
        return self.sweep(rho, with_source=False)

    def bbar(self):
        """b-bar = sum_j omega_j (D_j + Sigma_t)^{-1} (G + g^bc_j) (Eq. (rho_matrix_vec_def))."""
        return self.sweep(np.zeros(self.n_dof))

    def residual_inf(self, rho):
        """||(I - L) rho - b-bar||_inf, the quantity averaged into R^rho_inf (Sec. 4.1.2)."""
        return float(np.max(np.abs(rho - self.sweep(rho))))

    # ---- direct references for small cases ----------------------------------------------------
    def coupled_system(self):
        """Dense A and b of Eq. (one_equation): A_jj = D_j + Sigma_t - omega_j Sigma_s,
        A_ji = -omega_i Sigma_s, b_j = G + g^bc_j."""
        N, Nv = self.n_dof, self.n_angles
        A = np.zeros((Nv * N, Nv * N))
        Ss = self.Ss.toarray()
        for j in range(Nv):
            for i in range(Nv):
                blk = -self.w[i] * Ss
                if i == j:
                    blk = blk + (self.D(j) + self.St).toarray()
                A[j * N:(j + 1) * N, i * N:(i + 1) * N] = blk
        b = np.concatenate([self.G + self.gbc(j) for j in range(Nv)])
        return A, b

    def solve_direct(self):
        """f and rho from a dense solve of A f = b (only for small cases)."""
        A, b = self.coupled_system()
        f = np.linalg.solve(A, b).reshape(self.n_angles, self.n_dof)
        rho = np.einsum("j,jn->n", self.w, f)
        return rho, f

    def L_dense(self):
        """L as a dense matrix, one column per unit vector (small cases)."""
        N = self.n_dof
        L = np.zeros((N, N))
        for k in range(N):
            e = np.zeros(N)
            e[k] = 1.0
            L[:, k] = self.L(e)
        return L

    def solve_rho_direct(self):
        """rho from (I - L) rho = b-bar (Eq. (rho_matrix_vec_def)), dense (small cases)."""
        L = self.L_dense()
        return np.linalg.solve(np.eye(self.n_dof) - L, self.bbar())

    # ---- kinetic correction (Eq. (discrete_correction)), solved exactly --------------------------
    def exact_correction(self, R, L_dense=None):
        """delta rho of the discrete kinetic correction equation with source R = Sigma_s(rho* - rho):
        (D_j + Sigma_t) df_j = Sigma_s drho + R, drho = sum omega_j df_j, zero inflow, i.e.
        (I - L) drho = K R with K R = sum_j omega_j (D_j + Sigma_t)^{-1} R."""
        L = self.L_dense() if L_dense is None else L_dense
        KR = np.zeros(self.n_dof)
        for j in range(self.n_angles):
            KR += self.w[j] * self.lu(j).solve(R)
        return np.linalg.solve(np.eye(self.n_dof) - L, KR)


def cell_balance(tr: Transport, rho_prev, f):
    """Per-cell particle balance of one sweep (test function = the cell's indicator, whose
    gradient vanishes, in Eq. (DG)):
        sum_j omega_j int_{dT} (v_j.n) f_hat_j + int_T sigma_t rho* - int_T (sigma_s rho_prev + G),
    which is zero for an exact sweep.  Edge fluxes come from traces (``net_upwind_outflow``),
    not from D_j, so the check is independent of the assembled matrices."""
    dg = tr.dg
    P = dg.P
    n = dg.n_cells
    rho_star = np.einsum("j,jn->n", tr.w, f)
    area = dg.h if tr.dim == 1 else np.full(n, dg.hx * dg.hy)
    sq = np.sqrt(area)           # int_T u = sqrt(|T|) u_0 for the orthonormal basis
    rs, rp = rho_star.reshape(n, P), rho_prev.reshape(n, P)
    if tr.linear:
        # sigma = sbar + (sR - sL) xi / 2 and u = u_0 phi_0 + u_1 phi_1 on a cell of width h:
        # int sigma u = sqrt(h) (sbar u_0 + (sR - sL) u_1 / (2 sqrt 3))
        def moment(sl, sr, u):
            return 0.5 * (sl + sr) * u[:, 0] + (sr - sl) / (2.0 * np.sqrt(3.0)) * u[:, 1]
        bal = sq * (moment(tr.sigma_t_cell, tr.sigma_t_right, rs)
                    - moment(tr.sigma_s_cell, tr.sigma_s_right, rp) - tr.G.reshape(n, P)[:, 0])
    else:
        bal = sq * (tr.sigma_t_cell * rs[:, 0] - tr.sigma_s_cell * rp[:, 0]
                    - tr.G.reshape(n, P)[:, 0])
    for j in range(tr.n_angles):
        bal += tr.w[j] * dg.net_upwind_outflow(tr.v[j], f[j], tr.inflow)
    return bal
