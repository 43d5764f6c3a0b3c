"""POD reduced order models for the parametric problem and the kinetic correction equation
(paper Sec. 3).

* POD (Sec. 3.1.1): thin SVD of the snapshot matrix, truncation rank from Eq. (pod_truncation)
  read literally with singular values: the smallest l with sum_{k<=l} lambda_k / trace >= 1 - eps;
  or a fixed rank.
* Galerkin ROM (Eq. (rom_parametric)): U^T A_mu U c = U^T b_mu.
* Affine precomputation (Sec. 3.1.1): with materials m (cellwise constant, or in 1D linear across
  each cell between the materials of its two ends),
      A_mu = blockdiag_j(D_j + Sigma_t) - (1 omega^T) (x) Sigma_s
           = A_0 + sum_m sigma_{a,m} A_{a,m} + sum_m sigma_{s,m} A_{s,m},
      A_0 = blockdiag_j(D_j),  A_{a,m} = I (x) M_m,  A_{s,m} = I (x) M_m - (1 omega^T) (x) M_m,
  M_m the mass matrix of material m's share of sigma (its indicator, or in 1D the linear function
  that is 1 at the cell ends of material m and 0 at the others); A_{k,r} = U^T A_k U is stored.
* U^rho = sum_j omega_j U_j and U^iso = sum_j U_j (Eq. (rho_basis)).
* ROMIG (Sec. 3.1.1): rho^(0) = U^rho c with c the ROM solution.
* Correction snapshots without solving the correction equation (Sec. 3.2.1):
  delta f^{mu,(l)} = f^mu - f^{mu,(l)} for l <= w_mu = min(n_conv, w).
* ROMSA (Eq. (rom_correction)): (dU^T A_mu dU) dc = (dU^iso)^T Sigma_s (rho* - rho_prev),
  delta rho = dU^rho dc.
* ROMIG followed by ROMSAD (remark after Alg. 2): the correction snapshots must come from
  training runs that start from the ROMIG guess, since the corrections such a run needs differ
  from those of a run started at zero; correction_start="romig" collects them that way.
"""
from __future__ import annotations

import numpy as np

from .dsa import ConsistentDSA
from .sisa import sisa
from .transport import Transport


def pod_rank(sv, eps_pod):
    """Smallest l with sum_{k<=l} lambda_k / sum_k lambda_k >= 1 - eps_POD (Eq. (pod_truncation))."""
    c = np.cumsum(sv) / np.sum(sv)
    return int(np.argmax(c >= 1.0 - eps_pod) + 1)


class POD:
    def __init__(self, S, eps_pod=None, rank=None):
        U, sv, _ = np.linalg.svd(S, full_matrices=False)
        self.sv = sv
        if rank is None:
            rank = pod_rank(sv, eps_pod)
        rank = min(rank, int(np.sum(sv > 0)))
        self.r = rank
        self.U = U[:, :rank]
        # the eps_POD that this rank corresponds to (used for eps_ROMSAD when the rank is fixed)
        self.eps_equiv = float(1.0 - np.sum(sv[:rank]) / np.sum(sv))


class ReducedModel:
    """Reduced operators for a basis U [N_v * N_DOF, r] (angle-major row blocks U_j)."""

    def __init__(self, U, tr_any: Transport):
        tr = tr_any
        self.Nv, self.N = tr.n_angles, tr.n_dof
        self.r = U.shape[1]
        self.U = U
        Uj = U.reshape(self.Nv, self.N, self.r)
        self.w = tr.w.copy()
        self.U_rho = np.einsum("j,jnr->nr", tr.w, Uj)
        self.U_iso = Uj.sum(0)
        self.A0 = sum(Uj[j].T @ (tr.D(j) @ Uj[j]) for j in range(self.Nv))
        mat = tr.problem.mat_id
        mat_r = tr.problem.mat_id_right
        n_mat = tr.problem.n_mat
        self.Aa, self.As = [], []
        for m in range(n_mat):
            if mat_r is None:
                Mm = tr.dg.mass_matrix((mat == m).astype(np.float64))
            else:   # material m's share of a cell: its value at either end, linear in between
                Mm = tr.dg.mass_matrix((mat == m).astype(np.float64), (mat_r == m).astype(np.float64))
            Aam = sum(Uj[j].T @ (Mm @ Uj[j]) for j in range(self.Nv))
            self.Aa.append(Aam)
            self.As.append(Aam - self.U_iso.T @ (Mm @ self.U_rho))
        self._cache = {}

    def operator(self, sigma_t, sigma_s):
        """A_{mu,r} = A_0r + sum_m sigma_{a,m} A_{a,m,r} + sum_m sigma_{s,m} A_{s,m,r}."""
        A = self.A0.copy()
        for m in range(len(self.Aa)):
            A += (sigma_t[m] - sigma_s[m]) * self.Aa[m] + sigma_s[m] * self.As[m]
        return A

    def project_rhs(self, tr: Transport):
        """U^T b_mu with b_mu = (G + g^bc_j)_j (Eq. (rom_parametric) right-hand side)."""
        Uj = self.U.reshape(self.Nv, self.N, self.r)
        return sum(Uj[j].T @ (tr.G + tr.gbc(j)) for j in range(self.Nv))

    def _op_for(self, tr: Transport):
        return self.operator(tr.sigma_t_mat, tr.sigma_s_mat)

    def initial_guess(self, tr: Transport):
        """ROMIG: rho^(0) = U^rho c,  A_{mu,r} c = U^T b_mu."""
        c = np.linalg.solve(self._op_for(tr), self.project_rhs(tr))
        return self.U_rho @ c

    def romsa_correction(self, tr: Transport, R):
        """ROMSA: delta rho = dU^rho dc with (dU^T A_mu dU) dc = (dU^iso)^T R, R = Sigma_s(rho* - rho)."""
        # cache the reduced operator per parameter set (keyed by the values, not the object)
        key = (tuple(tr.sigma_t_mat), tuple(tr.sigma_s_mat))
        if key not in self._cache:
            self._cache = {key: self._op_for(tr)}
        dc = np.linalg.solve(self._cache[key], self.U_iso.T @ R)
        return self.U_rho @ dc


def training_snapshots(train_problem, eps_train, window, n_iter=2000, tol_mode="abs"):
    """The training solves of the offline stage: SI-DSA from rho = 0 for every training parameter,
    the converged angular flux f^mu as a column of F (Sec. 3.1.1) and the correction snapshots
    f^mu - f^{mu,(l)} for l = 1, ..., w_mu = min(n_conv, window), f^{mu,(l)} the angular flux of
    sweep l, as columns of delta F (Sec. 3.2.1).
    Returns (F, dF, n_conv, tr0) with tr0 the first instance's Transport."""
    F_cols, dF_cols, n_conv = [], [], []
    tr0 = None
    for b in range(train_problem.batch):
        tr = Transport(train_problem, b)
        if tr0 is None:
            tr0 = tr
        dsa = ConsistentDSA(tr)
        res = sisa(tr, np.zeros(tr.n_dof), eps_train, n_iter, "dsa", dsa=dsa,
                   window=window, keep_f=True, tol_mode=tol_mode)
        f = res["f"].reshape(-1)
        F_cols.append(f)
        n_conv.append(res["n_sweep"])
        w_mu = min(res["n_sweep"], window)
        for l in range(1, w_mu + 1):   # f_window[l - 1] is the angular flux of sweep l
            dF_cols.append(f - res["f_window"][l - 1].reshape(-1))
        if b > 0:
            tr._lu = [None] * tr.n_angles  # free the factors of finished instances
    return np.stack(F_cols, 1), np.stack(dF_cols, 1), n_conv, tr0


class OfflineROMs:
    """Offline stage: training SI-DSA solves, snapshot matrices F and delta F, two POD bases."""

    def __init__(self, train_problem, eps_train=1e-12, window=3, rank_p=None, rank_c=None,
                 eps_pod=None, n_iter=2000, tol_mode="abs", correction_start="zero"):
        assert correction_start in ("zero", "romig")
        self.F, self.dF, n_conv, tr0 = training_snapshots(train_problem, eps_train, window, n_iter,
                                                          tol_mode)
        self.n_conv = n_conv
        self.pod_p = POD(self.F, eps_pod, rank_p)
        self.rom_p = ReducedModel(self.pod_p.U, tr0)
        if correction_start == "romig":
            # second pass: the same training solves started from the ROMIG guess
            dF_cols, n_conv = [], []
            for b in range(train_problem.batch):
                tr = Transport(train_problem, b)
                rho0 = self.rom_p.initial_guess(tr)
                res = sisa(tr, rho0, eps_train, n_iter, "dsa", dsa=ConsistentDSA(tr),
                           window=window, keep_f=True, tol_mode=tol_mode)
                f = res["f"].reshape(-1)
                n_conv.append(res["n_sweep"])
                for l in range(1, min(res["n_sweep"], window) + 1):
                    dF_cols.append(f - res["f_window"][l - 1].reshape(-1))
            self.n_conv_romig = n_conv
            self.dF = np.stack(dF_cols, 1)
        self.pod_c = POD(self.dF, eps_pod, rank_c)
        self.rom_c = ReducedModel(self.pod_c.U, tr0)
        self.eps_train = eps_train
        self.eps_pod = self.pod_c.eps_equiv if eps_pod is None else eps_pod
