"""DSA-preconditioned restarted GMRES for (I - L) rho = b-bar: the paper's second comparison system
(Sec. 2.3, "DSA preconditioned Krylov solver"; App. A).  Test infrastructure only.

Reading of the preconditioned system.  Sec. 2.3 writes it as (I + C)(I - L) rho = (I + C) b-bar,
where C turns the change of rho into the DSA correction, delta rho = C Sigma_s (rho* - rho).  The
operator that makes one SI-DSA step a Richardson step is
    rho^(l) = rho^(l-1) + M^{-1} (b-bar - (I - L) rho^(l-1)),   M^{-1} = I + C Sigma_s,
so the left preconditioner is M^{-1} = I + C Sigma_s (the paper's "I + C" with Sigma_s folded in);
the first pin below checks exactly this identity against Alg. 1.

GMRES with restart every m inner steps (App. A): Arnoldi with modified Gram-Schmidt on
w = M^{-1} A v, Givens rotations that track the residual of the preconditioned system, and the
update x = x0 + V y once that residual estimate relative to ||M^{-1} b-bar|| is below rtol or after
m steps.  After every update the residual r = M^{-1}(b-bar - A x) is recomputed from x (App. A
computes it in both places); the solve stops when that recomputed residual meets rtol, otherwise
the next cycle starts from it.  (The recomputation matters when M^{-1} is applied inexactly: the
Arnoldi estimate then drifts from the true residual.)  Inner products are Euclidean on the DG
coefficient vectors (the basis is orthonormal, so this is the L2 inner product of the functions).

Transport sweeps are counted as the paper does: one to form b-bar, one per application of
A = I - L, one per residual recomputation (end of every cycle) and one for the starting residual
when x0 is not zero.
"""
from __future__ import annotations

import numpy as np


def pgmres(tr, rho0, rtol, m=25, max_outer=50, precond=None):
    """Solve (I - L) rho = b-bar for one instance.  precond(R) returns the correction for the
    source R = Sigma_s v (e.g. ConsistentDSA.correction) or None for no preconditioning.
    Returns dict(rho, n_sweep, n_iter, n_cycles, converged, res) with res the relative
    preconditioned residual estimate after every Arnoldi step."""
    n_sweep = 0

    def apply_A(v):
        nonlocal n_sweep
        n_sweep += 1
        return v - tr.L(v)

    def apply_Minv(v):
        if precond is None:
            return v.copy()
        return v + precond(tr.Ss @ v)

    bbar = tr.bbar()
    n_sweep += 1
    x = np.array(rho0, dtype=np.float64, copy=True)
    ref = float(np.linalg.norm(apply_Minv(bbar)))
    r = apply_Minv(bbar - apply_A(x)) if np.any(x) else apply_Minv(bbar)
    res_hist = []
    n_iter = n_cycles = 0
    for _ in range(max_outer):
        beta = float(np.linalg.norm(r))
        if ref == 0.0 or beta / ref <= rtol:
            return dict(rho=x, n_sweep=n_sweep, n_iter=n_iter, n_cycles=n_cycles, converged=True,
                        res=res_hist)
        n_cycles += 1
        V = np.zeros((m + 1, x.size))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        V[0] = r / beta
        g[0] = beta
        k = 0
        for i in range(m):
            w = apply_Minv(apply_A(V[i]))
            n_iter += 1
            for j in range(i + 1):                      # modified Gram-Schmidt
                H[j, i] = float(w @ V[j])
                w = w - H[j, i] * V[j]
            H[i + 1, i] = float(np.linalg.norm(w))
            if H[i + 1, i] > 0.0:
                V[i + 1] = w / H[i + 1, i]
            for j in range(i):                          # earlier rotations on the new column
                t = cs[j] * H[j, i] + sn[j] * H[j + 1, i]
                H[j + 1, i] = -sn[j] * H[j, i] + cs[j] * H[j + 1, i]
                H[j, i] = t
            d = float(np.hypot(H[i, i], H[i + 1, i]))
            cs[i], sn[i] = H[i, i] / d, H[i + 1, i] / d
            H[i, i], H[i + 1, i] = d, 0.0
            g[i + 1] = -sn[i] * g[i]
            g[i] = cs[i] * g[i]
            k = i + 1
            res_hist.append(abs(g[i + 1]) / ref)
            if abs(g[i + 1]) / ref <= rtol:
                break
        # x = x0 + V y with H y = g (upper triangular after the rotations)
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + V[:k].T @ y
        r = apply_Minv(bbar - apply_A(x))               # residual recomputed from the update
    converged = ref == 0.0 or float(np.linalg.norm(r)) / ref <= rtol
    return dict(rho=x, n_sweep=n_sweep, n_iter=n_iter, n_cycles=n_cycles, converged=converged,
                res=res_hist)
