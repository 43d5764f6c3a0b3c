"""Source Iteration with Synthetic Acceleration (paper Alg. 1) and the ROMSAD switch (Alg. 2).

    for l = 1, 2, ..., N_iter:
        sweep:       f^(l)_j = (D_j + Sigma_t)^{-1} (G~_j + Sigma_s rho^(l-1)),  rho^(l,*) = sum omega_j f^(l)_j
        stop test:   ||rho^(l,*) - rho^(l-1)||_inf < eps  ->  return rho^(l,*)
        correction:  rho^(l) = rho^(l,*) + delta rho^(l)

SA choices: 'none' (plain SI), 'exact' (the kinetic correction equation solved exactly,
Eq. (discrete_correction); small cases only), 'dsa' (App. B), 'romsa' (Eq. (rom_correction)),
'romsad' (Alg. 2: ROMSA after iteration l iff 1 <= l <= theta and the change is >= eps_ROMSAD,
otherwise DSA).

Reading of the stop test: the paper's test is absolute (Alg. 1); ``tol_mode='rel'`` divides the
change by ||rho^(l,*)||_inf.  The ROMSAD switch always compares the absolute change, as Alg. 2
writes it.  When N_iter sweeps pass without the test firing, the last corrected iterate
rho^(N_iter) is returned with converged = False.
"""
from __future__ import annotations

import numpy as np


def sisa(tr, rho0, eps, n_iter=1000, sa="dsa", dsa=None, rom_c=None, theta=0,
         eps_romsad=0.0, tol_mode="abs", window=0, keep_f=False, schedule=None,
         keep_iterates=False, L_dense=None):
    """Run Alg. 1 on one instance.  Returns a dict with rho, n_sweep, converged, the history of
    changes ||rho^(l,*) - rho^(l-1)||_inf and SA choices, and (window > 0) the angular fluxes
    f^(l) of the first ``window`` sweeps plus (keep_f) the final f."""
    rho_prev = np.array(rho0, dtype=np.float64, copy=True)
    hist = dict(delta=[], sa=[], f_window=[], rho_star_hist=[], rho_hist=[])
    store = keep_f or window > 0
    f = None
    for l in range(1, n_iter + 1):
        if store:
            rho_star, f = tr.sweep(rho_prev, store_f=True)
        else:
            rho_star = tr.sweep(rho_prev)
        delta = float(np.max(np.abs(rho_star - rho_prev)))
        hist["delta"].append(delta)
        if l <= window:
            hist["f_window"].append(f.copy())
        if keep_iterates:
            hist["rho_star_hist"].append(rho_star.copy())
        test = delta / float(np.max(np.abs(rho_star))) if tol_mode == "rel" else delta
        if test < eps:
            return dict(rho=rho_star, n_sweep=l, converged=True, f=f, **hist)
        R = tr.Ss @ (rho_star - rho_prev)
        choice = sa
        if sa == "romsad":
            if schedule is not None:
                choice = schedule[l - 1]
            else:
                choice = "romsa" if (1 <= l <= theta and delta >= eps_romsad) else "dsa"
        if choice == "none":
            drho = np.zeros_like(R)
        elif choice == "exact":
            drho = tr.exact_correction(R, L_dense)
        elif choice == "dsa":
            drho = dsa.correction(R)
        elif choice == "romsa":
            drho = rom_c.romsa_correction(tr, R)
        else:
            raise ValueError(choice)
        hist["sa"].append(choice)
        rho_prev = rho_star + drho
        if keep_iterates:
            hist["rho_hist"].append(rho_prev.copy())
    return dict(rho=rho_prev, n_sweep=n_iter, converged=False, f=f, **hist)


def romsad_eps(eps_train, eps_pod, eta=0.1):
    """eps_ROMSAD = eta * max(eps_SISA^train, eps_POD) (Eq. (romsad_parameters)); eta = 0.1 in
    all of the paper's tests (Sec. 4)."""
    return eta * max(eps_train, eps_pod)
