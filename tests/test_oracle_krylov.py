"""Pins for the oracle's DSA-preconditioned GMRES (Sec. 2.3; App. A).

* The preconditioned residual is one SI-DSA step: rho + M^{-1}(b-bar - (I - L) rho) equals the
  iterate Alg. 1 returns after one sweep and one DSA correction (pins M^{-1} = I + C Sigma_s and
  every sign in it).
* With the exact kinetic correction as "C", M^{-1} = (I - L)^{-1}, so GMRES stops after one step
  at the direct solution of (I - L) rho = b-bar.
* Without preconditioning GMRES terminates in at most n_dof steps (exact arithmetic property of
  Krylov methods), at the direct solution.
* With restarts the solution is the same; the sweep count exceeds the GMRES step count by one
  (b-bar) plus one per cycle (the residual recomputed after each update), plus one for a nonzero
  start (the paper's accounting: at most 3 more sweeps than steps when no restart happens).
"""
import numpy as np

from oracle.dsa import ConsistentDSA
from oracle.krylov import pgmres
from oracle.sisa import sisa
from oracle.transport import Transport
from paper_2402_10488_gb300 import inputs


def _lattice():
    return Transport(inputs.lattice_test(6, 8, 1, n_vz=2), 0)


def test_preconditioned_residual_is_one_si_dsa_step():
    for tr in (_lattice(), Transport(inputs.slab_random(12, 8, 3, seed=4, inflow=(0.5, 1.0)), 0)):
        dsa = ConsistentDSA(tr)
        rho = np.random.default_rng(3).uniform(0, 1, tr.n_dof)
        step = sisa(tr, rho, 0.0, 1, "dsa", dsa=dsa)["rho"]
        r = tr.bbar() - (rho - tr.L(rho))
        minv_r = r + dsa.correction(tr.Ss @ r)
        np.testing.assert_allclose(rho + minv_r, step, atol=1e-12 * np.abs(step).max())


def test_exact_correction_preconditioner_converges_in_one_step():
    tr = _lattice()
    Ld = tr.L_dense()
    exact = tr.solve_rho_direct()
    res = pgmres(tr, np.zeros(tr.n_dof), 1e-12, m=10, precond=lambda R: tr.exact_correction(R, Ld))
    assert res["converged"] and res["n_iter"] == 1 and res["n_cycles"] == 1
    np.testing.assert_allclose(res["rho"], exact, atol=1e-11 * np.abs(exact).max())


def test_unpreconditioned_gmres_terminates_within_n_dof_steps():
    tr = Transport(inputs.slab_random(4, 4, 2, seed=7, inflow=(1.0, 0.3)), 0)
    exact = tr.solve_rho_direct()
    res = pgmres(tr, np.zeros(tr.n_dof), 1e-13, m=tr.n_dof, max_outer=1)
    assert res["converged"] and res["n_iter"] <= tr.n_dof
    np.testing.assert_allclose(res["rho"], exact, atol=1e-11 * np.abs(exact).max())


def test_dsa_gmres_converges_and_counts_sweeps_with_restarts():
    tr = _lattice()
    dsa = ConsistentDSA(tr)
    exact = tr.solve_rho_direct()
    full = pgmres(tr, np.zeros(tr.n_dof), 1e-12, m=25, precond=dsa.correction)
    assert full["converged"]
    np.testing.assert_allclose(full["rho"], exact, atol=1e-10 * np.abs(exact).max())
    assert full["n_cycles"] == 1                          # converged before restart
    assert full["n_sweep"] == full["n_iter"] + 2
    assert all(np.diff(full["res"]) <= 1e-15)             # GMRES residuals never increase
    short = pgmres(tr, np.zeros(tr.n_dof), 1e-12, m=2, precond=dsa.correction)
    assert short["converged"] and short["n_cycles"] >= (short["n_iter"] + 1) // 2
    assert short["n_sweep"] == short["n_iter"] + 1 + short["n_cycles"]
    np.testing.assert_allclose(short["rho"], exact, atol=1e-10 * np.abs(exact).max())
    # a nonzero start costs one more sweep for its residual
    warm = pgmres(tr, 0.5 * exact, 1e-12, m=25, precond=dsa.correction)
    assert warm["converged"] and warm["n_sweep"] == warm["n_iter"] + 1 + warm["n_cycles"] + 1
