"""Pins for 1D cross sections linear inside each cell (the cross-regime problem of Sec. 4.1.1 has
sigma_s(x) = 0.1 + mu_s x, linear inside every cell).

* The mass matrix int sigma phi_k phi_l with linear sigma against scipy's adaptive quadrature of
  the same integral on cells of a non-uniform mesh, and equal to the cellwise-constant one when
  both ends carry the same value.
* Pure absorber: the outflow of one DG-P^1 cell with sigma going linearly from s_L to s_R is
  psi_in R(t_L, t_R), t = s h / |xi|, with R derived by hand from the 2x2 cell system:
      R = 6 (6 - t_L - t_R) / (36 + 12 (t_L + t_R) + t_L^2 + 4 t_L t_R + t_R^2)
  (t_L = t_R = t gives the (1,2) Pade ratio of the constant case); N cells multiply their ratios.
  R is symmetric in (t_L, t_R), so this pins the cell average and the diagonal of the mass
  matrix but not the sign of its off-diagonal; the particle balance below pins that sign.
* Particle balance of one sweep with the cell integrals int sigma u written in closed form
  (sqrt(h) (sbar u_0 + (s_R - s_L) u_1 / (2 sqrt 3))), independent of the assembled matrices.
* Consistent DSA built with the linear Sigma_a, Sigma_t keeps SI-DSA's fast contraction in a
  thick linear slab, where SI alone stalls; the converged solution equals the direct solve.
* The affine reduced operators (one term per material; material m's share of a cell is linear,
  1 at the cell ends carrying m) equal U^T A_mu U of the directly assembled A_mu.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle.dg import DG1D
from oracle.dsa import ConsistentDSA
from oracle.rom import OfflineROMs
from oracle.sisa import sisa
from oracle.transport import Transport, cell_balance
from paper_2402_10488_gb300 import inputs


def _basis(h, k, xi):
    """phi_0 = 1/sqrt(h), phi_1 = sqrt(3/h) xi on a cell of width h, xi in [-1, 1]."""
    return 1.0 / np.sqrt(h) if k == 0 else np.sqrt(3.0 / h) * xi


def test_linear_mass_matrix_against_adaptive_quadrature():
    edges = np.array([0.0, 0.13, 0.5, 0.61, 1.4])
    dg = DG1D(edges)
    rng = np.random.default_rng(11)
    sl, sr = rng.uniform(0.1, 5.0, 4), rng.uniform(0.1, 5.0, 4)
    M = dg.mass_matrix(sl, sr).toarray()
    for c in range(4):
        h, x0 = edges[c + 1] - edges[c], edges[c]
        for k in range(2):
            for l in range(2):
                def fun(x):
                    xi = 2.0 * (x - x0) / h - 1.0
                    sig = sl[c] + (sr[c] - sl[c]) * (x - x0) / h
                    return sig * _basis(h, k, xi) * _basis(h, l, xi)
                ref, _ = integrate.quad(fun, x0, x0 + h, epsabs=1e-15, epsrel=1e-12)
                assert abs(M[2 * c + k, 2 * c + l] - ref) < 1e-12
    # equal ends: the cellwise-constant matrix
    np.testing.assert_allclose(dg.mass_matrix(sl, sl).toarray(), dg.mass_matrix(sl).toarray(),
                               atol=1e-14)


def _ratio(tl, tr):
    return 6.0 * (6.0 - tl - tr) / (36.0 + 12.0 * (tl + tr) + tl * tl + 4.0 * tl * tr + tr * tr)


def test_linear_pure_absorber_closed_form():
    edges = np.array([0.0, 0.1, 0.25, 0.3, 0.55, 0.8])
    n = edges.size - 1
    x_nodes = edges
    sig_nodes = 1.0 + 6.0 * x_nodes ** 2          # values at the cell ends (materials = nodes)
    p = inputs.Problem(1, n, 1, (0.0, 0.8), "gl", 8, 0, np.arange(n, dtype=np.int32),
                       sig_nodes[None, :].copy(), np.zeros((1, n + 1)), np.zeros((1, n)),
                       np.array([[1.3, 0.7]]), None, "absorber_linear", edges,
                       mat_id_right=np.arange(1, n + 1, dtype=np.int32))
    tr = Transport(p)
    _, f = tr.sweep(np.zeros(tr.n_dof), store_f=True)
    h = np.diff(edges)
    for j in range(8):
        xi = tr.v[j, 0]
        fc = f[j].reshape(n, 2)
        if xi > 0:
            out = tr.dg.trace(n - 1, +1) @ fc[-1]
            expect = 1.3 * np.prod([_ratio(sig_nodes[c] * h[c] / xi, sig_nodes[c + 1] * h[c] / xi)
                                    for c in range(n)])
        else:
            out = tr.dg.trace(0, -1) @ fc[0]
            expect = 0.7 * np.prod([_ratio(sig_nodes[c + 1] * h[c] / -xi, sig_nodes[c] * h[c] / -xi)
                                    for c in range(n)])
        assert abs(out - expect) <= 1e-13 * max(1.3, 0.7)


@pytest.mark.parametrize("seed", [3, 4])
def test_particle_balance_of_one_linear_sweep(seed):
    p = inputs.slab_random(17, 8, 4, seed=seed, inflow=(1.0, 2.0), linear=True)
    p = inputs.replace(p, edges=np.sort(np.concatenate([[0.0, 1.0],
                                                        np.random.default_rng(seed).uniform(0, 1, 16)])))
    tr = Transport(p)
    assert tr.linear
    rho0 = np.random.default_rng(0).normal(size=tr.n_dof)
    _, f = tr.sweep(rho0, store_f=True)
    assert np.max(np.abs(cell_balance(tr, rho0, f))) < 1e-12


def test_planted_off_diagonal_sign_error_fails_the_balance():
    """The balance pin sees a flipped off-diagonal in the sweep's Sigma_t (the pure absorber's
    outflow cannot: R is symmetric)."""
    p = inputs.slab_random(17, 8, 4, seed=3, inflow=(1.0, 2.0), linear=True)
    tr = Transport(p)
    St = tr.St.tolil()
    for c in range(tr.dg.n_cells):
        St[2 * c, 2 * c + 1] = -St[2 * c, 2 * c + 1]
        St[2 * c + 1, 2 * c] = -St[2 * c + 1, 2 * c]
    tr.St = St.tocsr()
    rho0 = np.random.default_rng(0).normal(size=tr.n_dof)
    _, f = tr.sweep(rho0, store_f=True)
    assert np.max(np.abs(cell_balance(tr, rho0, f))) > 1e-6


def test_si_dsa_contracts_fast_in_thick_linear_slab():
    """Cross-regime profile made thick everywhere: sigma_s from 50 to 550 (c = 1 - 1e-4 at the
    ends: sigma_a = 1e-4 sigma_t)."""
    n = 100
    xe = np.linspace(0.0, 10.0, n + 1)
    st = 50.0 + 50.0 * xe
    p = inputs.Problem(1, n, 1, (0.0, 10.0), "gl", 16, 0, np.arange(n, dtype=np.int32),
                       st[None, :].copy(), (st * (1 - 1e-4))[None, :].copy(), np.full((1, n), 0.01),
                       np.zeros((1, 2)), None, "thick_linear",
                       mat_id_right=np.arange(1, n + 1, dtype=np.int32))
    tr = Transport(p)
    r = sisa(tr, np.zeros(tr.n_dof), 1e-10, 100, "dsa", dsa=ConsistentDSA(tr), tol_mode="rel")
    assert r["converged"] and r["n_sweep"] <= 15
    d = np.array(r["delta"])
    assert np.all(d[2:] / d[1:-1] < 0.3)
    si = sisa(tr, np.zeros(tr.n_dof), 1e-10, 30, "none", tol_mode="rel")
    assert not si["converged"]
    ref = tr.solve_rho_direct()
    np.testing.assert_allclose(r["rho"], ref, atol=1e-8 * np.abs(ref).max())


def test_affine_reduced_operators_with_linear_materials():
    train = inputs.cross_regime(10.0 + np.arange(5) * 2.5, n=24)
    off = OfflineROMs(train, eps_train=1e-12, window=2, rank_p=4, rank_c=6)
    test = inputs.cross_regime(np.array([12.3, 17.9]), n=24)
    for b in range(2):
        tr = Transport(test, b)
        A, bvec = tr.coupled_system()
        for rom in (off.rom_p, off.rom_c):
            U = rom.U
            ref = U.T @ A @ U
            np.testing.assert_allclose(rom.operator(test.sigma_t[b], test.sigma_s[b]), ref,
                                       atol=1e-10 * np.abs(ref).max())
            np.testing.assert_allclose(rom.project_rhs(tr), U.T @ bvec, atol=1e-12)


def test_cross_regime_linear_and_cellwise_readings_are_close():
    """sigma_s linear in cells vs its cell averages: the two discrete solutions differ by the
    O(h^2) difference of the two representations of sigma_s (1.7e-4 relative at 100 cells)."""
    lin = Transport(inputs.cross_regime([14.0], n=100))
    avg = Transport(inputs.cross_regime([14.0], n=100, linear=False))
    a, b = lin.solve_rho_direct(), avg.solve_rho_direct()
    rel = np.abs(a - b).max() / np.abs(b).max()
    assert 0.0 < rel < 1e-3
