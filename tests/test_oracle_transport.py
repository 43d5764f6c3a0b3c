"""Pins for the oracle's transport sweep and coupled system (Sec. 2.2-2.3.1): the pure-absorber
closed form, exact reproduction of manufactured Q^1 solutions, constant states, particle
balance, agreement of the two direct formulations, and the SI convergence statement."""
import numpy as np
import pytest

from oracle.dsa import ConsistentDSA
from oracle.sisa import sisa
from oracle.transport import Transport, cell_balance
from paper_2402_10488_gb300 import inputs


def pade_12(tau):
    """Outflow/inflow ratio of one DG-P^1 cell of optical depth tau for a pure absorber,
    derived by hand from the 2x2 cell system: (1 - tau/3) / (1 + 2 tau/3 + tau^2/6), the (1,2)
    Pade approximant of exp(-tau)."""
    return (1.0 - tau / 3.0) / (1.0 + 2.0 * tau / 3.0 + tau * tau / 6.0)


def outflow_value(tr, f, j):
    """Point value of direction j's solution at the slab end it leaves through."""
    fc = f[j].reshape(tr.dg.n_cells, 2)
    xi = tr.v[j, 0]
    if xi > 0:
        return tr.dg.trace(tr.dg.n_cells - 1, +1) @ fc[-1]
    return tr.dg.trace(0, -1) @ fc[0]


def test_pure_absorber_pade_closed_form():
    n, sig, g = 12, 3.0, 1.7
    p = inputs.slab(n, 8, sig, 0.0, G=0.0, inflow=(g, 2 * g), domain=(0.0, 1.5))
    tr = Transport(p)
    _, f = tr.sweep(np.zeros(tr.n_dof), store_f=True)
    h = 1.5 / n
    for j in range(8):
        xi = tr.v[j, 0]
        gin = g if xi > 0 else 2 * g
        expect = gin * pade_12(sig * h / abs(xi)) ** n
        assert abs(outflow_value(tr, f, j) - expect) <= 1e-13 * gin


def test_pure_absorber_converges_to_exponential_at_third_order():
    """As h -> 0 the outflow tends to psi_in exp(-sigma_t L / |xi|) (characteristics), with the
    O(h^3) global error of the (1,2) Pade step."""
    sig, L = 2.0, 1.0
    errs = []
    for n in (8, 16, 32):
        tr = Transport(inputs.slab(n, 2, sig, 0.0, G=0.0, inflow=(1.0, 0.0)))
        _, f = tr.sweep(np.zeros(tr.n_dof), store_f=True)
        j = int(np.argmax(tr.v[:, 0]))
        errs.append(abs(outflow_value(tr, f, j) - np.exp(-sig * L / tr.v[j, 0])))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.9) and np.all(rates < 3.1)


def _q1_moments(dg, fun):
    """Cell moments int fun phi_k with the test's own 4x4 Gauss rule (numpy's leggauss)."""
    x, w = np.polynomial.legendre.leggauss(4)
    out = np.zeros((dg.n_cells, 4))
    for c in range(dg.n_cells):
        j, i = divmod(c, dg.nx)
        xc, yc = dg.x0 + (i + 0.5) * dg.hx, dg.y0 + (j + 0.5) * dg.hy
        for qa in range(4):
            for qb in range(4):
                X, Y = xc + x[qa] * dg.hx / 2, yc + x[qb] * dg.hy / 2
                wt = w[qa] * w[qb] * dg.hx * dg.hy / 4
                px = np.array([1.0, np.sqrt(3.0) * x[qa]]) / np.sqrt(dg.hx)
                py = np.array([1.0, np.sqrt(3.0) * x[qb]]) / np.sqrt(dg.hy)
                phi = np.array([px[0] * py[0], px[1] * py[0], px[0] * py[1], px[1] * py[1]])
                out[c] += wt * fun(X, Y) * phi
    return out.reshape(-1)


def _inflow_moments(dg, v, fun):
    """-int over inflow boundary edges of fun phi_k (v.n), the test's own edge quadrature."""
    x, w = np.polynomial.legendre.leggauss(4)
    out = np.zeros((dg.n_cells, 4))
    for c in range(dg.n_cells):
        j, i = divmod(c, dg.nx)
        xc, yc = dg.x0 + (i + 0.5) * dg.hx, dg.y0 + (j + 0.5) * dg.hy
        edges = []
        if i == 0:
            edges.append(((-1.0, 0.0), "x", -1.0))
        if i == dg.nx - 1:
            edges.append(((1.0, 0.0), "x", 1.0))
        if j == 0:
            edges.append(((0.0, -1.0), "y", -1.0))
        if j == dg.ny - 1:
            edges.append(((0.0, 1.0), "y", 1.0))
        for n, axis, s in edges:
            vn = v[0] * n[0] + v[1] * n[1]
            if vn >= 0:
                continue
            for q in range(4):
                if axis == "x":
                    xi, eta, L = s, x[q], dg.hy
                else:
                    xi, eta, L = x[q], s, dg.hx
                X, Y = xc + xi * dg.hx / 2, yc + eta * dg.hy / 2
                px = np.array([1.0, np.sqrt(3.0) * xi]) / np.sqrt(dg.hx)
                py = np.array([1.0, np.sqrt(3.0) * eta]) / np.sqrt(dg.hy)
                phi = np.array([px[0] * py[0], px[1] * py[0], px[0] * py[1], px[1] * py[1]])
                out[c] += -w[q] * L / 2 * fun(X, Y) * phi * vn
    return out.reshape(-1)


def test_2d_sweep_reproduces_bilinear_solution_exactly():
    """A globally continuous bilinear psi_j lies in the DG space and satisfies the DG equations
    with source v.grad(psi) + sigma_t psi and inflow psi: the sweep must return it exactly."""
    p = inputs.random_2d(5, 4, 2, 1, seed=11, ny=4)
    p.sigma_s[:] = 0.0
    tr = Transport(p)
    sig = p.sigma_t[0, 0]
    dg = tr.dg
    rng = np.random.default_rng(3)
    coef = rng.normal(size=(tr.n_angles, 4))
    extra, expect = [], []
    for jd in range(tr.n_angles):
        a, b, c, d = coef[jd]
        vx, vy = tr.v[jd, 0], tr.v[jd, 1]
        psi = lambda X, Y, a=a, b=b, c=c, d=d: a + b * X + c * Y + d * X * Y
        q = lambda X, Y, a=a, b=b, c=c, d=d, vx=vx, vy=vy: (vx * (b + d * Y) + vy * (c + d * X)
                                                            + sig * (a + b * X + c * Y + d * X * Y))
        extra.append(_q1_moments(dg, q) + _inflow_moments(dg, tr.v[jd], psi))
        expect.append(_q1_moments(dg, psi))
    _, f = tr.sweep(np.zeros(tr.n_dof), with_source=False, store_f=True, extra_rhs=extra)
    np.testing.assert_allclose(f, np.array(expect), atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2])
def test_constant_state_with_scattering(dim):
    """Homogeneous medium, isotropic inflow g = G / sigma_a on every side: rho = G / sigma_a."""
    st, ss, G = 3.0, 2.5, 1.0
    g = G / (st - ss)
    if dim == 1:
        p = inputs.slab(6, 8, st, ss, G=G, inflow=(g, g))
    else:
        p = inputs.random_2d(5, 8, 2, 1, seed=1, inflow=(g,) * 4)
        p.sigma_t[:], p.sigma_s[:], p.source[:] = st, ss, G
    tr = Transport(p)
    rho = tr.solve_rho_direct().reshape(tr.dg.n_cells, tr.dg.P)
    area = tr.dg.h if dim == 1 else tr.dg.hx * tr.dg.hy
    np.testing.assert_allclose(rho[:, 0] / np.sqrt(area), g, rtol=1e-13)
    np.testing.assert_allclose(rho[:, 1:], 0.0, atol=1e-13)


@pytest.mark.parametrize("make", [
    lambda: inputs.slab_random(17, 8, 3, seed=3, inflow=(1.0, 2.0)),
    lambda: inputs.random_2d(7, 8, 2, 3, seed=2, inflow=(0.5, 1.0, 0.0, 2.0)),
])
def test_particle_balance_of_one_sweep(make):
    tr = Transport(make())
    rho0 = np.random.default_rng(0).normal(size=tr.n_dof)
    _, f = tr.sweep(rho0, store_f=True)
    assert np.max(np.abs(cell_balance(tr, rho0, f))) < 1e-12


def test_coupled_system_and_rho_system_agree_and_si_dsa_converges_to_them():
    p = inputs.random_2d(4, 4, 2, 2, seed=7, inflow=(1.0, 0.0, 0.5, 0.0))
    tr = Transport(p)
    rho_f, f = tr.solve_direct()          # A f = b, Eq. (one_equation)
    rho_r = tr.solve_rho_direct()         # (I - L) rho = b-bar, Eq. (rho_matrix_vec_def)
    np.testing.assert_allclose(rho_f, rho_r, atol=1e-13 * np.abs(rho_f).max())
    res = sisa(tr, np.zeros(tr.n_dof), 1e-14, 200, "dsa", dsa=ConsistentDSA(tr), keep_f=True)
    assert res["converged"]
    np.testing.assert_allclose(res["rho"], rho_f, atol=1e-12 * np.abs(rho_f).max())
    assert tr.residual_inf(res["rho"]) < 1e-13 * np.abs(rho_f).max()
    np.testing.assert_allclose(res["f"], f, atol=1e-12 * np.abs(f).max())


def test_mirror_directions_give_identical_fluxes():
    """X-Y geometry: directions differing only in the sign of v_z give identical f_j."""
    p = inputs.random_2d(6, 8, 4, 3, seed=9, inflow=(1.0, 0.0, 0.0, 0.5))
    tr = Transport(p)
    _, f = tr.sweep(np.random.default_rng(1).normal(size=tr.n_dof), store_f=True)
    nphi, nvz = p.n_phi, p.n_vz
    for j2 in range(nvz):
        np.testing.assert_array_equal(f[j2 * nphi:(j2 + 1) * nphi],
                                      f[(nvz - 1 - j2) * nphi:(nvz - j2) * nphi])


def test_si_slow_and_exact_correction_converges_in_two_sweeps():
    """SI stalls in a scattering-dominated slab (Sec. 1); with the kinetic correction equation
    solved exactly SI converges in at most two iterations (Sec. 2.3)."""
    p = inputs.slab(10, 8, 50.0, 49.9, G=1.0)
    tr = Transport(p)
    si = sisa(tr, np.zeros(tr.n_dof), 1e-10, 50, "none")
    assert not si["converged"] and si["delta"][-1] / si["delta"][-2] > 0.95
    Ld = tr.L_dense()
    ex = sisa(tr, np.zeros(tr.n_dof), 1e-10 * 0.01, 10, "exact", L_dense=Ld)
    assert ex["converged"] and ex["n_sweep"] <= 2
    np.testing.assert_allclose(ex["rho"], tr.solve_rho_direct(), rtol=1e-11)
