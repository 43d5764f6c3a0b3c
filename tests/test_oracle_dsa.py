"""Pins for the oracle's consistent DSA (App. B): the system equals the numerical 0th/1st
moments of the P1-ansatz-substituted DG operator; SI-DSA contracts fast where SI stalls; the
converged solution does not depend on the correction; a planted sign error is caught."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.dsa import ConsistentDSA
from oracle.sisa import sisa
from oracle.transport import Transport
from paper_2402_10488_gb300 import inputs


@pytest.mark.parametrize("dim", [1, 2])
def test_dsa_system_is_moments_of_p1_ansatz(dim):
    """For any drho, dJ: build delta f_j = drho + 3 v_j . dJ, apply the DG correction operator
    (D_j + Sigma_t) df_j - Sigma_s drho, and take sum_j omega_j (.) and sum_j omega_j v_j (.).
    Those are exactly the rows of the DSA system applied to (drho, dJ)."""
    if dim == 1:
        p = inputs.slab_random(11, 16, 3, seed=4)
    else:
        p = inputs.random_2d(5, 8, 2, 3, seed=4)
    tr = Transport(p)
    dsa = ConsistentDSA(tr)
    N = tr.n_dof
    rng = np.random.default_rng(1)
    fields = rng.normal(size=(dsa.n_fields, N))
    mom = np.zeros((dsa.n_fields, N))
    for j in range(tr.n_angles):
        vel = tr.v[j, :dim]
        df = fields[0] + 3.0 * sum(vel[d] * fields[1 + d] for d in range(dim))
        r = (tr.D(j) + tr.St) @ df - tr.Ss @ fields[0]
        mom[0] += tr.w[j] * r
        for d in range(dim):
            mom[1 + d] += tr.w[j] * vel[d] * r
    y = (dsa.M @ fields.reshape(-1)).reshape(dsa.n_fields, N)
    scale = np.abs(mom).max()
    np.testing.assert_allclose(y, mom, atol=1e-13 * scale)


def _rates(res):
    d = np.array(res["delta"])
    return d[1:] / d[:-1]


def test_si_dsa_contracts_fast_in_diffusive_slab():
    """Diffusive slab sigma_t = 100, sigma_a = 0.01 (c = 0.9999): SI stalls, SI-DSA contracts."""
    tr = Transport(inputs.slab_diffusive())
    dsa = ConsistentDSA(tr)
    r = sisa(tr, np.zeros(tr.n_dof), 1e-8, 100, "dsa", dsa=dsa, tol_mode="rel")
    assert r["converged"] and r["n_sweep"] <= 12
    assert np.all(_rates(r)[1:] < 0.25)
    si = sisa(tr, np.zeros(tr.n_dof), 1e-8, 40, "none", tol_mode="rel")
    assert not si["converged"] and np.all(_rates(si)[5:] > 0.99)


def test_si_dsa_contracts_fast_in_thick_2d_medium():
    p = inputs.random_2d(12, 8, 2, 1, seed=5)
    p.sigma_t[:], p.sigma_s[:] = 200.0, 199.8
    tr = Transport(p)
    r = sisa(tr, np.zeros(tr.n_dof), 1e-10, 100, "dsa", dsa=ConsistentDSA(tr), tol_mode="rel")
    assert r["converged"] and np.all(_rates(r) < 0.1)
    si = sisa(tr, np.zeros(tr.n_dof), 1e-10, 20, "none", tol_mode="rel")
    assert not si["converged"] and np.all(_rates(si)[4:] > 0.98)


def test_planted_sign_error_in_dsa_is_caught():
    """Flip the sign of the D_C coupling in a copy of the 1D system: the contraction pin fails."""
    tr = Transport(inputs.slab_diffusive(64, 16))
    dsa = ConsistentDSA(tr)
    N = tr.n_dof
    M = dsa.M.tolil()
    M[:N, N:] = -M[:N, N:]
    dsa.M, dsa._lu = sp.csc_matrix(M), None
    r = sisa(tr, np.zeros(tr.n_dof), 1e-8, 30, "dsa", dsa=dsa, tol_mode="rel")
    assert not (r["converged"] and r["n_sweep"] <= 12 and np.all(_rates(r)[1:] < 0.25))


def test_converged_solution_independent_of_correction():
    p = inputs.random_2d(6, 8, 2, 2, seed=8, inflow=(0.0, 1.0, 0.0, 0.0))
    p.sigma_t[:] = [[4.0, 9.0]]
    p.sigma_s[:] = [[3.5, 8.5]]
    tr = Transport(p)
    ref = tr.solve_rho_direct()
    for sa in ("none", "dsa"):
        r = sisa(tr, np.zeros(tr.n_dof), 1e-14, 3000, sa, dsa=ConsistentDSA(tr))
        assert r["converged"]
        np.testing.assert_allclose(r["rho"], ref, atol=1e-11 * np.abs(ref).max())


def test_2d_diagonal_blocks_couple_only_equal_parities():
    """Every cell's 12 x 12 diagonal block of the 2D DSA system (fields drho, dJx, dJy; moments
    k = kx + 2 ky) couples only unknowns of equal parities (kx xor [J_x], ky xor [J_y]) -- four
    3 x 3 blocks -- on a random material map and a non-square mesh, for interior, edge and corner
    cells, and so does its inverse.  The GPU smoother applies single-material blocks that way."""
    p = inputs.random_2d(6, 8, 2, 3, seed=9, ny=5)
    tr = Transport(p)
    M = ConsistentDSA(tr).M.tocsr()
    N = tr.n_dof

    def par(f, k):
        return ((k & 1) ^ (f == 1), (k >> 1) ^ (f == 2))

    unk = [(f, k) for f in range(3) for k in range(4)]
    same = np.array([[par(*a) == par(*b) for b in unk] for a in unk])
    assert same.sum() == 36
    for c in range(tr.n_dof // 4):
        idx = [f * N + 4 * c + k for f, k in unk]
        D = M[idx][:, idx].toarray()
        Di = np.linalg.inv(D)
        # zero up to the rounding of the oracle's quadrature-built operators
        assert np.abs(D[~same]).max() <= 1e-14 * np.abs(D).max(), c
        assert np.abs(Di[~same]).max() <= 1e-14 * np.abs(Di).max(), c
        assert np.count_nonzero(np.abs(D[same]) > 1e-8 * np.abs(D).max()) > 12   # not diagonal
