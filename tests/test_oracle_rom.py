"""Pins for the oracle's POD ROMs (Sec. 3): the truncation rule, orthonormality, the affine
reduced operators against a direct Galerkin projection of the dense A_mu, exact reproduction
of training parameters (ROMIG) and of a basis that contains the test's own correction (ROMSA),
and Alg. 2's switch."""
import numpy as np
import pytest

from oracle.dsa import ConsistentDSA
from oracle.rom import POD, OfflineROMs, ReducedModel, pod_rank
from oracle.sisa import romsad_eps, sisa
from oracle.transport import Transport
from paper_2402_10488_gb300 import inputs


def test_pod_rank_rule():
    sv = np.array([10.0, 5.0, 3.0, 1.0, 0.5, 0.5])      # trace 20
    assert pod_rank(sv, 0.5) == 1            # 10/20 >= 0.5
    assert pod_rank(sv, 0.25) == 2           # 15/20 = 0.75 >= 0.75
    assert pod_rank(sv, 0.2) == 3            # 0.9 >= 0.8, 0.75 < 0.8
    assert pod_rank(sv, 1e-12) == 6
    assert romsad_eps(1e-12, 1e-9) == pytest.approx(1e-10)


@pytest.fixture(scope="module")
def small_roms():
    train = inputs.lattice_train(6, 8, n_train=6, n_vz=2)
    return OfflineROMs(train, eps_train=1e-13, window=3, rank_p=4, rank_c=8)


def test_bases_orthonormal_and_ranks(small_roms):
    for pod in (small_roms.pod_p, small_roms.pod_c):
        np.testing.assert_allclose(pod.U.T @ pod.U, np.eye(pod.r), atol=1e-12)
    # the basis spans the leading left singular space of the snapshots
    F = small_roms.F
    P = small_roms.pod_p.U @ small_roms.pod_p.U.T
    sv = small_roms.pod_p.sv
    assert np.linalg.norm(F - P @ F, 2) <= sv[small_roms.pod_p.r] * (1 + 1e-8)


def test_affine_reduced_operator_equals_galerkin_projection(small_roms):
    test = inputs.lattice_test(6, 8, 2, n_vz=2)
    for b in range(2):
        tr = Transport(test, b)
        A, bvec = tr.coupled_system()
        for rom in (small_roms.rom_p, small_roms.rom_c):
            U = rom.U
            np.testing.assert_allclose(rom.operator(test.sigma_t[b], test.sigma_s[b]), U.T @ A @ U,
                                       atol=1e-10 * np.abs(U.T @ A @ U).max())
            np.testing.assert_allclose(rom.project_rhs(tr), U.T @ bvec, atol=1e-12)
            Uj = U.reshape(tr.n_angles, tr.n_dof, -1)
            np.testing.assert_allclose(rom.U_rho, np.einsum("j,jnr->nr", tr.w, Uj), atol=1e-15)


def test_romig_reproduces_training_parameter_in_one_sweep():
    train = inputs.lattice_train(6, 8, n_train=3, n_vz=2)
    off = OfflineROMs(train, eps_train=1e-14, window=1, rank_p=3, rank_c=3)
    tr = Transport(train, 1)
    rho0 = off.rom_p.initial_guess(tr)
    res = sisa(tr, rho0, 1e-11, 20, "dsa", dsa=ConsistentDSA(tr))
    assert res["n_sweep"] == 1


def test_romsa_with_own_correction_in_basis_converges_in_two_sweeps():
    """If dU spans the test trajectory's delta f^(1) = f - f^(1), the Galerkin ROM correction is
    the exact kinetic correction, so SI stops at the second sweep (Sec. 2.3, Sec. 3.2)."""
    test = inputs.lattice_test(6, 8, 1, n_vz=2)
    tr = Transport(test, 0)
    rho_exact, f_exact = tr.solve_direct()
    _, f1 = tr.sweep(np.zeros(tr.n_dof), store_f=True)
    dF = (f_exact - f1).reshape(-1, 1)
    rom = ReducedModel(POD(dF, rank=1).U, tr)
    res = sisa(tr, np.zeros(tr.n_dof), 1e-11, 20, "romsa", rom_c=rom)
    assert res["converged"] and res["n_sweep"] == 2
    np.testing.assert_allclose(res["rho"], rho_exact, atol=1e-11 * np.abs(rho_exact).max())


def test_romsad_switch_follows_alg2(small_roms):
    test = inputs.lattice_test(6, 8, 1, n_vz=2)
    tr = Transport(test, 0)
    eps_r = 1e-4
    res = sisa(tr, np.zeros(tr.n_dof), 1e-12, 200, "romsad", dsa=ConsistentDSA(tr),
               rom_c=small_roms.rom_c, theta=3, eps_romsad=eps_r)
    for l, (delta, choice) in enumerate(zip(res["delta"], res["sa"]), start=1):
        assert choice == ("romsa" if (l <= 3 and delta >= eps_r) else "dsa")
    # same converged answer as SI-DSA
    ref = sisa(tr, np.zeros(tr.n_dof), 1e-12, 200, "dsa", dsa=ConsistentDSA(tr))
    np.testing.assert_allclose(res["rho"], ref["rho"], atol=1e-10 * np.abs(ref["rho"]).max())


def test_correction_rank_not_below_parametric_rank():
    """r_p <= r_c for a common eps_POD (Sec. 4.2.1 observation)."""
    train = inputs.lattice_train(6, 8, n_train=6, n_vz=2)
    off = OfflineROMs(train, eps_train=1e-13, window=3, eps_pod=1e-6)
    assert off.pod_p.r <= off.pod_c.r


def test_romig_started_correction_snapshots_make_romig_romsa_exact():
    """Remark after Alg. 2: for ROMIG followed by ROMSA the correction basis must come from
    ROMIG-started training runs.  With window 1 and every snapshot kept, a training instance's
    ROMIG-started trajectory has its own delta f^(1) in the basis, so ROMIG + ROMSA is exact after
    the first correction and stops at the second sweep; the zero-started basis lacks that
    correction and needs more sweeps."""
    train = inputs.lattice_train(6, 8, n_train=3, n_vz=2)
    kw = dict(eps_train=1e-14, window=1, rank_p=1, rank_c=3)
    romig = OfflineROMs(train, correction_start="romig", **kw)
    zero = OfflineROMs(train, correction_start="zero", **kw)
    assert romig.dF.shape[1] == 3 and zero.dF.shape[1] == 3
    tr = Transport(train, 1)
    rho_exact = tr.solve_rho_direct()
    rho0 = romig.rom_p.initial_guess(tr)
    res = sisa(tr, rho0, 1e-11, 20, "romsa", rom_c=romig.rom_c)
    assert res["converged"] and res["n_sweep"] == 2
    np.testing.assert_allclose(res["rho"], rho_exact, atol=1e-10 * np.abs(rho_exact).max())
    res0 = sisa(tr, rho0, 1e-11, 20, "romsa", rom_c=zero.rom_c)
    assert res0["n_sweep"] > 2
