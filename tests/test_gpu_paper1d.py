"""The paper's 1D cross-regime problem (Sec. 4.1.1) at reduced size on the GPU against the oracle:
one material per cell (sigma_s = 0.1 + mu_s x taken at cell centres), 100 cells, S_16, 11
training slopes.  Checks: reduced dimensions under eps_POD = 1e-10 within one of numpy's SVD and
singular values to 1e-10 sigma_1 (the device Gram kernel runs many classes in chunks here);
ROMSA and ROMSAD solves converge to the oracle's direct solve within the tolerance their
absolute stop test at 1e-11 implies, with sweep counts within one of the oracle's.

Tolerance: an absolute change below 1e-11 with contraction c <= 0.9 leaves an error below
1e-10 absolute; relative to max rho (~1e-1 here) that is 1e-9."""
import numpy as np
import pytest

from oracle.dsa import ConsistentDSA
from oracle.rom import OfflineROMs
from oracle.sisa import romsad_eps, sisa
from oracle.transport import Transport
from paper_2402_10488_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rte():
    from paper_2402_10488_gb300 import build, rte
    build.build()
    return rte


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_cross_regime_rom_and_solves_match_oracle():
    rte = _rte()
    train = inputs.cross_regime(10.0 + np.arange(11), n=100)
    test = inputs.cross_regime(inputs.cross_regime_test(3), n=100)
    tb = rte.Batch.from_problem(train)
    rp, rc = rte.Rom.build(tb, eps_train=1e-11, window=3, rank_p=0, rank_c=0, eps_pod=1e-10,
                           max_iter=2000, dsa_rtol=1e-10)
    off = OfflineROMs(train, eps_train=1e-11, window=3, eps_pod=1e-10)
    assert rc.n_snap == off.dF.shape[1]
    assert abs(rp.r - off.pod_p.r) <= 1 and abs(rc.r - off.pod_c.r) <= 1
    np.testing.assert_allclose(rc.sv, off.pod_c.sv[:rc.n_snap], atol=1e-10 * off.pod_c.sv[0])
    batch = rte.Batch(tb.disc, 3)
    batch.set_params(test)
    eps_r = 0.1 * max(1e-11, 1e-10)  # eta max(eps_SISA, eps_POD), eps_POD the truncation tolerance
    for sa, name in ((rte.SA_ROMSA, "romsa"), (rte.SA_ROMSAD, "romsad")):
        rho = torch.zeros((3, test.n_dof), dtype=torch.float64, device="cuda")
        reps, _, st = batch.solve(rho, 1e-11, sa=sa, max_iter=2000, rom_c=rc, theta=3,
                                  eps_romsad=eps_r)
        assert st == rte.RTE_OK
        got = rho.cpu().numpy()
        for b in range(3):
            tr = Transport(test, b)
            exact = tr.solve_rho_direct()
            assert _rel(got[b], exact) < 1e-9
            ref = sisa(tr, np.zeros(tr.n_dof), 1e-11, 2000, name, dsa=ConsistentDSA(tr),
                       rom_c=off.rom_c, theta=3, eps_romsad=romsad_eps(1e-11, off.eps_pod))
            assert abs(reps[b]["n_sweep"] - ref["n_sweep"]) <= 1


def test_device_jacobi_svd_for_many_snapshots():
    """More than 256 correction snapshots (90 training slopes, window 3): the small factor R of
    the device QR is decomposed by the parallel one-sided Jacobi SVD on the GPU; singular values
    and the eps_POD truncation rank as numpy's SVD."""
    rte = _rte()
    train = inputs.cross_regime(10.0 + np.arange(90) / 9.0, n=100)
    tb = rte.Batch.from_problem(train)
    rp, rc = rte.Rom.build(tb, eps_train=1e-11, window=3, rank_p=0, rank_c=0, eps_pod=1e-10,
                           max_iter=2000, dsa_rtol=1e-10)
    off = OfflineROMs(train, eps_train=1e-11, window=3, eps_pod=1e-10)
    assert rc.n_snap == off.dF.shape[1] > 256
    np.testing.assert_allclose(rc.sv, off.pod_c.sv[:rc.n_snap], atol=1e-10 * off.pod_c.sv[0])
    assert abs(rc.r - off.pod_c.r) <= 1
