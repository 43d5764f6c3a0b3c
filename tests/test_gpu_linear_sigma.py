"""1D cross sections linear across cells (the cross-regime problem of Sec. 4.1.1) on the GPU,
against the oracle.

* One sweep (random linear materials on a non-uniform mesh, inflow on both sides) at the sweep
  tolerance 1e-12 relative; a right-end map equal to the left one gives the cellwise-constant
  path bit for bit.
* R = Sigma_s (rho* - rho_prev) with the 2x2 cell blocks, 1e-13 relative.
* SI-DSA (the consistent DSA with linear Sigma_a and Sigma_t) and DSA-preconditioned GMRES on the
  cross-regime problem converge to the oracle's direct solve of (I - L) rho = b-bar (1e-9); the
  SI-DSA sweep count is the oracle's (+-1).
* ROMIG: the device reduced operators (linear material shares) give the oracle's initial guess to
  1e-8 (the SVD accuracy of the two sides); a saved model loads back to the same guess, and a
  discretisation with another right-end map refuses it.
"""
import numpy as np
import pytest

from oracle.dsa import ConsistentDSA
from oracle.rom import OfflineROMs
from oracle.sisa import sisa
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


def _random_linear(seed, B=3):
    p = inputs.slab_random(41, 8, 5, seed=seed, B=B, inflow=(0.7, 1.3), linear=True)
    widths = np.random.default_rng(seed).uniform(0.3, 1.7, 41)
    edges = np.concatenate([[0.0], np.cumsum(widths)])
    edges *= 1.0 / edges[-1]
    edges[-1] = 1.0
    return inputs.replace(p, edges=edges)


def test_linear_sweep_matches_oracle():
    rte = _rte()
    p = _random_linear(7)
    batch = rte.Batch.from_problem(p)
    rho_in = np.random.default_rng(3).uniform(0, 1, (p.batch, p.n_dof))
    out = torch.empty((p.batch, p.n_dof), dtype=torch.float64, device="cuda")
    batch.sweep(torch.tensor(rho_in, device="cuda"), out)
    torch.cuda.synchronize()
    for b in range(p.batch):
        assert _rel(out.cpu().numpy()[b], Transport(p, b).sweep(rho_in[b])) < 1e-12


def test_equal_right_map_is_the_cellwise_path():
    rte = _rte()
    p = inputs.slab_random(41, 8, 5, seed=9, B=2, inflow=(0.7, 1.3))
    same = inputs.replace(p, mat_id_right=p.mat_id.copy())
    rho_in = torch.tensor(np.random.default_rng(4).uniform(0, 1, (2, p.n_dof)), device="cuda")
    outs = []
    for q in (p, same):
        batch = rte.Batch.from_problem(q)
        out = torch.empty_like(rho_in)
        batch.sweep(rho_in, out)
        outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_linear_correction_source_matches_oracle():
    rte = _rte()
    p = _random_linear(8, B=2)
    batch = rte.Batch.from_problem(p)
    rng = np.random.default_rng(5)
    rs, rp = rng.normal(size=(2, p.n_dof)), rng.normal(size=(2, p.n_dof))
    R = torch.empty((2, p.n_dof), dtype=torch.float64, device="cuda")
    batch.correction_source(torch.tensor(rs, device="cuda"), torch.tensor(rp, device="cuda"), R)
    torch.cuda.synchronize()
    for b in range(2):
        ref = Transport(p, b).Ss @ (rs[b] - rp[b])
        assert _rel(R.cpu().numpy()[b], ref) < 1e-13


def test_cross_regime_si_dsa_and_gmres_converge_to_direct_solve():
    rte = _rte()
    p = inputs.cross_regime(inputs.cross_regime_test(3), n=100)
    batch = rte.Batch.from_problem(p)
    rho = torch.zeros((3, p.n_dof), dtype=torch.float64, device="cuda")
    reps, _, st = batch.solve(rho, 1e-12, sa=rte.SA_DSA, max_iter=500)
    assert st == rte.RTE_OK
    rho2 = torch.zeros_like(rho)
    reps2, st2 = batch.pgmres(rho2, 1e-12, restart=25)
    assert st2 == rte.RTE_OK
    for b in range(3):
        tr = Transport(p, b)
        exact = tr.solve_rho_direct()
        assert _rel(rho.cpu().numpy()[b], exact) < 1e-9
        assert _rel(rho2.cpu().numpy()[b], exact) < 1e-9
        ref = sisa(tr, np.zeros(tr.n_dof), 1e-12, 500, "dsa", dsa=ConsistentDSA(tr))
        assert abs(reps[b]["n_sweep"] - ref["n_sweep"]) <= 1


def test_linear_romig_guess_save_and_load(tmp_path):
    rte = _rte()
    train = inputs.cross_regime(10.0 + np.arange(9) * 1.25, n=64)
    test = inputs.cross_regime(inputs.cross_regime_test(2), n=64)
    tb = rte.Batch.from_problem(train)
    rp, rc = rte.Rom.build(tb, eps_train=1e-12, window=2, rank_p=6, rank_c=8, max_iter=500,
                           dsa_rtol=1e-13)
    off = OfflineROMs(train, eps_train=1e-12, window=2, rank_p=6, rank_c=8)
    batch = rte.Batch(tb.disc, 2)
    batch.set_params(test)
    rho0 = torch.zeros((2, test.n_dof), dtype=torch.float64, device="cuda")
    rp.initial_guess(batch, rho0)
    got = rho0.cpu().numpy()
    for b in range(2):
        assert _rel(got[b], off.rom_p.initial_guess(Transport(test, b))) < 1e-8
    path = tmp_path / "rom_p.bin"
    rp.save(path)
    loaded = rte.Rom.load(tb.disc, path)
    rho1 = torch.zeros_like(rho0)
    loaded.initial_guess(batch, rho1)
    assert torch.equal(rho0, rho1)
    # the same mesh with cellwise-constant cross sections is another discretisation
    other = rte.Disc(inputs.replace(train, mat_id_right=None))
    with pytest.raises(rte.RTEError):
        rte.Rom.load(other, path)
