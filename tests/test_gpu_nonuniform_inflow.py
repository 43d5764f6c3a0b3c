"""Non-uniform 1D meshes and ROMIG with nonzero inflow on the GPU, against the oracle.

* 1D sweeps on a non-uniform mesh (the two-material mesh of Sec. 4.1.2 and a random one) at the
  sweep tolerance 1e-12 relative; SI-DSA on the two-material problem (inflow 5 at x = 0) converges
  to the oracle's direct solve, with the sweep count of the oracle's SI-DSA.
* ROMIG with isotropic inflow: U^T b_mu includes the inflow's projection, in 1D (two-material)
  and 2D (lattice with inflow on all sides); the device guess agrees with the oracle's (its
  projection sums U_j^T (G + g^bc_j) over all directions), up to the SVD accuracy of the two sides
  (1e-8 relative)."""
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


def _random_nonuniform(seed, B=2):
    rng = np.random.default_rng(seed)
    widths = rng.uniform(0.2, 1.8, 37)
    edges = np.concatenate([[0.0], np.cumsum(widths)])
    edges *= 3.0 / edges[-1]
    p = inputs.slab_random(37, 8, 3, seed=seed, B=B, inflow=(0.7, 1.3))
    return inputs.replace(p, domain=(0.0, 3.0), edges=edges)


@pytest.mark.parametrize("which", ["two_material", "random"])
def test_nonuniform_1d_sweep_matches_oracle(which):
    rte = _rte()
    p = (inputs.two_material(inputs.two_material_test(2)) if which == "two_material"
         else _random_nonuniform(5))
    batch = rte.Batch.from_problem(p)
    rho_in = np.random.default_rng(3).uniform(0, 1, (p.batch, p.n_dof))
    out = torch.empty((p.batch, p.n_dof), dtype=torch.float64, device="cuda")
    batch.sweep(torch.tensor(rho_in, device="cuda"), out)
    torch.cuda.synchronize()
    for b in range(p.batch):
        ref = Transport(p, b).sweep(rho_in[b])
        assert _rel(out.cpu().numpy()[b], ref) < 1e-12


def test_two_material_si_dsa_converges_to_direct_solve():
    rte = _rte()
    p = inputs.two_material(inputs.two_material_test(3))
    batch = rte.Batch.from_problem(p)
    rho = torch.zeros((3, p.n_dof), dtype=torch.float64, device="cuda")
    reps, _, st = batch.solve(rho, 1e-12, sa=rte.SA_DSA, max_iter=500)
    assert st == rte.RTE_OK
    for b in range(3):
        tr = Transport(p, b)
        assert _rel(rho.cpu().numpy()[b], tr.solve_rho_direct()) < 1e-9
        ref = sisa(tr, np.zeros(tr.n_dof), 1e-12, 500, "dsa", dsa=ConsistentDSA(tr))
        assert abs(reps[b]["n_sweep"] - ref["n_sweep"]) <= 1


def _lattice_with_inflow(problem, g=(0.5, 1.0, 0.2, 0.0)):
    return inputs.replace(problem, inflow=np.tile(np.array(g), (problem.batch, 1)))


@pytest.mark.parametrize("dim", [1, 2])
def test_romig_with_inflow_matches_oracle(dim):
    rte = _rte()
    if dim == 1:
        mus = inputs.two_material_train()[::23]           # 20 of the 451 training pairs
        train = inputs.two_material(mus)
        test = inputs.two_material(inputs.two_material_test(2))
    else:
        train = _lattice_with_inflow(inputs.lattice_train(8, 8, n_train=8, n_vz=2))
        test = _lattice_with_inflow(inputs.lattice_test(8, 8, 2, n_vz=2))
    tb = rte.Batch.from_problem(train)
    rp, rc = rte.Rom.build(tb, eps_train=1e-12, window=2, rank_p=6, rank_c=6, max_iter=500,
                           dsa_rtol=1e-13)
    off = OfflineROMs(train, eps_train=1e-12, window=2, rank_p=6, rank_c=6)
    batch = rte.Batch(tb.disc, 2)
    batch.set_params(test)
    rho0 = torch.zeros((2, test.n_dof), dtype=torch.float64, device="cuda")
    rp.initial_guess(batch, rho0)
    got = rho0.cpu().numpy()
    for b in range(2):
        ref = off.rom_p.initial_guess(Transport(test, b))
        assert _rel(got[b], ref) < 1e-8
