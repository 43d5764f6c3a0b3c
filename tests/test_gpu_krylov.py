"""GPU DSA-preconditioned GMRES (Sec. 2.3, App. A) against the oracle's, through the C ABI.

Tolerances: with the DSA inside M^{-1} solved to 1e-13 (FGMRES mode) both sides run GMRES on the
same preconditioned operator up to rounding, so they take the same number of steps (same sweep
count) and their results agree to the stopping tolerance times the conditioning; stopping at a
relative preconditioned residual of 1e-12 puts both within 1e-9 of the direct solve.  The GPU
orthogonalises by classical Gram-Schmidt twice, the oracle by modified Gram-Schmidt: equal in
exact arithmetic."""
import numpy as np
import pytest

from oracle.dsa import ConsistentDSA
from oracle.krylov import pgmres
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


@pytest.mark.parametrize("case", ["lattice", "random_inflow", "slab"])
def test_pgmres_matches_oracle(case):
    rte = _rte()
    if case == "lattice":
        p = inputs.lattice_test(12, 16, 2, n_vz=2)
    elif case == "random_inflow":
        p = inputs.random_2d(10, 8, 2, 3, seed=21, B=2, inflow=(0.4, 0.0, 1.0, 0.2), ny=14)
    else:
        p = inputs.slab_random(40, 8, 3, seed=5, B=2, inflow=(1.0, 0.5))
    batch = rte.Batch.from_problem(p)
    rho = torch.zeros((p.batch, p.n_dof), dtype=torch.float64, device="cuda")
    reps, st = batch.pgmres(rho, 1e-12, restart=25, dsa_rtol=1e-13, dsa_max_it=3000)
    assert st == rte.RTE_OK
    got = rho.cpu().numpy()
    for b in range(p.batch):
        tr = Transport(p, b)
        ref = pgmres(tr, np.zeros(tr.n_dof), 1e-12, m=25, precond=ConsistentDSA(tr).correction)
        assert reps[b]["converged"] and ref["converged"]
        assert abs(reps[b]["n_sweep"] - ref["n_sweep"]) <= 1
        exact = tr.solve_rho_direct()
        assert _rel(got[b], exact) < 1e-9
        assert _rel(got[b], ref["rho"]) < 1e-9


def test_unpreconditioned_and_restarted_from_a_start():
    rte = _rte()
    p = inputs.lattice_test(8, 8, 2, n_vz=2)
    batch = rte.Batch.from_problem(p)
    exact = np.array([Transport(p, b).solve_rho_direct() for b in range(2)])
    # no preconditioner: same step count as the oracle
    rho = torch.zeros((2, p.n_dof), dtype=torch.float64, device="cuda")
    reps, st = batch.pgmres(rho, 1e-11, restart=60, max_iter=2000, precond=False)
    assert st == rte.RTE_OK
    for b in range(2):
        tr = Transport(p, b)
        ref = pgmres(tr, np.zeros(tr.n_dof), 1e-11, m=60, max_outer=40)
        assert abs(reps[b]["n_sweep"] - ref["n_sweep"]) <= 1
        assert _rel(rho.cpu().numpy()[b], exact[b]) < 1e-8
    # a nonzero start with short cycles: restarts, the start's residual costs one sweep each
    x0 = torch.tensor(0.5 * exact, device="cuda")
    reps, st = batch.pgmres(x0, 1e-11, restart=3, dsa_rtol=1e-13, dsa_max_it=3000, zero_start=False)
    assert st == rte.RTE_OK
    for b in range(2):
        tr = Transport(p, b)
        ref = pgmres(tr, 0.5 * exact[b], 1e-11, m=3, precond=ConsistentDSA(tr).correction)
        assert abs(reps[b]["n_sweep"] - ref["n_sweep"]) <= 1
        assert _rel(x0.cpu().numpy()[b], exact[b]) < 1e-8


def test_pgmres_with_vcycle_preconditioner_converges():
    """The bench configuration: M^{-1} with one FP32 multigrid V-cycle (a fixed linear operator
    up to FP32 rounding)."""
    rte = _rte()
    p = inputs.lattice_test(32, 16, 3)
    batch = rte.Batch.from_problem(p)
    rho = torch.zeros((3, p.n_dof), dtype=torch.float64, device="cuda")
    reps, st = batch.pgmres(rho, 1e-10, restart=25, dsa_rtol=0.0, dsa_max_it=1)
    assert st == rte.RTE_OK and all(r["converged"] for r in reps)
    ref = torch.zeros_like(rho)
    batch.solve(ref, 1e-13, sa=rte.SA_DSA, rel=True, max_iter=400, dsa_rtol=1e-3)
    assert _rel(rho.cpu().numpy(), ref.cpu().numpy()) < 1e-8
