"""GPU parity of the float-float sweep (rte_sweep_ff), the precision variant's outer sweep, against
the oracle's FP64 sweep (Eq. (transport_sweep)) and the library's FP64 sweep, through the C ABI,
and of a precision-variant solve whose FP64-grade sweeps run this way.

Tolerance, derived: a float-float value has a unit roundoff of 2^-48 (a 48-bit significand), 32
times FP64's 2^-53, and each float-float FMA rounds a few times that relative to |a b| + |c| (the
product lo * lo is dropped and the error terms are added in FP32).  The cell solves are the FP64
sweep's chains of FMAs in the same order, with the sources formed in FP64 and the partial sums
reduced in FP64, so the error is the FP64 sweep's with the roundoff 32 times larger: the FP64
parity bound of 1e-12 ||rho*||_inf becomes 3e-11 ||rho*||_inf.  Each decomposition is
deterministic (bit-identical on a second call)."""
import numpy as np
import pytest

from oracle.dsa import ConsistentDSA
from oracle.sisa import sisa
from oracle.transport import Transport
from paper_2402_10488_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOLFF = 3e-11

CASES = [
    (5, 3, 4, 2),       # tiny, nx < 32
    (12, 20, 8, 2),     # nx < 32, several row blocks
    (37, 19, 8, 4),     # nx > 32, ny not a multiple of the block height
    (33, 70, 4, 2),     # several row blocks with a ragged tail
    (64, 64, 16, 4),    # 32 distinct directions
    (96, 80, 4, 2),     # an odd number of row blocks
]


def _rte():
    from paper_2402_10488_gb300 import build, rte
    build.build()
    return rte


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("nx,ny,nphi,nvz", CASES)
def test_ff_sweep_matches_oracle_every_decomposition(nx, ny, nphi, nvz):
    rte = _rte()
    p = inputs.random_2d(nx, nphi, nvz, 3, seed=nx + ny, B=3, inflow=(0.4, 1.1, 0.0, 0.6), ny=ny)
    rho = np.random.default_rng(nx).uniform(0.0, 1.0, (3, p.n_dof))
    ref = np.array([Transport(p, b).sweep(rho[b]) for b in range(3)])
    batch = rte.Batch.from_problem(p)
    rin = torch.tensor(rho, device="cuda")
    for dpw in (1, 2, 4, 8):   # 8 runs as 4 (the partial-sum buffer holds the finer groups)
        batch.tune(dpw)
        out = torch.full_like(rin, float("nan"))
        batch.sweep_ff(rin, out)
        again = torch.full_like(rin, float("nan"))
        batch.sweep_ff(rin, again)
        f64 = torch.empty_like(rin)
        batch.sweep(rin, f64)
        torch.cuda.synchronize()
        assert torch.equal(out, again), dpw
        got = out.cpu().numpy()
        assert _rel(got, ref) < TOLFF, (dpw, _rel(got, ref))
        assert _rel(got, f64.cpu().numpy()) < TOLFF, (dpw, _rel(got, f64.cpu().numpy()))


def test_ff_sweep_masked_instances_untouched():
    rte = _rte()
    p = inputs.lattice_test(48, 32, 4)
    rho = np.random.default_rng(5).uniform(0.0, 1.0, (4, p.n_dof))
    ref = np.array([Transport(p, b).sweep(rho[b]) for b in range(4)])
    batch = rte.Batch.from_problem(p)
    rin = torch.tensor(rho, device="cuda")
    out = torch.full_like(rin, -3.0)
    act = torch.tensor([1, 0, 1, 0], dtype=torch.uint8, device="cuda")
    batch.sweep_ff(rin, out, active=act)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(got[1] == -3.0) and np.all(got[3] == -3.0)
    for b in (0, 2):
        assert _rel(got[b], ref[b]) < TOLFF, _rel(got[b], ref[b])


def test_ff_sweep_without_room_for_finer_groups_runs_the_fp64_sweep():
    """A batch whose partial-sum buffer holds only the groups of 8 directions per warp (many
    instances of a small mesh with 8 directions per quadrant: the default decomposition is 8 per
    warp) cannot run the float-float sweep, which takes at most 4: the FP64 sweep runs instead,
    bit for bit.  Which one ran shows in the batch's timing counters."""
    rte = _rte()
    p = inputs.random_2d(8, 16, 4, 3, seed=3, B=160, inflow=(0.2, 0.0, 0.9, 0.0), ny=8)
    rho = np.random.default_rng(2).uniform(0.0, 1.0, (p.batch, p.n_dof))
    batch = rte.Batch.from_problem(p)
    rin = torch.tensor(rho, device="cuda")
    out = torch.empty_like(rin)
    batch.timing(1)
    batch.sweep_ff(rin, out)
    t = batch.timing(0)
    f64 = torch.empty_like(rin)
    batch.sweep(rin, f64)
    torch.cuda.synchronize()
    assert (t["sweep_launches"], t["sweepff_launches"]) in ((1, 0), (0, 1)), t
    if t["sweep_launches"] == 1:
        assert torch.equal(out, f64)
    ref = np.array([Transport(p, b).sweep(rho[b]) for b in range(0, p.batch, 40)])
    assert _rel(out.cpu().numpy()[::40], ref) < TOLFF


@pytest.mark.parametrize("switch", [1e-4, 0.0])
def test_refinement_with_ff_outer_sweeps_reaches_the_fp64_solution(switch):
    """The precision variant with its FP64-grade sweeps in float-float (rte_solve_opts.outer_ff):
    no FP64 sweep runs, and the result is the FP64 transport solution (the oracle's SI-DSA to 1e-14)
    to the stop tolerance, as with FP64 outer sweeps.  The stop test, a relative change of 1e-11,
    sits a hundred times above the float-float sweep's rounding."""
    rte = _rte()
    p = inputs.lattice_test(32, 16, 3, n_vz=2)
    common = dict(sa=rte.SA_DSA, rel=True, max_iter=300, dsa_rtol=0.0, dsa_max_it=2,
                  fp32_switch=switch, refine_kappa=0.05, refine_inner=8)
    out = {}
    for ff in (False, True):
        batch = rte.Batch.from_problem(p)
        rho = torch.zeros((3, p.n_dof), dtype=torch.float64, device="cuda")
        batch.timing(1)
        rep, _, st = batch.solve(rho, 1e-11, outer_ff=ff, **common)
        t = batch.timing(0)
        assert st == 0 and all(r["converged"] for r in rep)
        out[ff] = (rho.cpu().numpy(), rep, t)
    _, rep, t = out[True]
    assert t["sweep_launches"] == 0 and t["sweepff_launches"] >= 1, t
    assert out[False][2]["sweepff_launches"] == 0
    for b in range(3):
        tr = Transport(p, b)
        ref = sisa(tr, np.zeros(tr.n_dof), 1e-14, 400, "dsa", dsa=ConsistentDSA(tr), tol_mode="rel")
        for ff in (False, True):
            assert _rel(out[ff][0][b], ref["rho"]) < 1e-9, (ff, _rel(out[ff][0][b], ref["rho"]))
        assert rep[b]["n_sweep"] - rep[b]["n_sweep32"] >= 1
