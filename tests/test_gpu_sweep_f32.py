"""GPU parity of the FP32 sweep of the precision variant (rte_sweep_f32) against the oracle's FP64
sweep (Eq. (transport_sweep)), through the C ABI, for every work decomposition.

Tolerance, derived: the sources and sweep tables are rounded to FP32 (relative u = 2^-24 ~ 6e-8
each) and each cell solve adds ~10 roundings of a chain of FMAs, so one cell's solution carries
~16u relative error; the inflow from upwind cells carries their error on, adding at most that much
per cell crossed, i.e. <= (n_x + n_y) * 16u along a characteristic (2e-4 for the largest mesh
here); the partial sums over directions add ~n_dirs u.  Rounding errors of independent cells
largely cancel, so the test bounds the error by 3e-5 ||rho*||_inf, well inside the worst case.  The
decompositions add the same FP32 terms in different groupings, so they agree to the same bound;
each is deterministic (bit-identical on a second call)."""
import numpy as np
import pytest

from oracle.transport import Transport
from paper_2402_10488_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 3e-5

CASES = [
    (5, 3, 4, 2),       # tiny, nx < 32
    (12, 20, 8, 2),     # nx < 32, several row blocks
    (37, 19, 8, 4),     # nx > 32, ny not a multiple of the block height
    (33, 70, 4, 2),     # several row blocks with a ragged tail
    (64, 64, 16, 4),    # 32 distinct directions
    (70, 100, 8, 2),    # two row blocks per warp, a ragged last row block
    (96, 80, 4, 2),     # two row blocks per warp, an odd number of row blocks
]


def _rte():
    from paper_2402_10488_gb300 import build, rte
    build.build()
    return rte


@pytest.mark.parametrize("nx,ny,nphi,nvz", CASES)
def test_fp32_sweep_matches_oracle_every_decomposition(nx, ny, nphi, nvz):
    rte = _rte()
    p = inputs.random_2d(nx, nphi, nvz, 3, seed=nx + ny, B=3, inflow=(0.4, 1.1, 0.0, 0.6), ny=ny)
    rho = np.random.default_rng(nx).uniform(0.0, 1.0, (3, p.n_dof))
    ref = np.array([Transport(p, b).sweep(rho[b]) for b in range(3)])
    scale = np.abs(ref).max()
    batch = rte.Batch.from_problem(p)
    rin = torch.tensor(rho, device="cuda")
    outs = {}
    for dpw in (1, 2, 4, 8):
        batch.tune(dpw)
        out = torch.full_like(rin, float("nan"))
        batch.sweep_f32(rin, out)
        again = torch.full_like(rin, float("nan"))
        batch.sweep_f32(rin, again)
        torch.cuda.synchronize()
        assert torch.equal(out, again), dpw
        got = out.cpu().numpy()
        err = np.abs(got - ref).max() / scale
        assert err < TOL32, (dpw, err)
        outs[dpw] = got
    base = outs[1]
    for k, v in outs.items():
        assert np.abs(v - base).max() / scale < TOL32, k


def test_fp32_sweep_masked_instances_untouched_and_autotuned():
    """The active mask leaves skipped instances' outputs untouched; after the autotuner has chosen a
    decomposition per running count, the FP32 sweep still matches the oracle."""
    rte = _rte()
    p = inputs.lattice_test(48, 32, 4)
    rho = np.random.default_rng(5).uniform(0.0, 1.0, (4, p.n_dof))
    ref = np.array([Transport(p, b).sweep(rho[b]) for b in range(4)])
    batch = rte.Batch.from_problem(p)
    rin = torch.tensor(rho, device="cuda")
    out = torch.full_like(rin, -3.0)
    act = torch.tensor([1, 0, 1, 0], dtype=torch.uint8, device="cuda")
    batch.sweep_f32(rin, out, active=act)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(got[1] == -3.0) and np.all(got[3] == -3.0)
    for b in (0, 2):
        assert np.abs(got[b] - ref[b]).max() / np.abs(ref[b]).max() < TOL32
    batch.autotune()
    out2 = torch.empty_like(rin)
    batch.sweep_f32(rin, out2)
    torch.cuda.synchronize()
    got2 = out2.cpu().numpy()
    for b in range(4):
        assert np.abs(got2[b] - ref[b]).max() / np.abs(ref[b]).max() < TOL32
