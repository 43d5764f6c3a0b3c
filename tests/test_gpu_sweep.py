"""GPU parity of the transport sweep fused with the scalar-flux reduction (Alg. 1,
Eq. (transport_sweep)) against the CPU oracle, through the C ABI.

Tolerance: the sweep is a sequence of well-conditioned 4x4 (2x2) cell solves in FP64; both sides
round differently (table inverse vs sparse LU), so agreement is to a few ulps of ||rho||_inf
amplified along the sweep: 1e-12 relative to ||rho||_inf."""
import numpy as np
import pytest

from oracle.transport import Transport
from paper_2402_10488_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-12


def _rte():
    from paper_2402_10488_gb300 import build, rte
    build.build()
    return rte


def _gpu_sweep(rte, problem, rho_in, with_source=True, psi=False, active=None):
    batch = rte.Batch.from_problem(problem)
    rin = torch.tensor(rho_in, dtype=torch.float64, device="cuda").contiguous()
    rout = torch.full_like(rin, 7.0)
    psi_t = None
    if psi:
        psi_t = torch.zeros((problem.batch, batch.disc.n_dirs, batch.disc.n_dof), dtype=torch.float64,
                            device="cuda")
    act = None if active is None else torch.tensor(active, dtype=torch.uint8, device="cuda")
    batch.sweep(rin, rout, psi_t, with_source=with_source, active=act)
    torch.cuda.synchronize()
    return batch, rout.cpu().numpy(), None if psi_t is None else psi_t.cpu().numpy()


def _oracle_sweep(problem, rho_in, with_source=True):
    out, fs = [], []
    for b in range(problem.batch):
        tr = Transport(problem, b)
        r, f = tr.sweep(rho_in[b], with_source=with_source, store_f=True)
        out.append(r)
        fs.append((tr, f))
    return np.array(out), fs


def _check(gpu, ref):
    scale = np.abs(ref).max()
    err = np.abs(gpu - ref).max() / scale
    assert err < RTOL, err


CASES_2D = [
    (5, 3, 4, 2),       # tiny, nx < 32
    (12, 20, 8, 2),     # nx < 32 < ... ragged blocks
    (37, 19, 8, 4),     # nx > 32, ny not a multiple of the block height
    (33, 70, 4, 2),     # several row blocks with a ragged tail
    (64, 64, 16, 4),    # multiple full blocks, 32 distinct directions
]


@pytest.mark.parametrize("nx,ny,nphi,nvz", CASES_2D)
def test_sweep_2d_parity(nx, ny, nphi, nvz):
    rte = _rte()
    p = inputs.random_2d(nx, nphi, nvz, 3, seed=nx * 100 + ny, B=2, inflow=(0.3, 1.2, 0.7, 0.0), ny=ny)
    rng = np.random.default_rng(5)
    rho_in = rng.normal(size=(2, p.n_dof))
    _, gpu, _ = _gpu_sweep(rte, p, rho_in)
    ref, _ = _oracle_sweep(p, rho_in)
    _check(gpu, ref)
    # the operator L (no source, no inflow)
    _, gpu0, _ = _gpu_sweep(rte, p, rho_in, with_source=False)
    ref0, _ = _oracle_sweep(p, rho_in, with_source=False)
    _check(gpu0, ref0)


def test_sweep_2d_angular_flux_output_matches_oracle():
    rte = _rte()
    p = inputs.random_2d(20, 8, 4, 2, seed=3, B=1, inflow=(1.0, 0.0, 0.5, 2.0), ny=11)
    rho_in = np.random.default_rng(1).normal(size=(1, p.n_dof))
    batch, gpu, psi = _gpu_sweep(rte, p, rho_in, psi=True)
    ref, fs = _oracle_sweep(p, rho_in)
    tr, f = fs[0]
    dirs = batch.directions()
    assert dirs.shape[0] == p.n_angles // 2
    np.testing.assert_allclose(dirs[:, 2].sum(), 1.0, atol=1e-15)
    for k, (vx, vy, w, mult) in enumerate(dirs):
        j = int(np.argmin(np.abs(tr.v[:, 0] - vx) + np.abs(tr.v[:, 1] - vy)))
        assert abs(tr.v[j, 0] - vx) < 1e-15 and abs(tr.v[j, 1] - vy) < 1e-15
        assert mult == 2
        scale = np.abs(f[j]).max()
        assert np.abs(psi[0, k] - f[j]).max() < RTOL * scale * 10


def test_sweep_1d_parity_and_batch_and_active_mask():
    rte = _rte()
    p = inputs.slab_random(45, 16, 4, seed=8, B=3, inflow=(1.5, 0.25))
    rho_in = np.random.default_rng(2).normal(size=(3, p.n_dof))
    _, gpu, _ = _gpu_sweep(rte, p, rho_in, active=[1, 0, 1])
    ref, _ = _oracle_sweep(p, rho_in)
    _check(gpu[[0, 2]], ref[[0, 2]])
    assert np.all(gpu[1] == 7.0)          # inactive instance untouched


def test_sweep_config1_slab_and_change_norm():
    rte = _rte()
    p = inputs.slab_diffusive()
    rho_in = np.random.default_rng(3).uniform(0, 1, size=(1, p.n_dof))
    batch, gpu, _ = _gpu_sweep(rte, p, rho_in)
    ref, _ = _oracle_sweep(p, rho_in)
    _check(gpu, ref)
    rs = torch.tensor(gpu, device="cuda")
    rp = torch.tensor(rho_in, device="cuda")
    norms = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    batch.change_norm(rs, rp, norms)
    n = norms.cpu().numpy()[0]
    assert n[0] == np.abs(gpu - rho_in).max() and n[1] == np.abs(gpu).max()
    R = torch.zeros_like(rs)
    batch.correction_source(rs, rp, R)
    tr = Transport(p)
    np.testing.assert_allclose(R.cpu().numpy()[0], tr.Ss @ (gpu[0] - rho_in[0]), rtol=1e-15, atol=0)


@pytest.mark.slow
def test_sweep_lattice_128_full_size():
    """Full-size lattice workload (128 x 128, CL(16,4)): one sweep per instance vs the oracle."""
    rte = _rte()
    p = inputs.lattice_test(128, 64, 2)
    rho_in = np.random.default_rng(4).uniform(0, 1, size=(2, p.n_dof))
    _, gpu, _ = _gpu_sweep(rte, p, rho_in)
    ref, _ = _oracle_sweep(p.subset([0]), rho_in[:1])
    _check(gpu[:1], ref)


@pytest.mark.parametrize("dpw", [1, 2, 4, 8])
def test_sweep_work_decomposition_does_not_change_results(dpw):
    rte = _rte()
    p = inputs.random_2d(40, 16, 4, 3, seed=77, B=2, inflow=(0.2, 0.0, 1.0, 0.5), ny=33)
    batch = rte.Batch(rte.Disc(p), 2)
    batch.tune(dpw)
    batch.set_params(p)
    rho_in = np.random.default_rng(6).normal(size=(2, p.n_dof))
    rin = torch.tensor(rho_in, device="cuda")
    rout = torch.empty_like(rin)
    batch.sweep(rin, rout)
    torch.cuda.synchronize()
    ref, _ = _oracle_sweep(p, rho_in)
    _check(rout.cpu().numpy(), ref)


def test_autotuned_decomposition_keeps_results():
    """The empirical autotuner only changes which directions share a warp: results stay within
    the sweep tolerance of the oracle, and every table entry is an allowed value."""
    rte = _rte()
    p = inputs.random_2d(48, 16, 4, 3, seed=78, B=6, inflow=(0.2, 0.0, 1.0, 0.5), ny=40)
    batch = rte.Batch.from_problem(p)
    table = batch.autotune()
    assert [n for n, _ in table] == sorted(n for n, _ in table) and table[-1][0] == 6
    assert all(d in (1, 2, 4, 8) for _, d in table)
    rho_in = np.random.default_rng(9).normal(size=(6, p.n_dof))
    rin = torch.tensor(rho_in, device="cuda")
    rout = torch.empty_like(rin)
    batch.sweep(rin, rout)
    torch.cuda.synchronize()
    ref, _ = _oracle_sweep(p, rho_in)
    _check(rout.cpu().numpy(), ref)
