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
    """The empirical autotuner only changes which directions share a warp and how many warps walk
    a direction group's row blocks: results stay within the sweep tolerance of the oracle, and
    every table entry is an allowed value."""
    rte = _rte()
    p = inputs.random_2d(48, 16, 4, 3, seed=78, B=6, inflow=(0.2, 0.0, 1.0, 0.5), ny=40)
    batch = rte.Batch.from_problem(p)
    table = batch.autotune()
    assert [n for n, _ in table] == sorted(n for n, _ in table) and table[-1][0] == 6
    assert all(d in (1, 2, 4, 8) for _, d in table)
    # the FP64 choice with its warps per direction group (40 rows: two row blocks at most)
    wide = batch.tuned()
    assert [(n, d) for n, d, _ in wide] == table
    assert all(w in (1, 2) for _, _, w in wide)
    rho_in = np.random.default_rng(9).normal(size=(6, p.n_dof))
    rin = torch.tensor(rho_in, device="cuda")
    rout = torch.empty_like(rin)
    batch.sweep(rin, rout)
    torch.cuda.synchronize()
    ref, _ = _oracle_sweep(p, rho_in)
    _check(rout.cpu().numpy(), ref)


def test_masked_2d_sweep_uses_compact_partials_and_finer_groups():
    """With a mask the launch sums partials only for the running instances (indexed by their rank),
    so a batch with few running instances may sweep with finer direction groups than its
    partial-sum buffer holds for all instances: results of running instances match the oracle,
    the others are untouched."""
    rte = _rte()
    p = inputs.random_2d(36, 16, 4, 2, seed=91, B=5, inflow=(0.3, 0.0, 0.8, 0.1), ny=40)
    batch = rte.Batch.from_problem(p)
    rho_in = np.random.default_rng(12).normal(size=(5, p.n_dof))
    for mask in ([0, 1, 0, 1, 1], [0, 0, 0, 0, 1], [1, 1, 1, 1, 1]):
        _, gpu, _ = _gpu_sweep(rte, p, rho_in, active=mask)
        on = [b for b in range(5) if mask[b]]
        ref, _ = _oracle_sweep(p.subset(on), rho_in[on])
        _check(gpu[on], ref)
        off = [b for b in range(5) if not mask[b]]
        assert np.all(gpu[off] == 7.0)


def test_finer_groups_than_the_buffer_holds_for_all_instances():
    """136^2 with CL(64,4) (128 swept directions): one direction per warp needs 76 MB of partial
    sums per instance, above the 64 MB bound, so the batch is sized for two directions per warp.
    With one instance running, the launch sweeps one direction per warp (its partials fit in the
    buffer by rank); the result equals the two-directions-per-warp sweep of all instances to
    rounding (only the summation order of the partials differs)."""
    rte = _rte()
    p = inputs.lattice_test(136, 256, 4)
    batch = rte.Batch.from_problem(p)
    assert batch.info()["min_dirs_per_warp"] == 2
    rho_in = torch.tensor(np.random.default_rng(13).uniform(0, 1, (4, p.n_dof)), device="cuda")
    full = torch.empty_like(rho_in)
    batch.sweep(rho_in, full)
    one = torch.full_like(rho_in, 7.0)
    batch.sweep(rho_in, one, active=torch.tensor([0, 0, 1, 0], dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    f, o = full.cpu().numpy(), one.cpu().numpy()
    assert np.abs(o[2] - f[2]).max() <= 1e-13 * np.abs(f[2]).max()
    assert np.all(o[[0, 1, 3]] == 7.0)


@pytest.mark.parametrize("nx,ny", [(96, 200), (130, 77)])
def test_pipelined_multi_warp_sweep_matches_oracle(nx, ny):
    """Launches with fewer (instance, group) warps than SM sub-partitions share each direction
    group's row blocks among several warps of a CTA (pipelined, block barriers): one instance
    here, 7 and 3 row blocks, inflow on every side, angular flux output included."""
    rte = _rte()
    p = inputs.random_2d(nx, 8, 2, 3, seed=nx + ny, B=1, inflow=(0.6, 0.2, 1.1, 0.4), ny=ny)
    rho_in = np.random.default_rng(14).normal(size=(1, p.n_dof))
    batch, gpu, psi = _gpu_sweep(rte, p, rho_in, psi=True)
    ref, fs = _oracle_sweep(p, rho_in)
    _check(gpu, ref)
    tr, f = fs[0]
    for k, (vx, vy, w, mult) in enumerate(batch.directions()):
        j = int(np.argmin(np.abs(tr.v[:, 0] - vx) + np.abs(tr.v[:, 1] - vy)))
        assert np.abs(psi[0, k] - f[j]).max() < RTOL * np.abs(f[j]).max() * 10


def _corner(problem, b, i0, j0, k, rho):
    """The k x k block of cells starting at (i0, j0) as a problem of its own, with the block's
    materials, sources, incoming scalar flux and the domain's inflow values (only the sides that
    are domain sides matter for the directions compared)."""
    n = problem.nx
    cells = np.array([(j0 + j) * n + (i0 + i) for j in range(k) for i in range(k)])
    h = (problem.domain[1] - problem.domain[0]) / n
    sub = inputs.Problem(2, k, k, (0.0, k * h, 0.0, k * h), "cl", problem.n_phi, problem.n_vz,
                         problem.mat_id[cells].astype(np.int32), problem.sigma_t[b:b + 1].copy(),
                         problem.sigma_s[b:b + 1].copy(), problem.source[b:b + 1, cells].copy(),
                         problem.inflow[b:b + 1].copy(), None, "corner")
    sub_rho = rho.reshape(-1, 4)[cells].reshape(-1)
    return sub, cells, sub_rho


@pytest.mark.slow
def test_sweep_at_the_largest_serving_size_matches_oracle_in_the_inflow_corners():
    """256 x 256 cells, CL(64,4) (128 distinct directions; the largest mesh and angle count of the
    serving workload), random materials and inflow on every side, two instances.  A direction of
    quadrant (sx, sy) sees, in the k x k block of cells at its inflow corner, only that block and
    the inflow on the two domain sides it enters through, so the oracle solves that block alone and
    its angular flux must equal the GPU's there, for every direction of the quadrant.  The scalar
    flux is the weighted sum of the GPU's own angular fluxes (the fused reduction) everywhere."""
    rte = _rte()
    N, k = 256, 12
    p = inputs.random_2d(N, 64, 4, 3, seed=23, B=2, inflow=(0.5, 1.0, 0.2, 0.7))
    rho_in = np.random.default_rng(21).uniform(0, 1, size=(2, p.n_dof))
    batch, rho_out, psi = _gpu_sweep(rte, p, rho_in, psi=True)
    dirs = batch.directions()
    w = np.array([d[2] for d in dirs])
    recon = np.einsum("k,bkn->bn", w, psi)
    assert np.abs(recon - rho_out).max() <= 1e-13 * np.abs(rho_out).max()
    for b in range(2):
        for sx, sy in ((1, 1), (-1, 1), (1, -1), (-1, -1)):
            i0 = 0 if sx > 0 else N - k
            j0 = 0 if sy > 0 else N - k
            sub, cells, sub_rho = _corner(p, b, i0, j0, k, rho_in[b])
            tr = Transport(sub, 0)
            _, f = tr.sweep(sub_rho, store_f=True)
            dof = (cells[:, None] * 4 + np.arange(4)[None, :]).reshape(-1)
            for kd, (vx, vy, _, _) in enumerate(dirs):
                if np.sign(vx) != sx or np.sign(vy) != sy:
                    continue
                j = int(np.argmin(np.abs(tr.v[:, 0] - vx) + np.abs(tr.v[:, 1] - vy)))
                ref = f[j]
                assert np.abs(psi[b, kd, dof] - ref).max() <= RTOL * np.abs(ref).max() * 10
