"""GPU checks of a solution in FP64 (rte_residual, rte_solve_opts.verify) against the oracle, through
the C ABI: the residual ||(I - L) rho - b-bar||_inf of Eq. (rho_matrix_vec) that the paper averages
into R^rho_inf (notation table of Sec. 4), the per-cell particle balance of one sweep (the DG
equation tested with a cell's indicator function) and the global balance absorption + net
leakage = source; and the per-sweep record of Alg. 2's correction choices.

Tolerances, derived: the GPU sweep agrees with the oracle's to 1e-12 relative to ||rho*||_inf (the
sweep parity bar), so the residual max|rho - rho*| agrees to 1e-12 ||rho*||_inf.  The per-cell
balance is a sum of terms of size sq|T| sigma_t |rho*_0|; an exact sweep makes it zero, and both
sides' rounding leaves ~1e-15 of the largest such term, so both must vanish to 1e-12 of it and
agree to that bound.  The global balance sums n_cells such terms with cancellation: compared at
1e-11 of the summed magnitudes.  An unconverged random rho keeps every compared quantity of order
one, so agreement is not agreement of two round-off values."""
import numpy as np
import pytest

from oracle.transport import Transport, cell_balance
from paper_2402_10488_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rte():
    from paper_2402_10488_gb300 import build, rte
    build.build()
    return rte


def _sq(tr):
    dg = tr.dg
    return np.sqrt(dg.h) if tr.dim == 1 else np.full(dg.n_cells, np.sqrt(dg.hx * dg.hy))


def _oracle(problem, b, rho):
    """R_inf, per-cell balance, global balance defect and int G of one instance from the oracle:
    leakage from its edge traces (net_upwind_outflow), volume integrals from its mass matrices."""
    tr = Transport(problem, b)
    rho_star, f = tr.sweep(rho, store_f=True)
    r_inf = tr.residual_inf(rho)
    bal = cell_balance(tr, rho, f)
    n, P = tr.dg.n_cells, tr.dg.P
    sq = _sq(tr)
    leak = sum(tr.w[j] * tr.dg.net_upwind_outflow(tr.v[j], f[j], tr.inflow) for j in range(tr.n_angles))
    absorb = sq * (tr.Sa @ rho_star).reshape(n, P)[:, 0]     # int_T sigma_a rho* per cell
    src = sq * tr.G.reshape(n, P)[:, 0]                      # int_T G per cell
    glob = leak.sum() + absorb.sum() - src.sum()
    mag = np.abs(leak).sum() + np.abs(absorb).sum() + np.abs(src).sum()
    term = np.abs(sq * tr.sigma_t_cell * rho_star.reshape(n, P)[:, 0]).max()
    return r_inf, bal, glob, src.sum(), mag, term, np.abs(rho_star).max()


CASES = [
    ("2d_random_inflow", lambda: inputs.random_2d(37, 8, 2, 3, seed=5, B=3, inflow=(0.3, 0.0, 1.2, 0.7), ny=19)),
    ("2d_lattice", lambda: inputs.lattice_test(24, 32, 2)),
    ("1d_slab_inflow", lambda: inputs.slab_random(50, 16, 3, seed=7, B=2, inflow=(1.0, 0.4))),
    ("1d_linear_sigma", lambda: inputs.slab_random(40, 8, 4, seed=9, B=2, inflow=(0.0, 2.0), linear=True)),
    ("1d_nonuniform_inflow", lambda: inputs.two_material(np.array([[0.7, 12.0], [1.3, 25.0]]))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_residual_and_balance_match_oracle(name, make):
    rte = _rte()
    p = make()
    batch = rte.Batch.from_problem(p)
    rho = np.random.default_rng(11).uniform(0.0, 1.0, (p.batch, p.n_dof))
    rin = torch.tensor(rho, device="cuda")
    out = torch.full((p.batch, 4), 7.0, dtype=torch.float64, device="cuda")
    cb = torch.full((p.batch, p.n_cells), 7.0, dtype=torch.float64, device="cuda")
    batch.residual(rin, out, cb)
    torch.cuda.synchronize()
    got, gcb = out.cpu().numpy(), cb.cpu().numpy()
    for b in range(p.batch):
        r_inf, bal, glob, src, mag, term, rs_max = _oracle(p, b, rho[b])
        assert r_inf > 1e-3 * rs_max   # an unconverged rho: the residual is of order one
        assert abs(got[b, 0] - r_inf) <= 1e-12 * rs_max, (b, got[b, 0], r_inf)
        assert np.abs(gcb[b]).max() <= 1e-12 * term, np.abs(gcb[b]).max() / term
        assert np.abs(bal).max() <= 1e-12 * term
        assert np.abs(gcb[b] - bal).max() <= 1e-12 * term
        assert abs(got[b, 1] - np.abs(gcb[b]).max()) == 0.0
        assert abs(glob) > 1e-6 * mag   # not a cancellation to round-off
        assert abs(got[b, 2] - glob) <= 1e-11 * mag, (b, got[b, 2], glob)
        assert abs(got[b, 3] - src) <= 1e-13 * max(abs(src), 1e-300) + 1e-300


def test_residual_with_mask_and_repeat():
    """Masked instances are left untouched, and a second call (the batch keeps its face-outflow
    buffer) gives bit-identical results."""
    rte = _rte()
    p = inputs.random_2d(40, 8, 2, 2, seed=3, B=4, inflow=(0.5, 0.1, 0.0, 0.2), ny=33)
    batch = rte.Batch.from_problem(p)
    rho = torch.tensor(np.random.default_rng(2).uniform(0, 1, (4, p.n_dof)), device="cuda")
    full = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    batch.residual(rho, full)
    masked = torch.full((4, 4), -1.0, dtype=torch.float64, device="cuda")
    act = torch.tensor([0, 1, 0, 1], dtype=torch.uint8, device="cuda")
    batch.residual(rho, masked, active=act)
    again = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    batch.residual(rho, again)
    torch.cuda.synchronize()
    assert torch.equal(full, again)
    assert torch.equal(masked[1], full[1]) and torch.equal(masked[3], full[3])
    assert bool((masked[0] == -1.0).all()) and bool((masked[2] == -1.0).all())


def test_verified_solve_reports_paper_level_residual():
    """SI-DSA converged tightly with verify: the report's R^rho_inf is at the level the paper prints
    (1e-12 .. 1e-14) and equals the oracle's residual of the returned rho; the global balance
    vanishes with it; the per-sweep record says DSA after every sweep but the last."""
    rte = _rte()
    p = inputs.lattice_test(16, 32, 2)
    batch = rte.Batch.from_problem(p)
    rho = torch.zeros((2, p.n_dof), dtype=torch.float64, device="cuda")
    reps, hist, st = batch.solve(rho, 1e-14, rel=True, max_iter=200, dsa_rtol=1e-13,
                                 dsa_max_it=3000, verify=True, history=True)
    assert st == rte.RTE_OK
    got = rho.cpu().numpy()
    for b in range(2):
        r = reps[b]
        tr = Transport(p, b)
        ref = tr.residual_inf(got[b])
        scale = np.abs(got[b]).max()
        assert r["r_inf"] < 1e-12 * scale
        assert abs(r["r_inf"] - ref) <= 1e-12 * scale
        # G = 1 on the unit square: int G = 1; the largest per-cell term is sq|T| sigma_t rho_0
        term = np.abs(_sq(tr) * tr.sigma_t_cell * got[b].reshape(-1, 4)[:, 0]).max()
        assert abs(r["balance"]) < 1e-10
        assert r["balance_cell"] < 1e-12 * term
        codes = r["sa_history"]
        assert len(codes) == r["n_sweep"]
        assert list(codes[:-1]) == [rte.SA_DSA] * (r["n_sweep"] - 1) and codes[-1] == rte.SA_NONE


def test_sa_history_marks_fp32_sweeps():
    """Precision variant: the sweeps marked FP32 in the record are exactly the report's n_sweep32,
    and the last (stopping) sweep is an FP64 one."""
    rte = _rte()
    p = inputs.lattice_test(16, 32, 2)
    batch = rte.Batch.from_problem(p)
    rho = torch.zeros((2, p.n_dof), dtype=torch.float64, device="cuda")
    reps, _, st = batch.solve(rho, 1e-10, rel=True, max_iter=200, dsa_rtol=0.0, dsa_max_it=2,
                              fp32_switch=1e-4, refine_kappa=0.1, refine_inner=8, history=True,
                              verify=True)
    assert st == rte.RTE_OK
    for r in reps:
        codes = r["sa_history"]
        assert int(np.sum((codes & 0x10) != 0)) == r["n_sweep32"] > 0
        assert codes[-1] == rte.SA_NONE
        assert all((c & 0x0F) == rte.SA_DSA for c in codes[:-1])
        assert r["r_inf"] < 1e-9 * r["rho_inf"]
