"""BF16 tensor-core POD products (rte_pod_project_bf16, rte_pod_lift_bf16) and their use in ROMSA.

Pins, derived:
  * Operands that are small integers are exact in BF16, and every partial sum of their products
    stays an integer below 2^24, so the FP32 accumulators are exact too: the products must equal
    the FP64 integer result exactly.  Any misplaced element in the shared-memory layout, the
    tensor-memory read-out or the chunk reduction breaks this.
  * General operands: each operand is rounded once to BF16 (relative error <= u = 2^-8), so each
    product has relative error <= 2u + u^2; FP32 accumulation of at most k terms adds at most
    k * 2^-22 of the sum of magnitudes (2^-22 rather than the IEEE 2^-24: the tensor cores'
    accumulator rounding is not specified as round-to-nearest).  Hence |got - exact| <=
    (2u + u^2 + k 2^-22) * sum |U||X| elementwise (k <= n).
  * In ROMSA the products only change the correction, not the FP64 fixed point: a solve with BF16
    ROM products converges to the oracle's solution at the FP64 tolerance (1e-10) and needs at most
    two more sweeps than with FP64 products.
"""
import time

import numpy as np
import pytest

from oracle.dsa import ConsistentDSA
from oracle.sisa import sisa
from oracle.transport import Transport
from paper_2402_10488_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8   # BF16 keeps 8 significant bits: round-to-nearest error <= 2^-8 relative


def _rte():
    from paper_2402_10488_gb300 import build, rte
    build.build()
    return rte


def _ints(rng, shape):
    return torch.tensor(rng.integers(-8, 9, shape).astype(np.float64), device="cuda")


@pytest.mark.parametrize("r,n,B", [(20, 5003, 150), (32, 8, 1), (1, 65536, 152), (7, 130, 300)])
def test_project_exact_on_integer_operands(r, n, B):
    rte = _rte()
    rng = np.random.default_rng(r * 1000 + B)
    U, X = _ints(rng, (r, n)), _ints(rng, (B, n))
    out = torch.full((B, r), float("nan"), dtype=torch.float64, device="cuda")
    work = rte.pod_workspace(r, n, B)
    for _ in range(2):   # the second call reuses the workspace
        rte.pod_project_bf16(U, X, out, work)
        torch.cuda.synchronize()
        assert torch.equal(out, X @ U.T)
    assert int(work[:4].view(torch.int32)[0]) == 0


@pytest.mark.parametrize("r,n,B", [(20, 1000, 300), (32, 128, 16), (5, 77, 1), (20, 65536, 152)])
def test_lift_exact_on_integer_operands(r, n, B):
    rte = _rte()
    rng = np.random.default_rng(r * 7 + B)
    U, C = _ints(rng, (r, n)), _ints(rng, (B, r))
    Y = torch.full((B, n), float("nan"), dtype=torch.float64, device="cuda")
    work = rte.pod_workspace(r, n, B)
    rte.pod_lift_bf16(U, C, Y, work)
    torch.cuda.synchronize()
    assert torch.equal(Y, C @ U)
    assert int(work[:4].view(torch.int32)[0]) == 0


def test_inactive_instances_are_untouched():
    rte = _rte()
    rng = np.random.default_rng(3)
    r, n, B = 12, 999, 40
    U, X, C = _ints(rng, (r, n)), _ints(rng, (B, n)), _ints(rng, (B, r))
    act = torch.tensor(rng.integers(0, 2, B).astype(np.uint8), device="cuda")
    out = torch.full((B, r), -7.0, dtype=torch.float64, device="cuda")
    Y = torch.full((B, n), -7.0, dtype=torch.float64, device="cuda")
    work = rte.pod_workspace(r, n, B)
    rte.pod_project_bf16(U, X, out, work, active=act)
    rte.pod_lift_bf16(U, C, Y, work, active=act)
    torch.cuda.synchronize()
    on = act.bool()
    assert torch.equal(out[on], (X @ U.T)[on]) and bool((out[~on] == -7.0).all())
    assert torch.equal(Y[on], (C @ U)[on]) and bool((Y[~on] == -7.0).all())


def test_general_operands_within_the_bf16_bound():
    rte = _rte()
    g = torch.Generator(device="cuda").manual_seed(11)
    r, n, B = 20, 65536, 152
    U = torch.randn((r, n), dtype=torch.float64, device="cuda", generator=g)
    X = torch.randn((B, n), dtype=torch.float64, device="cuda", generator=g)
    C = torch.randn((B, r), dtype=torch.float64, device="cuda", generator=g)
    out = torch.empty((B, r), dtype=torch.float64, device="cuda")
    Y = torch.empty((B, n), dtype=torch.float64, device="cuda")
    work = rte.pod_workspace(r, n, B)
    rte.pod_project_bf16(U, X, out, work)
    rte.pod_lift_bf16(U, C, Y, work)
    torch.cuda.synchronize()
    c = 2 * U_BF16 + U_BF16 ** 2 + n * 2.0 ** -22
    assert bool(((out - X @ U.T).abs() <= c * (X.abs() @ U.abs().T)).all())
    c = 2 * U_BF16 + U_BF16 ** 2 + r * 2.0 ** -22
    assert bool(((Y - C @ U).abs() <= c * (C.abs() @ U.abs())).all())
    # and the bound is not vacuous: the products are far from exact in FP64 terms
    assert float((out - X @ U.T).abs().max()) > 0


def test_bad_sizes_are_rejected():
    rte = _rte()
    U = torch.zeros((33, 64), dtype=torch.float64, device="cuda")
    X = torch.zeros((2, 64), dtype=torch.float64, device="cuda")
    out = torch.zeros((2, 33), dtype=torch.float64, device="cuda")
    work = rte.pod_workspace(32, 64, 2)
    with pytest.raises(rte.RTEError) as e:
        rte.pod_project_bf16(U, X, out, work)
    assert e.value.status == rte.RTE_EINVAL


@pytest.mark.parametrize("refine", [False, True])
def test_romsad_with_bf16_rom_products_reaches_the_fp64_solution(refine):
    rte = _rte()
    p = inputs.lattice_test(32, 16, 3, n_vz=2)
    batch = rte.Batch.from_problem(p)
    train = inputs.lattice_train(32, 16, n_train=6, n_vz=2)
    tb = rte.Batch(batch.disc, 6)
    tb.set_params(train)
    _, rc = rte.Rom.build(tb, eps_train=1e-12, window=3, rank_p=4, rank_c=6, max_iter=300,
                          dsa_rtol=1e-10)
    kw = dict(sa=rte.SA_ROMSAD, rom_c=rc, theta=5, eps_romsad=0.1 * max(1e-12, rc.eps_pod),
              rel=True, max_iter=300, dsa_rtol=0.0, dsa_max_it=2)
    if refine:
        kw.update(fp32_switch=1e-4, refine_kappa=0.1, refine_inner=8, gang_wait=4)
    reps = []
    for bf16 in (False, True):
        rho = torch.zeros((3, p.n_dof), dtype=torch.float64, device="cuda")
        rep, _, st = batch.solve(rho, 1e-13, rom_bf16=bf16, **kw)
        assert st == 0
        reps.append(rep)
    for b in range(3):
        assert reps[1][b]["n_romsa"] >= 1
        assert reps[1][b]["n_sweep"] <= reps[0][b]["n_sweep"] + 2, (reps[0][b], reps[1][b])
        tr = Transport(p, b)
        ref = sisa(tr, np.zeros(tr.n_dof), 1e-14, 400, "dsa", dsa=ConsistentDSA(tr), tol_mode="rel")
        assert np.abs(rho.cpu().numpy()[b] - ref["rho"]).max() / np.abs(ref["rho"]).max() < 1e-10


def test_injected_wait_timeout_sets_status_and_leaves_the_context_usable():
    """Failure path of the device-side waits: an injected fault makes the next lift launch issue no
    MMA, so its bounded mbarrier wait runs out (about a second); the status word reports it, nothing
    is left in flight, and the next call on the same context is exact again.  Inside a solve with
    BF16 ROM products the same fault ends the solve with RTE_ETIMEOUT, and the following solve on
    the same batch and ROM succeeds."""
    rte = _rte()
    rng = np.random.default_rng(5)
    r, n, B = 8, 256, 4
    U, C = _ints(rng, (r, n)), _ints(rng, (B, r))
    Y = torch.zeros((B, n), dtype=torch.float64, device="cuda")
    work = rte.pod_workspace(r, n, B)
    rte.fault_inject(rte.FAULT_LIFT_NO_MMA)
    t0 = time.perf_counter()
    rte.pod_lift_bf16(U, C, Y, work)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 30.0
    assert int(work[:4].view(torch.int32)[0]) == 1
    work.zero_()
    rte.pod_lift_bf16(U, C, Y, work)   # one-shot: this call is clean
    torch.cuda.synchronize()
    assert torch.equal(Y, C @ U) and int(work[:4].view(torch.int32)[0]) == 0

    p = inputs.lattice_test(16, 16, 2, n_vz=2)
    batch = rte.Batch.from_problem(p)
    train = inputs.lattice_train(16, 16, n_train=4, n_vz=2)
    tb = rte.Batch(batch.disc, 4)
    tb.set_params(train)
    _, rc = rte.Rom.build(tb, eps_train=1e-12, window=2, rank_p=3, rank_c=4, max_iter=300,
                          dsa_rtol=1e-10)
    kw = dict(sa=rte.SA_ROMSAD, rom_c=rc, theta=5, eps_romsad=0.1 * max(1e-12, rc.eps_pod),
              rel=True, max_iter=300, dsa_rtol=0.0, dsa_max_it=2, rom_bf16=True)
    rho = torch.zeros((2, p.n_dof), dtype=torch.float64, device="cuda")
    rte.fault_inject(rte.FAULT_LIFT_NO_MMA)
    with pytest.raises(rte.RTEError) as e:
        batch.solve(rho, 1e-12, **kw)
    assert e.value.status == rte.RTE_ETIMEOUT
    rho.zero_()
    rep, _, st = batch.solve(rho, 1e-12, **kw)
    assert st == rte.RTE_OK and all(x["converged"] and x["n_romsa"] >= 1 for x in rep)
