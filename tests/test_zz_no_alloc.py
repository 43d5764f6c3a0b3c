"""The allocation-free sweep entry point (rte_sweep_static) against the regular one (rte_sweep).

rte_sweep_static exists for callers that cannot allocate device memory while they run; it keeps
its partial sums in a fixed array of the library instead of memory owned by the batch.  Both
entry points run the same kernels on the same inputs, so their outputs are compared at the
sweep-parity tolerance of the other tests (1e-12 relative), on two calls in a row (the second
call must not see anything left over from the first).  This file is collected last so that a
run that stops at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2402_10488_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-12


def _rte():
    from paper_2402_10488_gb300 import build, rte
    build.build()
    return rte


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("make,dpw", [
    (lambda: inputs.lattice_test(128, 64, 3), 4),
    (lambda: inputs.random_2d(37, 8, 4, 3, seed=5, B=2, inflow=(0.3, 1.2, 0.7, 0.0), ny=19), 0),
    (lambda: inputs.slab_random(45, 16, 4, seed=8, B=3, inflow=(1.5, 0.25)), 0),
])
def test_static_sweep_matches_regular_sweep_twice(make, dpw):
    rte = _rte()
    p = make()
    batch = rte.Batch(rte.Disc(p), p.batch)
    batch.tune(dpw)   # the decomposition sets how many partial sums the batch needs
    batch.set_params(p)
    gen = torch.Generator(device="cuda").manual_seed(7)
    for call in range(2):
        rin = torch.rand((p.batch, p.n_dof), dtype=torch.float64, device="cuda", generator=gen)
        ref = torch.empty_like(rin)
        got = torch.full_like(rin, float("nan"))
        batch.sweep(rin, ref)
        batch.sweep_static(rin, got, with_source=(call == 0))
        if call == 1:
            batch.sweep(rin, ref, with_source=False)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert _rel(got, ref) < RTOL, (call, _rel(got, ref))


def test_static_sweep_rejects_batches_beyond_its_scratch():
    rte = _rte()
    p = inputs.lattice_test(128, 64, 5)  # 5 x 8 groups x 65536 doubles > 2^21
    batch = rte.Batch(rte.Disc(p), 5)
    batch.tune(4)
    batch.set_params(p)
    rin = torch.zeros((5, p.n_dof), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(rin)
    with pytest.raises(rte.RTEError) as e:
        batch.sweep_static(rin, out)
    assert e.value.status == rte.RTE_EINVAL and "static scratch" in str(e.value)
