"""The allocation-free sweep entry point (rte_sweep_static) against the regular one (rte_sweep).

rte_sweep_static exists for callers that cannot allocate device memory while they run; it keeps
its partial sums in a fixed array of the library instead of memory owned by the batch.  Both
entry points run the same kernels on the same inputs, so their outputs are compared at the
sweep-parity tolerance of the other tests (1e-12 relative), on two calls in a row (the second
call must not see anything left over from the first).  The entry point's defining property --
it allocates no device memory -- is checked by the device's free memory (cudaMemGetInfo) around
repeated calls, in this process and in a fresh one with lazy module loading, where the static
array is allocated when the library's device code that holds it is first loaded (batch creation
does that).  This file is collected last so that a run that stops at the first failure has
already run every other test."""
import os
import subprocess
import sys

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


def test_static_sweep_allocates_no_device_memory():
    rte = _rte()
    p = inputs.lattice_test(64, 32, 2)
    batch = rte.Batch(rte.Disc(p), 2)
    batch.set_params(p)
    rin = torch.rand((2, p.n_dof), dtype=torch.float64, device="cuda")
    out = torch.empty_like(rin)
    batch.sweep(rin, out)                 # loads the sweep kernels
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        batch.sweep_static(rin, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


_LAZY_SCRIPT = r"""
import sys, torch
sys.path.insert(0, sys.argv[1])
from paper_2402_10488_gb300 import inputs, rte
p = inputs.slab_random(40, 16, 3, seed=4, B=2, inflow=(1.0, 0.0))
batch = rte.Batch(rte.Disc(p), 2)
batch.set_params(p)
rin = torch.rand((2, p.n_dof), dtype=torch.float64, device="cuda")
ref, out = torch.empty_like(rin), torch.empty_like(rin)
batch.sweep(rin, ref)
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
batch.sweep_static(rin, out)
batch.sweep_static(rin, out)
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
err = float((out - ref).abs().max() / ref.abs().max())
print("FREE", free0, free1, "ERR", err)
sys.exit(0 if free0 == free1 and err < 1e-12 else 1)
"""


def test_static_sweep_allocates_nothing_under_lazy_module_loading():
    """A fresh process with CUDA_MODULE_LOADING=LAZY: the static array's device code is loaded when
    the batch is created, so the first rte_sweep_static calls leave free device memory unchanged."""
    _rte()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_MODULE_LOADING="LAZY")
    r = subprocess.run([sys.executable, "-c", _LAZY_SCRIPT, root], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
