"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every entry point
declared in include/rte.h; the Python binding declares exactly those entry points."""
import os
import re

import pytest

from paper_2402_10488_gb300 import build, rte

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "rte.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(rte_\w+)\s*\(", text, re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    L = rte.lib()
    syms = declared_symbols()
    assert len(syms) >= 20
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing
    assert set(syms) == set(rte.SIGNATURES), set(syms) ^ set(rte.SIGNATURES)
    assert L.rte_version() == 10200


def test_calls_without_gpu_fail_cleanly():
    """Without a device the calls return a status and a message; nothing crashes."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2402_10488_gb300 import inputs
    with pytest.raises(rte.RTEError) as e:
        rte.Disc(inputs.slab(4, 2, 1.0, 0.5))
    assert e.value.status in (rte.RTE_ECUDA, rte.RTE_EINVAL)
