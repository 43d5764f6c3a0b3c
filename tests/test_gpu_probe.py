"""The FMA throughput probe that supplies the sweep's roofline denominators (rte_fma_peak): it runs,
reports a finite positive rate for both pipes, and the FP32 pipe is far wider than the FP64 one on
this GPU (GB300 issues FP64 FMAs at a small fraction of the FP32 rate); bad arguments are refused."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fma_peak_probe():
    from paper_2402_10488_gb300 import build, rte
    build.build()
    f64, f32 = rte.fma_peak("fp64"), rte.fma_peak("fp32")
    assert math.isfinite(f64) and math.isfinite(f32) and 0 < f64 < f32
    assert f32 > 10 * f64
    with pytest.raises(rte.RTEError) as e:
        rte.check(rte.lib().rte_fma_peak(0, 7, None, None))
    assert e.value.status == rte.RTE_EINVAL
    with pytest.raises(rte.RTEError):
        rte.fma_peak("fp64", device=1000)
