"""Parameters from device memory (rte_batch_set_params_device) against the host path.

* The device intake (table copies, source moments G sqrt|T|, inflow layout) and the set-up give
  bit-identical sweeps and solves to rte_batch_set_params, in 2D and in 1D (non-uniform mesh,
  cross sections linear across cells).
* Invalid values are caught on the device and reported by the next call that uses the
  parameters (RTE_EINVAL), after which the batch has no parameters (RTE_ESTATE) until they are
  set again.  Invalid values only enter arithmetic, so nothing faults.
"""
import numpy as np
import pytest

from paper_2402_10488_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rte():
    from paper_2402_10488_gb300 import build, rte
    build.build()
    return rte


def _dev(p):
    return [torch.tensor(x, dtype=torch.float64, device="cuda")
            for x in (p.sigma_t, p.sigma_s, p.source, p.inflow)]


def _nonuniform_linear():
    p = inputs.slab_random(29, 8, 4, seed=12, B=3, inflow=(0.4, 1.1), linear=True)
    w = np.random.default_rng(12).uniform(0.5, 1.5, 29)
    edges = np.concatenate([[0.0], np.cumsum(w)])
    edges /= edges[-1]
    edges[-1] = 1.0
    return inputs.replace(p, edges=edges)


@pytest.mark.parametrize("which", ["2d", "1d"])
def test_device_parameters_equal_host_parameters(which):
    rte = _rte()
    if which == "2d":
        p = inputs.random_2d(20, 8, 2, 3, seed=4, B=3, inflow=(0.5, 1.0, 0.2, 0.0))
    else:
        p = _nonuniform_linear()
    disc = rte.Disc(p)
    bh, bd = rte.Batch(disc, p.batch), rte.Batch(disc, p.batch)
    bh.set_params(p)
    bd.set_params_device(*_dev(p))
    rho_in = torch.tensor(np.random.default_rng(1).uniform(0, 1, (p.batch, p.n_dof)), device="cuda")
    oh, od = torch.empty_like(rho_in), torch.empty_like(rho_in)
    bh.sweep(rho_in, oh)
    bd.sweep(rho_in, od)
    assert torch.equal(oh, od)
    rh, rd = torch.zeros_like(rho_in), torch.zeros_like(rho_in)
    reps_h, _, _ = bh.solve(rh, 1e-10, sa=rte.SA_DSA, max_iter=300, dsa_rtol=1e-10)
    reps_d, _, _ = bd.solve(rd, 1e-10, sa=rte.SA_DSA, max_iter=300, dsa_rtol=1e-10)
    assert torch.equal(rh, rd)
    assert [r["n_sweep"] for r in reps_h] == [r["n_sweep"] for r in reps_d]


@pytest.mark.parametrize("bad", ["nan_source", "sigma_s_above_sigma_t", "inf_inflow"])
def test_invalid_device_parameters_are_reported_by_the_next_call(bad):
    rte = _rte()
    p = inputs.random_2d(8, 4, 2, 2, seed=5, B=2)
    batch = rte.Batch.from_problem(p)
    st, ss, src, inf = _dev(p)
    if bad == "nan_source":
        src[1, 3] = float("nan")
    elif bad == "sigma_s_above_sigma_t":
        ss[0, 1] = st[0, 1] * 1.5
    else:
        inf[1, 0] = float("inf")
    batch.set_params_device(st, ss, src, inf)
    rho = torch.zeros((2, p.n_dof), dtype=torch.float64, device="cuda")
    out = torch.empty_like(rho)
    with pytest.raises(rte.RTEError) as e:
        batch.sweep(rho, out)
    assert e.value.status == rte.RTE_EINVAL
    with pytest.raises(rte.RTEError) as e:
        batch.solve(rho, 1e-8)
    assert e.value.status == rte.RTE_ESTATE
    # valid parameters make the batch usable again
    batch.set_params_device(*_dev(p))
    batch.sweep(rho, out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
