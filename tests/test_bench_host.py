"""CPU checks of bench.py's host logic: the precision-variant methods map to the solver options
their description states (the measured settings of the FP64 outer residual correction), and the
options round-trip through the binding's rte_solve_opts."""
import sys

from paper_2402_10488_gb300 import rte


def _defaults(monkeypatch):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    return bench, bench.parse()


def test_precision_methods_map_to_solver_options(monkeypatch):
    bench, a = _defaults(monkeypatch)
    assert bench.precision_kw("romsad", a) == {}
    assert bench.precision_kw("si_dsa", a) == {}
    assert bench.precision_kw("romsad_mixed", a) == dict(fp32_switch=1e-5)
    kw = bench.precision_kw("romsad_refine", a)
    assert kw == dict(fp32_switch=1e-5, refine_kappa=0.1, refine_inner=8, gang_wait=4,
                      rom_bf16=False)
    o = rte.solve_opts(2e-7, rte.SA_ROMSAD, rel=True, theta=5, eps_romsad=1e-4, **kw)
    assert (o.fp32_switch, o.refine_kappa, o.refine_inner, o.gang_wait, o.rom_bf16) == \
        (1e-5, 0.1, 8, 4, 0)
    assert o.sa == rte.SA_ROMSAD and o.rel == 1 and o.theta == 5


def test_default_bench_runs_every_method_on_one_sm_per_instance(monkeypatch):
    _, a = _defaults(monkeypatch)
    assert a.batch == 152 and a.n == 128 and a.angles == 64 and a.rank == 20
    methods = a.methods.split(",")
    assert methods[0] == "romsad"
    assert {"si_dsa", "romig", "romsad_mixed", "romsad_refine", "pgmres"} <= set(methods)
    assert a.warmup >= 3 and a.dsa_smoother == -1
