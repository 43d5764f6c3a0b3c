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
    assert o.sa == rte.SA_ROMSAD and o.rel == 1 and o.theta == 5 and o.outer_ff == 0
    kff = bench.precision_kw("romsad_refine_ff", a)
    assert kff == dict(kw, outer_ff=True)
    assert rte.solve_opts(2e-7, rte.SA_ROMSAD, rel=True, **kff).outer_ff == 1


def test_default_bench_runs_every_method_on_one_sm_per_instance(monkeypatch):
    _, a = _defaults(monkeypatch)
    assert a.batch == 152 and a.n == 128 and a.angles == 64 and a.rank == 20
    methods = a.methods.split(",")
    assert methods[0] == "romsad"
    assert {"si_dsa", "romig", "romsad_mixed", "romsad_refine", "romsad_refine_ff",
            "pgmres"} <= set(methods)
    assert a.warmup >= 3 and a.dsa_smoother == -1


def _tiny(monkeypatch, steps=3, warmup=1):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--n", "8", "--angles", "8",
                                      "--ntrain", "4", "--rank", "3", "--steps", str(steps),
                                      "--warmup", str(warmup), "--eps", "1e-8"])
    return bench, bench.parse()


def test_reference_arm_times_whole_oracle_solves(monkeypatch):
    """The reference arm on a tiny lattice: the oracle's own offline stage, then K complete ROMSAD
    solves timed as one concurrent region; the timed region is the steps' wall time (so K x
    ms_per_step is inside the run), every solve converges and the counts are the oracle's own."""
    import time
    bench, a = _tiny(monkeypatch)
    t0 = time.perf_counter()
    line = bench.run_reference(a, 1, 0)
    total = time.perf_counter() - t0
    assert line["impl"] == "reference" and line["steps"] == 3 and line["warmup"] == 1
    assert line["steps"] * line["ms_per_step"] / 1e3 <= total
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == bench.oracle_workers()
    assert line["config"]["global_batch"] == max(3, bench.oracle_workers())
    assert line["value"] == cb["value"] == line["e2e"]["value"] > 0
    # a correction follows every sweep but the one that stopped the solve
    assert cb["n_romsa_mean"] >= 1
    assert abs(cb["n_sweep_mean"] - (cb["n_romsa_mean"] + cb["n_dsa_mean"] + 1)) < 1e-12
    assert bench.run_reference(a, 2, 1) is None   # other ranks do no work


def test_cpu_baseline_leg_runs_one_instance_per_core(monkeypatch):
    bench, a = _tiny(monkeypatch)
    cb = bench.cpu_baseline_leg(a, dict(n_sweep=4.4))
    assert cb["cores"] == bench.oracle_workers() and cb["value"] > 0
    assert "4 iterations" in cb["sample"]


def test_lattice_methods_without_the_headline_are_refused(monkeypatch):
    """The lattice workload's JSON line is ROMSAD's: a --methods list without it is refused with a
    message at parse time instead of failing after the GPU work."""
    import pytest
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--methods", "si_dsa,romsad_refine"])
    with pytest.raises(SystemExit):
        bench.parse()
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "mixed", "--methods", "si_dsa"])
    assert bench.parse().methods == "si_dsa"
