"""Benchmark: parametric lattice solves per second at 1e-6 scalar-flux error on one GB300.

Workload: two-material lattice cell on [0,1]^2, 128 x 128 DG-Q1 cells, CL(16,4) (64 angles),
sigma_s ~ U[1,100] in the centred 0.4-wide inclusion and U[0.1,1] outside, sigma_a ~ U[0.01,0.1],
G = 1, vacuum inflow.  Offline (untimed, as in the paper's T_rel): 32 training instances,
SI-DSA to 1e-12, POD ranks 20/20, window 3.  One step = one batch of B test instances solved
from scratch: per-instance set-up (cell tables, DSA multigrid hierarchy, reduced operators)
plus SI with the chosen correction, each instance stopping on its own relative change.  A solve
counts only if its scalar flux is within 1e-6 (relative, inf-norm) of a tightly converged
reference.  The headline value is ROMSAD (ROMSA for l <= theta = 5, then DSA; Alg. 2); SI-DSA
and ROMIG are timed on the same GPU in the same run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): instances are sharded across ranks with no data-path collective
(weak scaling); the barrier and the max over ranks of the timed region stay.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s at 1e-6 φ error (ROMSAD vs SI-DSA, same GPU); sweep GB/s; p50/p99 ms"
FP64_PEAK_NOMINAL = 1.25    # GB300 FP64 rate from the unit table (used only if the probe fails)
# 32 FMA per cell and distinct direction: 8 to form the right-hand side s + E_x t_x + E_y t_y, 16
# to apply M^-1, 4 for the outflow traces, 4 for the scalar-flux accumulation
FLOP_PER_CELL_DIR = 64
BYTES_PER_CELL_SWEEP = 76   # rho_in 32 B + G0 8 B + material id 4 B + rho_out 32 B
# DRAM bytes per sweep launch from the committed ncu capture, valid only for the 2D sweep
# kernels' device code it was taken with (sha1 of that part of sweep.cu, sweep_source_sha1)
NCU_TRAFFIC = {"sha1": "32a0ca5935ea53a2bf4d4e7a16f14e57c612f105", "bytes_per_launch": 723429811,
               "batch": 152, "n": 128, "angles": 64,
               "workload": "lattice128x128_CL(16,4) batch 152, mean of the 10 sweep2d_kernel launches "
                           "of one ROMSAD step"}


def sweep_source_sha1():
    """sha1 of the 2D sweep kernels' device code: sweep.cu up to the 1D sweep's argument struct
    (the cell solve, sweep2d_warp and the kernels built on it) and the 2D argument struct in
    common.cuh."""
    csrc = os.path.join(ROOT, "paper_2402_10488_gb300", "csrc")
    with open(os.path.join(csrc, "sweep.cu"), "rb") as fh:
        src = fh.read()
    with open(os.path.join(csrc, "common.cuh"), "rb") as fh:
        hdr = fh.read()
    b = src.find(b"struct Sweep1DArgs {")
    a0, a1 = hdr.find(b"struct Sweep2DArgs {"), hdr.find(b"struct SweepItem {")
    part = (src[:b] if b > 0 else src) + (hdr[a0:a1] if 0 <= a0 < a1 else hdr)
    return hashlib.sha1(part).hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=152,
                    help="test instances per step per GPU (152 = one per SM: with 4 directions "
                         "per warp, exactly two warps per SM sub-partition)")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--angles", type=int, default=64)
    ap.add_argument("--ntrain", type=int, default=32)
    ap.add_argument("--rank", type=int, default=20)
    ap.add_argument("--eps", type=float, default=2e-7, help="relative stop tolerance")
    ap.add_argument("--dsa-rtol", type=float, default=0.0, help="0: fixed V-cycles")
    ap.add_argument("--dsa-vcycles", type=int, default=1)
    ap.add_argument("--dsa-nu", type=int, default=2, help="DSA multigrid smoothing sweeps per level")
    ap.add_argument("--dsa-smoother", type=int, default=-1,
                    help="DSA smoother form: 0 global, 1 shared-memory tiles, 2 temporally "
                         "blocked, -1 the library default")
    ap.add_argument("--fp32-switch", type=float, default=1e-5,
                    help="precision variant: FP32 sweeps until the relative change is below this")
    ap.add_argument("--dpw", type=int, default=-1,
                    help="sweep directions per warp (0 = occupancy rule per launch, -1 = measured "
                         "by the autotuner before timing)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--refine-kappa", type=float, default=0.1,
                    help="romsad_refine: FP32 correction sweeps after an FP64 sweep until their "
                         "change is this fraction of the FP64 one")
    ap.add_argument("--refine-inner", type=int, default=8,
                    help="romsad_refine: at most this many FP32 correction sweeps per FP64 sweep")
    ap.add_argument("--gang-wait", type=int, default=4,
                    help="romsad_refine: an instance due for an FP64 sweep waits up to this many "
                         "iterations while others still sweep in FP32 (fuller FP64 launches)")
    ap.add_argument("--refine-rom-bf16", type=int, default=0,
                    help="romsad_refine: ROMSA's project/lift products in BF16 on the tensor cores")
    ap.add_argument("--refine-switch", type=float, default=1e-5,
                    help="romsad_refine: FP32 sweeps (with sources) until the relative change is "
                         "below this, then the FP64 outer residual correction")
    ap.add_argument("--methods", default="romsad,romsad_interleaved,si_dsa,romig,romig_romsad,"
                                         "romsad_mixed,romsad_refine,romsad_refine_ff,pgmres,"
                                         "romig_pgmres")
    ap.add_argument("--gmres-rtol", type=float, default=1e-7,
                    help="pgmres: relative residual of the preconditioned system")
    ap.add_argument("--profile-window", action="store_true",
                    help="bracket the timed ROMSAD steps with cudaProfilerStart/Stop (for ncu)")
    ap.add_argument("--workload", default="lattice",
                    choices=["lattice", "mixed", "serving", "paper", "paper1d"],
                    help="lattice: one discretisation, batches of --batch instances; mixed: 256 "
                         "instances over 12 (mesh, angles) buckets solved together; serving: a "
                         "Poisson request stream over 20 buckets through the serving loop")
    ap.add_argument("--instances", type=int, default=256, help="mixed: instances per step per GPU")
    ap.add_argument("--mixed-exec", default="streams", choices=["lockstep", "streams"],
                    help="mixed: FP64 methods iterate all buckets in lockstep with one sweep launch "
                         "per iteration (rte_solve_lockstep), or each bucket on its own stream "
                         "(rte_solve_many); the precision variants always use the streams")
    ap.add_argument("--requests", type=int, default=2000, help="serving: requests in the stream")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: mean arrivals per second")
    ap.add_argument("--mem-gb", type=float, default=96.0,
                    help="serving: device memory for slots, shared equally by the buckets")
    ap.add_argument("--max-slots", type=int, default=64, help="serving: slots per bucket at most")
    ap.add_argument("--cellwise-sigma", action="store_true",
                    help="paper1d workload: the cross-regime sigma_s at its cell averages instead "
                         "of linear inside each cell")
    ap.add_argument("--paper-dsa", default="fgmres", choices=["fgmres", "vcycle"],
                    help="paper workload: DSA solved by FGMRES to 1e-8 (sweep counts comparable "
                         "with the paper's AMG) or by --dsa-vcycles FP32 V-cycles (speed)")
    ap.add_argument("--kappa", type=float, default=0.1,
                    help="mixed/serving: stop at relative change kappa * error target")
    a = ap.parse_args()
    if a.impl == "ours" and a.workload == "lattice" and "romsad" not in a.methods.split(","):
        ap.error("--methods must include romsad: the lattice workload's headline line is ROMSAD's")
    return a


def precision_kw(method, a):
    """Solver options of the precision variants: romsad_mixed sweeps in FP32 until the change is
    below --fp32-switch and in FP64 afterwards; romsad_refine follows its FP32 phase with the FP64
    outer residual correction (FP64 sweeps of the iterate, FP32 sweeps of the error equation);
    romsad_refine_ff is romsad_refine with those FP64 sweeps in float-float arithmetic."""
    if method == "romsad_mixed":
        return dict(fp32_switch=a.fp32_switch)
    if method in ("romsad_refine", "romsad_refine_ff"):
        kw = dict(fp32_switch=a.refine_switch, refine_kappa=a.refine_kappa,
                  refine_inner=a.refine_inner, gang_wait=a.gang_wait,
                  rom_bf16=bool(a.refine_rom_bf16))
        if method == "romsad_refine_ff":
            kw["outer_ff"] = True
        return kw
    return {}


# ---- multi-process plumbing ----------------------------------------------------------------

def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return ws, rank, local


def test_seeds(rank, B):
    """Test-instance seeds of one rank: instances are sharded across ranks (weak scaling)."""
    from paper_2402_10488_gb300 import inputs
    return [inputs.TEST_SEED0 + rank * B + k for k in range(B)]


def _reduce_device():
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(ws, solves_local, seconds_local):
    """Whole-job solves/s: solves of all ranks over the slowest rank's timed region."""
    return sum_over_ranks(ws, solves_local) / max_over_ranks(ws, seconds_local)


# ---- clocks ----------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = os.path.join("/tmp", f"rte_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ---- the GPU arm -----------------------------------------------------------------------------

def measured_peaks(rte, dev):
    """FP64 and FP32 FMA throughput of this GPU now (rte_fma_peak): the roofline denominators of the
    FP64 and FP32 sweeps, which are bound by FMA issue.  Falls back to the nominal FP64 rate."""
    try:
        return dict(fp64=rte.fma_peak("fp64", dev), fp32=rte.fma_peak("fp32", dev),
                    source="measured in this run: rte_fma_peak (independent FMA chains, 4 x 256 "
                           "threads per SM, best of 5 CUDA-event-timed launches)")
    except Exception as e:   # the bench line must still be printed
        return dict(fp64=FP64_PEAK_NOMINAL, fp32=None,
                    source=f"nominal FP64 1.25 TFLOP/s (probe failed: {str(e)[:120]})")


def residual_stats(rte, batch, rho, torch):
    """R^rho_inf = ||(I - L) rho - b-bar||_inf (absolute, as the paper reports it) and the global
    particle balance of every instance's result, from one extra FP64 sweep (rte_residual)."""
    out = torch.zeros((batch.B, 4), dtype=torch.float64, device="cuda")
    batch.residual(rho, out)
    v = out.cpu().numpy()
    scale = np.abs(rho.cpu().numpy()).max(1)
    return dict(r_inf_mean=float(v[:, 0].mean()), r_inf_max=float(v[:, 0].max()),
                r_inf_rel_max=float((v[:, 0] / scale).max()),
                balance_rel_max=float((np.abs(v[:, 2]) / np.maximum(v[:, 3], 1e-300)).max()))


def run_ours(a, ws, rank, local):
    import torch

    import __graft_entry__
    from paper_2402_10488_gb300 import inputs, rte

    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = local
    nvz = 4
    nphi = a.angles // nvz
    B = a.batch
    train = inputs.lattice(a.n, a.angles, [inputs.TRAIN_SEED0 + k for k in range(a.ntrain)], nvz)
    test = inputs.lattice(a.n, a.angles, test_seeds(rank, B), nvz)
    disc = rte.Disc(train, device=dev)
    tb = rte.Batch(disc, train.batch)
    tb.set_params(train)
    t0 = time.time()
    rom_p, rom_c = rte.Rom.build(tb, eps_train=1e-12, window=3, rank_p=a.rank, rank_c=a.rank,
                                 max_iter=500, dsa_rtol=1e-8)
    methods = [m for m in a.methods.split(",") if m]
    rom_ci = None
    if "romig_romsad" in methods:  # correction ROM trained from ROMIG-started runs
        _, rom_ci = rte.Rom.build(tb, eps_train=1e-12, window=3, rank_p=a.rank, rank_c=a.rank,
                                  max_iter=500, dsa_rtol=1e-8, correction_start="romig")
    offline_s = time.time() - t0
    eps_train = 1e-12
    eps_romsad = 0.1 * max(eps_train, rom_c.eps_pod)
    eps_romsad_i = 0.1 * max(eps_train, rom_ci.eps_pod) if rom_ci else None
    batch = rte.Batch(disc, B)
    batch.tune(max(a.dpw, 0))
    batch.dsa_smoothing(a.dsa_nu)
    if a.dsa_smoother >= 0:
        batch.dsa_smoother(a.dsa_smoother)
    batch.set_params(test)
    tuned = batch.autotune() if a.dpw < 0 else None
    if tuned:   # (count, dirs per warp, warps per direction group) of the FP64 sweep
        tuned = batch.tuned() or tuned
    n_dof = disc.n_dof
    # romsad_interleaved: the same instances as two halves (separate batches, each with its own copy
    # of the correction ROM) solved by rte_solve_interleaved
    halves, half_roms, half_streams = [], [], []
    if "romsad_interleaved" in methods:
        h = B // 2
        seeds = test_seeds(rank, B)
        with tempfile.TemporaryDirectory() as tmp:
            rom_c.save(os.path.join(tmp, "rom_c.bin"))
            half_roms = [rom_c, rte.Rom.load(disc, os.path.join(tmp, "rom_c.bin"))]
        for lo, hi in ((0, h), (h, B)):
            hb = rte.Batch(disc, hi - lo)
            hb.tune(max(a.dpw, 0))
            hb.dsa_smoothing(a.dsa_nu)
            if a.dsa_smoother >= 0:
                hb.dsa_smoother(a.dsa_smoother)
            hb.set_params(inputs.lattice(a.n, a.angles, seeds[lo:hi], nvz))
            if a.dpw < 0:
                hb.autotune()
            halves.append((lo, hi, hb))
        half_streams = [torch.cuda.Stream() for _ in halves]
    # tightly converged references (untimed)
    ref = torch.zeros((B, n_dof), dtype=torch.float64, device="cuda")
    rep_ref, _, _ = batch.solve(ref, 1e-13, sa=rte.SA_DSA, rel=True, max_iter=400, dsa_rtol=1e-3)
    ref_np = ref.cpu().numpy()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()

    # the test parameters resident in HBM (value) or in pinned host memory (e2e, copied every step)
    par_dev = [torch.tensor(x, dtype=torch.float64, device="cuda")
               for x in (test.sigma_t, test.sigma_s, test.source, test.inflow)]
    par_host = [t.cpu().pin_memory() for t in par_dev]
    par_in = [torch.empty_like(t) for t in par_dev]

    def step_interleaved(rho):
        # the halves' parameters from the same resident tensors, then both halves solved together
        for lo, hi, hb in halves:
            hb.set_params_device(*[t[lo:hi] for t in par_dev])
        rho.zero_()
        cur = torch.cuda.current_stream()
        for s_ in half_streams:
            s_.wait_stream(cur)
        opts = [rte.solve_opts(a.eps, rte.SA_ROMSAD, rel=True, max_iter=400, theta=5,
                               eps_romsad=eps_romsad, dsa_rtol=a.dsa_rtol,
                               dsa_max_it=a.dsa_vcycles if a.dsa_rtol == 0 else 100)
                for _ in halves]
        reps, _ = rte.solve_many([hb for _, _, hb in halves], [rho[lo:hi] for lo, hi, _ in halves],
                                 opts, roms=half_roms, streams=half_streams, interleaved=True)
        return [x for rr in reps for x in rr]

    def step(method, rho, host_out=None):
        if method == "romsad_interleaved":
            return step_interleaved(rho)
        if host_out is not None:
            for d, h in zip(par_in, par_host):
                d.copy_(h, non_blocking=True)
            batch.set_params_device(*par_in)
        else:
            batch.set_params_device(*par_dev)
        rho.zero_()
        if method == "romig":
            rom_p.initial_guess(batch, rho)
            sa, kw = rte.SA_DSA, {}
        elif method == "romsad":
            sa, kw = rte.SA_ROMSAD, dict(rom_c=rom_c, theta=5, eps_romsad=eps_romsad)
        elif method in ("romsad_mixed", "romsad_refine", "romsad_refine_ff"):
            sa, kw = rte.SA_ROMSAD, dict(rom_c=rom_c, theta=5, eps_romsad=eps_romsad,
                                         **precision_kw(method, a))
        elif method == "romig_romsad":
            rom_p.initial_guess(batch, rho)
            sa, kw = rte.SA_ROMSAD, dict(rom_c=rom_ci, theta=5, eps_romsad=eps_romsad_i)
        elif method in ("pgmres", "romig_pgmres"):
            # the paper's comparison system: DSA-preconditioned GMRES(25) on (I - L) rho = b-bar
            if method == "romig_pgmres":
                rom_p.initial_guess(batch, rho)
            rep, _ = batch.pgmres(rho, a.gmres_rtol, restart=25, max_iter=400,
                                  dsa_rtol=a.dsa_rtol,
                                  dsa_max_it=a.dsa_vcycles if a.dsa_rtol == 0 else 100,
                                  zero_start=method == "pgmres")
            if host_out is not None:
                host_out.copy_(rho, non_blocking=True)
            return rep
        else:
            sa, kw = rte.SA_DSA, {}
        rep, _, st = batch.solve(rho, a.eps, sa=sa, rel=True, max_iter=400, dsa_rtol=a.dsa_rtol,
                                 dsa_max_it=a.dsa_vcycles if a.dsa_rtol == 0 else 100, **kw)
        if host_out is not None:
            host_out.copy_(rho, non_blocking=True)
        return rep

    def measure(method, steps, warmup, host=False):
        rho = torch.zeros((B, n_dof), dtype=torch.float64, device="cuda")
        hbuf = torch.empty((B, n_dof), dtype=torch.float64, pin_memory=True) if host else None
        for _ in range(warmup):
            step(method, rho, hbuf)
        torch.cuda.synchronize()
        times, reps = [], []
        launches0 = rte.launch_count()
        timed = [hb for _, _, hb in halves] if method == "romsad_interleaved" else [batch]
        for tb_ in timed:
            tb_.timing(1)
        barrier(ws)
        prof = a.profile_window and method == methods[0] and not host
        if prof:
            torch.cuda.profiler.start()
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            reps = step(method, rho, hbuf)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        if prof:
            torch.cuda.profiler.stop()
        barrier(ws)
        phs = [tb_.timing(0) for tb_ in timed]
        ph = {k: sum(p_[k] for p_ in phs) for k in phs[0]}
        sweep_ms, launches, units = ph["sweep_ms"], ph["sweep_launches"], ph["sweep_units"]
        n_launch = rte.launch_count() - launches0
        got = (hbuf.numpy() if host else rho.cpu().numpy())
        err = np.abs(got - ref_np).max(1) / np.abs(ref_np).max(1)
        resid = residual_stats(rte, batch, rho, torch)   # untimed check of the last step's results
        return dict(times=np.array(times), reps=reps, err=err, sweep_ms=sweep_ms,
                    sweep_launches=launches, sweep_units=units, launches=n_launch, phases=ph,
                    resid=resid)

    results = {}
    clocks = ClockSampler(dev)
    clocks.start()
    for m in methods:
        results[m] = measure(m, a.steps, a.warmup)
    peaks = measured_peaks(rte, dev)
    clk = clocks.stop()
    e2e = measure("romsad", max(2, a.steps // 2), 1, host=True)

    def summary(r):
        ok = int(np.sum(r["err"] <= 1e-6))
        ms = float(np.mean(r["times"]))
        ns = [x["n_sweep"] for x in r["reps"]]
        return dict(ms_per_step=ms, solves_per_s=ok / (ms / 1e3), solves_ok=ok, batch=B,
                    err_max=float(r["err"].max()), n_sweep_mean=float(np.mean(ns)),
                    n_romsa_mean=float(np.mean([x["n_romsa"] for x in r["reps"]])),
                    n_dsa_mean=float(np.mean([x["n_dsa"] for x in r["reps"]])),
                    dsa_iters_mean=float(np.mean([x["dsa_iters"] for x in r["reps"]])),
                    n_sweep32_mean=float(np.mean([x["n_sweep32"] for x in r["reps"]])),
                    sweep_share=r["sweep_ms"] / float(np.sum(r["times"])),
                    phase_share={k: r["phases"][k + "_ms"] / float(np.sum(r["times"]))
                                 for k in ("sweep", "sweep32", "sweepff", "dsa", "rom", "setup")},
                    sweep_tflops=(r["sweep_units"] * FLOP_PER_CELL_DIR / (r["sweep_ms"] / 1e3) / 1e12
                                  if r["sweep_ms"] > 0 else None),
                    sweep32_tflops=(r["phases"]["sweep32_units"] * FLOP_PER_CELL_DIR /
                                    (r["phases"]["sweep32_ms"] / 1e3) / 1e12
                                    if r["phases"]["sweep32_ms"] > 0 else None),
                    # the float-float sweep's rate in the FP64 sweep's FLOPs (each of its FP64
                    # operations costs ~15 FP32 operations)
                    sweepff_tflops=(r["phases"]["sweepff_units"] * FLOP_PER_CELL_DIR /
                                    (r["phases"]["sweepff_ms"] / 1e3) / 1e12
                                    if r["phases"]["sweepff_ms"] > 0 else None),
                    p50_ms=float(np.percentile(r["times"], 50)),
                    p99_ms=float(np.percentile(r["times"], 99)), **r["resid"])

    summ = {m: summary(r) for m, r in results.items()}
    for v in summ.values():
        v["sweep_frac_fp64"] = v["sweep_tflops"] / peaks["fp64"] if v["sweep_tflops"] else None
        v["sweep32_frac_fp32"] = (v["sweep32_tflops"] / peaks["fp32"]
                                  if v["sweep32_tflops"] and peaks["fp32"] else None)
    head = results["romsad"]
    t_local = float(np.sum(head["times"])) / 1e3
    value = job_throughput(ws, float(summ["romsad"]["solves_ok"] * a.steps), t_local)
    # roofline of the dominant kernel (the sweep), from its CUDA-event time inside the timed region
    flops = head["sweep_units"] * FLOP_PER_CELL_DIR
    achieved = flops / (head["sweep_ms"] / 1e3) / 1e12
    sweep_cells = head["sweep_units"] / disc.n_dirs
    sweep_gbs = sweep_cells * BYTES_PER_CELL_SWEEP / (head["sweep_ms"] / 1e3) / 1e9
    traffic = None
    if (NCU_TRAFFIC["sha1"] == sweep_source_sha1() and (B, a.n, a.angles) ==
            (NCU_TRAFFIC["batch"], NCU_TRAFFIC["n"], NCU_TRAFFIC["angles"]) and a.dpw <= 0):
        traffic = NCU_TRAFFIC["bytes_per_launch"]
    e2e_ms = float(np.mean(e2e["times"]))
    e2e_ok = int(np.sum(e2e["err"] <= 1e-6))
    h2d = 8 * (2 * B * train.n_mat + B * train.n_cells + 4 * B)
    d2h = 8 * B * n_dof
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": float(np.mean(head["times"])),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded lattice instances; no dataset)",
        "config": {"workload": f"lattice{a.n}x{a.n}_CL({nphi},{nvz})_ROMSAD", "mesh": f"{a.n}x{a.n}",
                   "angles": a.angles, "distinct_directions": disc.n_dirs, "global_batch": B * ws,
                   "n_train": a.ntrain, "rank": a.rank, "window": 3, "theta": 5,
                   "eps_romsad": eps_romsad, "stop": f"relative change < {a.eps:g}",
                   "dsa": (f"{a.dsa_vcycles} FP32 multigrid V-cycles, {a.dsa_nu} red-black "
                           "smoothing sweeps per level" if a.dsa_rtol == 0 else
                           f"FGMRES rtol {a.dsa_rtol}"), "error_target": 1e-6,
                   "dirs_per_warp": (a.dpw if a.dpw > 0 else
                                     "measured per running count (count, directions per warp, "
                                     f"warps per direction group) {tuned}" if tuned else
                                     "occupancy rule per launch"),
                   "l2": "256 MB buffer written between timed steps",
                   "parallelism": "instances sharded across ranks, no collective"},
        "roofline": {"bound": "alu", "kernel": "sweep2d_kernel (FP64 DFMA)", "achieved": achieved,
                     "peak": peaks["fp64"], "unit": "TFLOP/s", "frac": achieved / peaks["fp64"],
                     "peak_source": "FP64 " + peaks["source"], "fp32_peak": peaks["fp32"],
                     "traffic": traffic, "launches": head["sweep_launches"],
                     "avg_launch_ms": head["sweep_ms"] / max(head["sweep_launches"], 1)},
        "sweep_gbs": sweep_gbs,
        "e2e": {"value": e2e_ok / (e2e_ms / 1e3), "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": head["launches"],
        "clocks": clk,
        "latency_ms": {"p50": summ["romsad"]["p50_ms"], "p99": summ["romsad"]["p99_ms"],
                       "note": "per batch of instances solved together"},
        "methods": summ,
        "r_inf": {"mean": summ["romsad"]["r_inf_mean"], "max": summ["romsad"]["r_inf_max"],
                  "note": "||(I - L) rho - b-bar||_inf of the ROMSAD results (absolute), one FP64 "
                          "sweep each, untimed"},
        "offline_s": offline_s,
        "rom": {"r_p": rom_p.r, "r_c": rom_c.r, "eps_pod_c": rom_c.eps_pod,
                "eps_pod_c_romig_started": rom_ci.eps_pod if rom_ci else None},
    }
    # the comparison the metric names: ROMSAD (and the precision variant) against plain FP64 SI-DSA
    # on the same GPU, same instances, same error target
    if "si_dsa" in summ:
        sid = summ["si_dsa"]["solves_per_s"]
        line["si_dsa_solves_per_s"] = sid
        line["romsad_vs_si_dsa"] = summ["romsad"]["solves_per_s"] / sid
        for m in ("romsad_refine", "romsad_refine_ff"):
            if m in summ:
                line[m + "_solves_per_s"] = summ[m]["solves_per_s"]
                line[m + "_vs_si_dsa"] = summ[m]["solves_per_s"] / sid
    return line, dict(n_sweep=summ["romsad"]["n_sweep_mean"], n_dsa=summ["romsad"]["n_dsa_mean"],
                      n_romsa=summ["romsad"]["n_romsa_mean"], n=a.n, angles=a.angles)


# ---- mixed-size batched workload and the serving loop ----------------------------------------

def build_bucket_rom(rte, inputs, side, angles, ntrain, rank, dev):
    """Offline stage of one (mesh side, angles) bucket: ntrain lattice training instances,
    SI-DSA to 1e-12, POD ranks `rank` (untimed)."""
    train = inputs.lattice(side, angles, [inputs.TRAIN_SEED0 + k for k in range(ntrain)], 4)
    disc = rte.Disc(train, device=dev)
    tb = rte.Batch(disc, train.batch)
    tb.set_params(train)
    rom_p, rom_c = rte.Rom.build(tb, eps_train=1e-12, window=3, rank_p=rank, rank_c=rank,
                                 max_iter=500, dsa_rtol=1e-8)
    tb.close()
    return disc, rom_p, rom_c, 0.1 * max(1e-12, rom_c.eps_pod)


def run_mixed(a, ws, rank, local):
    """Batched parametric solves of uneven sizes: a.instances lattice instances, mesh side from
    {64,96,128,192} and angles from {32,64,128}; one ROM per (side, angles) bucket.  A step sets
    every instance's parameters and solves all buckets together with rte_solve_many (one stream
    per bucket, one host thread relaunching whichever bucket has its stop-test norms back)."""
    import torch

    import __graft_entry__
    from paper_2402_10488_gb300 import inputs, rte

    __graft_entry__.build()
    torch.cuda.set_device(local)
    spec = inputs.mixed_batch_spec(a.instances, seed=inputs.BATCH_SEED + rank)
    keys = sorted({(s_, n_) for s_, n_, _ in spec})
    t0 = time.time()
    B = []
    for side, ang in keys:
        disc, rp, rc, eps_rs = build_bucket_rom(rte, inputs, side, ang, a.ntrain, a.rank, local)
        mu = np.array([m for s_, n_, m in spec if (s_, n_) == (side, ang)])
        prob = inputs.lattice_from_params(side, ang // 4, 4, mu)
        bt = rte.Batch(disc, prob.batch)
        bt.set_params(prob)
        B.append(dict(key=(side, ang), disc=disc, rom_p=rp, rom_c=rc, eps_romsad=eps_rs,
                      prob=prob, batch=bt, stream=torch.cuda.Stream(),
                      par=[torch.tensor(x, dtype=torch.float64, device="cuda")
                           for x in (prob.sigma_t, prob.sigma_s, prob.source, prob.inflow)],
                      rho=torch.zeros((prob.batch, disc.n_dof), dtype=torch.float64, device="cuda")))
    offline_s = time.time() - t0
    # tightly converged references (untimed)
    refs = []
    for k in B:
        r = torch.zeros_like(k["rho"])
        k["batch"].solve(r, 1e-13, sa=rte.SA_DSA, rel=True, max_iter=400, dsa_rtol=1e-3)
        refs.append(r.cpu().numpy())
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    eps = a.kappa * 1e-6

    def opts_for(method, k):
        kw = dict(rel=True, max_iter=400, dsa_rtol=a.dsa_rtol,
                  dsa_max_it=a.dsa_vcycles if a.dsa_rtol == 0 else 100)
        if method == "si_dsa":
            return rte.solve_opts(eps, rte.SA_DSA, **kw), None
        return (rte.solve_opts(eps, rte.SA_ROMSAD, theta=5, eps_romsad=k["eps_romsad"],
                               **precision_kw(method, a), **kw), k["rom_c"])

    def step(method):
        for k in B:
            k["batch"].set_params_device(*k["par"])
            k["rho"].zero_()
        torch.cuda.synchronize()
        oo = [opts_for(method, k) for k in B]
        reps, st = rte.solve_many([k["batch"] for k in B], [k["rho"] for k in B],
                                  [o for o, _ in oo], roms=[r for _, r in oo],
                                  streams=[k["stream"] for k in B], lockstep=lockstep(method))
        return reps

    def lockstep(method):
        return a.mixed_exec == "lockstep" and method in ("romsad", "si_dsa")

    methods = [m for m in a.methods.split(",")
               if m in ("romsad", "si_dsa", "romsad_mixed", "romsad_refine")]
    results = {}
    clocks = ClockSampler(local)
    clocks.start()
    for m in methods:
        for _ in range(a.warmup):
            step(m)
        for k in B:
            k["batch"].timing(1)
        launches0 = rte.launch_count()
        times = []
        barrier(ws)
        for _ in range(a.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            reps = step(m)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        barrier(ws)
        n_launch = rte.launch_count() - launches0
        units = sum(k["batch"].timing(0)["sweep_units"] for k in B)
        err = np.concatenate([np.abs(k["rho"].cpu().numpy() - refs[i]).max(1) /
                              np.abs(refs[i]).max(1) for i, k in enumerate(B)])
        ns = np.concatenate([[x["n_sweep"] for x in rr] for rr in reps])
        ms = float(np.mean(times))
        results[m] = dict(exec="lockstep" if lockstep(m) else "streams",
                          ms_per_step=ms, solves_ok=int(np.sum(err <= 1e-6)),
                          solves_per_s=float(np.sum(err <= 1e-6)) / (ms / 1e3),
                          err_max=float(err.max()), n_sweep_mean=float(ns.mean()),
                          launches_per_step=n_launch / a.steps,
                          sweep_tflops_whole_step=units / a.steps * FLOP_PER_CELL_DIR / (ms / 1e3) / 1e12,
                          times=times)
    peaks = measured_peaks(rte, local)
    clk = clocks.stop()
    head = results[methods[0]]
    value = job_throughput(ws, float(head["solves_ok"] * a.steps), float(np.sum(head["times"])) / 1e3)
    for r in results.values():
        r.pop("times")
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded lattice instances; no dataset)",
        "config": {"workload": f"mixed{a.instances}_lattice_sides64-192_angles32-128_{methods[0]}",
                   "buckets": [f"{s_}x{s_}_CL({n_ // 4},4):{k['prob'].batch}"
                               for (s_, n_), k in zip(keys, B)],
                   "global_batch": a.instances * ws, "n_train": a.ntrain, "rank": a.rank,
                   "stop": f"relative change < {eps:g}", "error_target": 1e-6,
                   "l2": "256 MB buffer written between timed steps",
                   "execution": ("FP64 methods: rte_solve_lockstep, one work-queue sweep launch over "
                                 "every bucket per iteration; precision variants: rte_solve_many, one "
                                 "stream per bucket" if a.mixed_exec == "lockstep" else
                                 "rte_solve_many: one stream per bucket, event-driven relaunch"),
                   "parallelism": "instances sharded across ranks, no collective"},
        "roofline": {"bound": "alu", "kernel": "sweep2d_kernel (FP64 DFMA), whole step",
                     "achieved": head["sweep_tflops_whole_step"], "peak": peaks["fp64"],
                     "unit": "TFLOP/s", "frac": head["sweep_tflops_whole_step"] / peaks["fp64"],
                     "peak_source": "FP64 " + peaks["source"],
                     "traffic": None,
                     "note": "sweep FLOPs of all buckets over the whole step time (streams overlap)"},
        "gpu_launches": int(head["launches_per_step"] * a.steps),
        "clocks": clk, "methods": results, "offline_s": offline_s,
    }
    return line


def run_serving(a, ws, rank, local):
    """Serving: a Poisson stream of lattice solve requests over 20 (mesh side, angles) buckets,
    each with its own ROM and a slot batch sized by device memory, through the library's
    continuous-batching loop (rte_server_*).  Reports completed solves/s and p50/p99 latency
    (submit to result in host memory) for ROMSAD and, on the same stream, plain SI-DSA."""
    import torch

    import __graft_entry__
    from paper_2402_10488_gb300 import inputs, rte

    __graft_entry__.build()
    torch.cuda.set_device(local)
    keys = [(s_, n_) for s_ in inputs.MESH_SIDES_SERVE for n_ in inputs.ANGLES_SERVE]
    t0 = time.time()
    buckets = {}
    for side, ang in keys:
        disc, rp, rc, eps_rs = build_bucket_rom(rte, inputs, side, ang, a.ntrain, a.rank, local)
        one = inputs.lattice_test(side, ang, 1)
        probe = rte.Batch(disc, 1)
        probe.set_params(one)
        per_slot = probe.info()["bytes"]
        probe.close()
        slots = int(max(1, min(a.max_slots, a.mem_gb * 2**30 / len(keys) / per_slot)))
        buckets[(side, ang)] = dict(disc=disc, rom_c=rc, rom_p=rp, eps_romsad=eps_rs, slots=slots,
                                    slot_bytes=per_slot)
    offline_s = time.time() - t0
    reqs = inputs.serving_requests(a.requests, a.rate, seed=inputs.SERVE_SEED + rank)

    def serve(method, stream_reqs):
        srv = rte.Server(local)
        ids = {}
        keep = []
        for key in keys:
            b = buckets[key]
            bt = rte.Batch(b["disc"], b["slots"])
            bt.set_params(inputs.lattice_test(key[0], key[1], b["slots"]))  # builds the hierarchy
            kw = dict(rel=True, max_iter=400, dsa_rtol=a.dsa_rtol,
                      dsa_max_it=a.dsa_vcycles if a.dsa_rtol == 0 else 100)
            if method == "si_dsa":
                ids[key] = srv.add_bucket(bt, None, None, sa=rte.SA_DSA, **kw)
            else:
                ids[key] = srv.add_bucket(bt, None, b["rom_c"], sa=rte.SA_ROMSAD, theta=5,
                                          eps_romsad=b["eps_romsad"], **precision_kw(method, a),
                                          **kw)
            keep.append(bt)
        srv.start()
        # warm-up: one request per bucket
        warm = []
        for key in keys:
            p = inputs.lattice_test(key[0], key[1], 1, first=900)
            warm.append(srv.submit(ids[key], p.sigma_t[0], p.sigma_s[0], p.source[0], p.inflow[0], 1e-6))
        for t in warm:
            srv.wait(t, timeout=600.0, want_rho=False)
        launches0 = rte.launch_count()
        st0 = srv.stats()
        tickets = []
        start = time.perf_counter()
        for t_arr, side, ang, mu, tol in stream_reqs:
            now = time.perf_counter() - start
            if t_arr > now:
                time.sleep(t_arr - now)
            p = inputs.lattice_from_params(side, ang // 4, 4, mu[None])
            tickets.append(srv.submit(ids[(side, ang)], p.sigma_t[0], p.sigma_s[0], p.source[0],
                                      p.inflow[0], a.kappa * tol))
        out = [srv.wait(t, timeout=1800.0) for t in tickets]
        st1 = srv.stats()
        n_launch = rte.launch_count() - launches0
        srv.close()
        for bt in keep:
            bt.close()
        return out, st0, st1, n_launch

    methods = [m for m in a.methods.split(",")
               if m in ("romsad", "si_dsa", "romsad_mixed", "romsad_refine")]
    results = {}
    clocks = ClockSampler(local)
    clocks.start()
    raw = {}
    for m in methods:
        out, st0, st1, n_launch = serve(m, reqs)
        raw[m] = out
        lat = np.array([r["t_done"] - r["t_submit"] for _, r in out]) * 1e3
        t_first = min(r["t_submit"] for _, r in out)
        t_last = max(r["t_done"] for _, r in out)
        ok = [r["status"] == 0 and r["converged"] for _, r in out]  # stop test met (error: sample)
        results[m] = dict(solves_per_s=float(np.sum(ok)) / (t_last - t_first),
                          completed=len(out), converged=int(np.sum(ok)),
                          p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                          wall_s=t_last - t_first, sweep_launches=st1["launches"] - st0["launches"],
                          max_queue=st1["max_queue"], gpu_launches=n_launch,
                          n_sweep_mean=float(np.mean([r["n_sweep"] for _, r in out])))
    clk = clocks.stop()
    head = methods[0]
    # accuracy of every request: each bucket's requests re-solved tightly (SI-DSA to a relative
    # change of 1e-13) in batches, untimed, and every method's result compared with them
    errs = {m: [] for m in methods}
    by_bucket = {}
    for k, (t_arr, side, ang, mu, tol) in enumerate(reqs):
        by_bucket.setdefault((side, ang), []).append(k)
    for key, ks in by_bucket.items():
        step_ = max(1, min(64, buckets[key]["slots"]))   # the bucket's slot count fits in memory
        for i0 in range(0, len(ks), step_):
            chunk = ks[i0:i0 + step_]
            p = inputs.lattice_from_params(key[0], key[1] // 4, 4, np.stack([reqs[k][3] for k in chunk]))
            bt = rte.Batch(buckets[key]["disc"], len(chunk))
            bt.set_params(p)
            ref = torch.zeros((len(chunk), p.n_dof), dtype=torch.float64, device="cuda")
            bt.solve(ref, 1e-13, sa=rte.SA_DSA, rel=True, max_iter=400, dsa_rtol=1e-3)
            ref_np = ref.cpu().numpy()
            bt.close()
            for j, k in enumerate(chunk):
                scale = np.abs(ref_np[j]).max()
                for m in methods:
                    errs[m].append((reqs[k][4], float(np.abs(raw[m][k][0] - ref_np[j]).max() / scale)))

    def sample_errors(m):
        e = errs[m]
        out = {"n": len(e), "note": "every request against a tight SI-DSA solve of its parameters"}
        for tol in (1e-6, 1e-8):
            et = [x for t, x in e if t == tol]
            out[f"max_rel_err_tol_{tol:g}"] = max(et or [0.0])
            out[f"within_tol_{tol:g}"] = int(sum(x <= tol for x in et))
            out[f"requests_tol_{tol:g}"] = len(et)
        return out

    for m in methods:
        results[m]["sample_errors"] = sample_errors(m)
    hr = results[head]
    line = {
        "metric": METRIC, "value": hr["solves_per_s"], "unit": "solves/s", "n_gpus": ws,
        "steps": 1, "warmup": 1, "ms_per_step": hr["wall_s"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Poisson request stream of lattice instances; no dataset)",
        "config": {"workload": f"serving_poisson{a.rate:g}_sides64-256_angles32-256_{head}",
                   "requests": a.requests, "rate_per_s": a.rate, "tolerances": [1e-6, 1e-8],
                   "stop": f"relative change < {a.kappa:g} x the request's tolerance",
                   "buckets": {f"{k[0]}x{k[0]}_CL({k[1] // 4},4)": buckets[k]["slots"] for k in keys},
                   "slot_memory_gb": a.mem_gb, "n_train": a.ntrain, "rank": a.rank,
                   "parallelism": "one GPU, one worker thread, one stream per bucket"},
        "latency_ms": {"p50": hr["p50_ms"], "p99": hr["p99_ms"],
                       "note": "per request, submit to result in host memory, queueing included"},
        "gpu_launches": hr["gpu_launches"], "clocks": clk, "methods": results,
        "sample_errors": hr["sample_errors"],
        "offline_s": offline_s,
    }
    return line


# ---- the paper's own 2D test problems -------------------------------------------------------

# n_sweep, T_rel and reduced dimensions printed in the paper: Tab. "Results for the problem with
# homogeneous medium" (Sec. 4.2.1) and Tab. "Results for the pin-cell problem" (Sec. 4.2.3);
# Matlab on the paper's hardware, averages over its own 10 random test parameters.
PAPER_TABLES = {
    "homogeneous": {"n_sweep": {"DSA": 14.6, "ROMIG": 3.0, "ROMSA": 2.9, "ROMSAD": 2.9,
                                "PGMRES": 11.0, "PGMRES-ROMIG": 4.8},
                    "T_rel": {"DSA": 1.0, "ROMIG": 0.19512, "ROMSA": 0.16578, "ROMSAD": 0.17853,
                              "PGMRES": 0.78778, "PGMRES-ROMIG": 0.33966},
                    "r_p": 5, "r_c": 14},
    "pin_cell": {"n_sweep": {"DSA": 39.3, "ROMIG": 5.3, "ROMSAD": 4.0, "PGMRES": 16.2,
                             "PGMRES-ROMIG": 5.6},
                 "T_rel": {"DSA": 1.0, "ROMIG": 0.13143, "ROMSAD": 0.09336, "PGMRES": 0.40070,
                           "PGMRES-ROMIG": 0.13781},
                 "r_p": 21, "r_c": 59},
    # Tab. "Results for the variable scattering problem" (Sec. 4.2.4)
    "variable_scattering": {"n_sweep": {"DSA": 17.0, "ROMIG": 2.6, "ROMSAD": 4.2, "PGMRES": 12.0,
                                        "PGMRES-ROMIG": 3.8},
                            "T_rel": {"DSA": 1.0, "ROMIG": 0.14357, "ROMSAD": 0.19879,
                                      "PGMRES": 0.68760, "PGMRES-ROMIG": 0.20627},
                            "r_p": 9, "r_c": 18},
}


def run_paper(a, ws, rank, local):
    """The paper's homogeneous-medium (Sec. 4.2.1) and pin-cell (Sec. 4.2.3) problems on the GPU:
    80x80 mesh, CL(30,6), the paper's training sets, tolerances, eps_POD = 1e-9, window 3 and
    theta; 10 seeded random test parameters.  Every method solves the 10 test instances as one
    batch from its own start; n_sweep, the GPU time relative to SI-DSA, the residual
    ||(I - L) rho - b-bar||_inf and the reduced dimensions are reported next to the paper's."""
    import torch

    import __graft_entry__
    from paper_2402_10488_gb300 import inputs, rte

    __graft_entry__.build()
    torch.cuda.set_device(local)
    setups = {
        "homogeneous": dict(make=inputs.homogeneous_medium, train=inputs.homogeneous_train(),
                            test=inputs.homogeneous_test(10, seed=inputs.TEST_SEED0 + rank),
                            eps=1e-12, gmres_rtol=1e-11, theta=3,
                            methods=["DSA", "ROMIG", "ROMSA", "ROMSAD", "PGMRES", "PGMRES-ROMIG"]),
        "pin_cell": dict(make=inputs.pin_cell, train=inputs.pin_cell_train(),
                         test=inputs.pin_cell_test(10, seed=inputs.TEST_SEED0 + rank),
                         eps=1e-11, gmres_rtol=2.5e-11, theta=5,
                         methods=["DSA", "ROMIG", "ROMSAD", "PGMRES", "PGMRES-ROMIG"]),
        "variable_scattering": dict(make=inputs.variable_scattering,
                                    train=inputs.variable_scattering_train(),
                                    test=inputs.variable_scattering_test(10, seed=inputs.TEST_SEED0 + rank),
                                    eps=1e-12, gmres_rtol=2.5e-11, theta=5, eps_pod=1e-11,
                                    methods=["DSA", "ROMIG", "ROMSAD", "PGMRES", "PGMRES-ROMIG"]),
    }
    dsa = (dict(dsa_rtol=1e-8, dsa_max_it=200) if a.paper_dsa == "fgmres" else
           dict(dsa_rtol=0.0, dsa_max_it=a.dsa_vcycles))
    out = {}
    stream = torch.cuda.current_stream()
    head_value = None
    for name, S in setups.items():
        train, test = S["make"](S["train"]), S["make"](S["test"])
        disc = rte.Disc(train, device=local)
        tb = rte.Batch(disc, train.batch)
        tb.set_params(train)
        t0 = time.time()
        eps_pod = S.get("eps_pod", 1e-9)
        rom_p, rom_c = rte.Rom.build(tb, eps_train=S["eps"], window=3, rank_p=0, rank_c=0,
                                     eps_pod=eps_pod, max_iter=2000, dsa_rtol=1e-10)
        offline_s = time.time() - t0
        tb.close()
        eps_rs = 0.1 * max(S["eps"], eps_pod)  # eta max(eps_SISA, eps_POD), eps_POD the truncation tolerance
        batch = rte.Batch(disc, test.batch)
        batch.set_params(test)
        rho = torch.zeros((test.batch, disc.n_dof), dtype=torch.float64, device="cuda")
        chk = torch.empty_like(rho)

        def run(m):
            rho.zero_()
            if m in ("ROMIG", "PGMRES-ROMIG"):
                rom_p.initial_guess(batch, rho)
            if m in ("PGMRES", "PGMRES-ROMIG"):
                reps, _ = batch.pgmres(rho, S["gmres_rtol"], restart=25, max_iter=500,
                                       zero_start=m == "PGMRES", **dsa)
                return reps
            sa = {"DSA": rte.SA_DSA, "ROMIG": rte.SA_DSA, "ROMSA": rte.SA_ROMSA,
                  "ROMSAD": rte.SA_ROMSAD}[m]
            reps, _, _ = batch.solve(rho, S["eps"], sa=sa, rel=False, max_iter=2000,
                                     rom_c=rom_c if sa in (rte.SA_ROMSA, rte.SA_ROMSAD) else None,
                                     theta=S["theta"], eps_romsad=eps_rs, **dsa)
            return reps

        res = {}
        for m in S["methods"]:
            for _ in range(max(1, a.warmup)):
                run(m)
            times = []
            for _ in range(max(1, a.steps)):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                reps = run(m)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            batch.sweep(rho, chk)
            torch.cuda.synchronize()
            resid = (rho - chk).abs().amax(1).cpu().numpy()
            res[m] = dict(n_sweep=float(np.mean([r["n_sweep"] for r in reps])),
                          converged=int(sum(r["converged"] for r in reps)),
                          ms=float(np.mean(times)), residual_inf=float(np.mean(resid)),
                          n_romsa=float(np.mean([r["n_romsa"] for r in reps])))
        for m in res:
            res[m]["T_rel"] = res[m]["ms"] / res["DSA"]["ms"]
        out[name] = dict(ours=res, paper=PAPER_TABLES[name], r_p=rom_p.r, r_c=rom_c.r,
                         offline_s=offline_s, eps_pod_c=rom_c.eps_pod)
        if name == "pin_cell":
            head_value = test.batch / (res["ROMSAD"]["ms"] / 1e3)
    line = {
        "metric": METRIC, "value": head_value, "unit": "solves/s", "n_gpus": ws,
        "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": out["pin_cell"]["ours"]["ROMSAD"]["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (the paper's parametric problems, seeded test parameters)",
        "config": {"workload": "paper_2d_homogeneous_pin_cell_variable_scattering_80x80_CL(30,6)",
                   "dsa": (f"FGMRES rtol {dsa['dsa_rtol']:g} (the paper: AMG)" if dsa["dsa_rtol"] > 0
                           else f"{dsa['dsa_max_it']} FP32 multigrid V-cycles (the paper: AMG)"),
                   "value": "ROMSAD solves/s on the 10 pin-cell test instances (one batch)"},
        "problems": out,
    }
    return line


# n_sweep and reduced dimensions printed in the paper for the 1D cross-regime problem (Sec. 4.1.1:
# Tab. of reduced dimensions and Tab. "Results for the cross-regime problem", eps_SISA = 1e-11).
PAPER_TABLES_1D = {
    1e-9: {"r_p": 6, "r_c": {1: 6, 3: 15},
           "n_sweep": {"DSA": 15, "ROMIG": 9, "ROMSA-1": 23.75, "ROMSAD-1,3": 6.55,
                       "ROMSA-3": 42.25, "ROMSAD-3,3": 6.85}},
    1e-10: {"r_p": 6, "r_c": {1: 6, 3: 18},
            "n_sweep": {"DSA": 15, "ROMIG": 9, "ROMSA-1": 23.75, "ROMSAD-1,3": 6.6,
                        "ROMSA-3": 12.05, "ROMSAD-3,3": 5.8}},
    1e-11: {"r_p": 7, "r_c": {1: 7, 3: 21},
            "n_sweep": {"DSA": 15, "ROMIG": 9, "ROMSA-1": 7.05, "ROMSAD-1,3": 5.65,
                        "ROMSA-3": 4.55, "ROMSAD-3,3": 4.5}},
}


# The two-material problem (Sec. 4.1.2: Tab. "Results for the two-material problem"; ROMSAD with
# theta = 1, 3, 5 performs identically there, window 3 and 5 too).
PAPER_TABLES_1D_TWO = {
    1e-6: {"r_p": 21, "r_c": {3: 49, 5: 54}, "n_sweep": {"DSA": 14.6, "ROMIG": 8.1, "ROMSAD-3,3": 8.9,
                                                          "ROMSAD-5,3": 9.05}},
    1e-9: {"r_p": 44, "r_c": {3: 101, 5: 120}, "n_sweep": {"DSA": 14.6, "ROMIG": 4.2, "ROMSAD-3,3": 5.35,
                                                            "ROMSAD-5,3": 5.35}},
    1e-10: {"r_p": 53, "r_c": {3: 123, 5: 147}, "n_sweep": {"DSA": 14.6, "ROMIG": 3.35, "ROMSAD-3,3": 4.25,
                                                             "ROMSAD-5,3": 4.25}},
}


def run_two_material(rte, inputs, torch, local, rank):
    """Sec. 4.1.2: two-material slab on the paper's non-uniform mesh, inflow 5 at x = 0, 451
    training pairs, eps_SISA = 1e-12, eps_POD in {1e-6, 1e-9, 1e-10}, windows 3 and 5, theta 3;
    20 seeded random test pairs."""
    train = inputs.two_material(inputs.two_material_train())
    test = inputs.two_material(inputs.two_material_test(20, seed=inputs.TEST_SEED0 + rank))
    disc = rte.Disc(train, device=local)
    tb = rte.Batch(disc, train.batch)
    tb.set_params(train)
    batch = rte.Batch(disc, test.batch)
    batch.set_params(test)
    rho = torch.zeros((test.batch, disc.n_dof), dtype=torch.float64, device="cuda")
    chk = torch.empty_like(rho)
    eps = 1e-12

    def run(sa, rom_c=None, rom_p=None, theta=0, eps_rs=0.0):
        rho.zero_()
        if rom_p is not None:
            rom_p.initial_guess(batch, rho)
        reps, _, _ = batch.solve(rho, eps, sa=sa, rel=False, max_iter=2000, rom_c=rom_c,
                                 theta=theta, eps_romsad=eps_rs)
        batch.sweep(rho, chk)
        torch.cuda.synchronize()
        return dict(n_sweep=float(np.mean([r["n_sweep"] for r in reps])),
                    converged=int(sum(r["converged"] for r in reps)),
                    residual_inf=float((rho - chk).abs().amax(1).mean().item()))

    out = {}
    dsa = run(rte.SA_DSA)
    for eps_pod in (1e-6, 1e-9, 1e-10):
        res = {"DSA": dsa}
        ranks = {}
        t0 = time.time()
        for w in (3, 5):
            rom_p, rom_c = rte.Rom.build(tb, eps_train=eps, window=w, rank_p=0, rank_c=0,
                                         eps_pod=eps_pod, max_iter=2000, dsa_rtol=1e-10)
            ranks["r_p"] = rom_p.r
            ranks[f"r_c(w={w})"] = rom_c.r
            ranks[f"n_snap_c(w={w})"] = rom_c.n_snap
            if w == 3:
                res["ROMIG"] = run(rte.SA_DSA, rom_p=rom_p)
            res[f"ROMSAD-{w},3"] = run(rte.SA_ROMSAD, rom_c=rom_c, theta=3,
                                       eps_rs=0.1 * max(eps, eps_pod))
        out[f"{eps_pod:g}"] = dict(ours=res, ranks=ranks, paper=PAPER_TABLES_1D_TWO[eps_pod],
                                   offline_s=time.time() - t0)
    return out


def run_paper1d(a, ws, rank, local):
    """The paper's 1D cross-regime problem (Sec. 4.1.1) on the GPU: 400 cells on [0,10], S_16,
    41 training slopes, eps_SISA = 1e-11 (absolute), eps_POD in {1e-9, 1e-10, 1e-11}, windows 1
    and 3, theta = 3; 20 seeded random test slopes solved as one batch per method.  Reports
    n_sweep and the reduced dimensions next to the paper's tables.  sigma_s is linear inside each
    cell as in the paper (``--cellwise-sigma``: its cell averages instead)."""
    import torch

    import __graft_entry__
    from paper_2402_10488_gb300 import inputs, rte

    __graft_entry__.build()
    torch.cuda.set_device(local)
    lin = not a.cellwise_sigma
    train = inputs.cross_regime(inputs.cross_regime_train(), linear=lin)
    test = inputs.cross_regime(inputs.cross_regime_test(20, seed=inputs.TEST_SEED0 + rank), linear=lin)
    disc = rte.Disc(train, device=local)
    tb = rte.Batch(disc, train.batch)
    tb.set_params(train)
    batch = rte.Batch(disc, test.batch)
    batch.set_params(test)
    rho = torch.zeros((test.batch, disc.n_dof), dtype=torch.float64, device="cuda")
    chk = torch.empty_like(rho)
    eps = 1e-11
    out = {}
    t_all = time.time()

    def run(sa, rom_c=None, rom_p=None, theta=0, eps_rs=0.0):
        rho.zero_()
        if rom_p is not None:
            rom_p.initial_guess(batch, rho)
        reps, _, _ = batch.solve(rho, eps, sa=sa, rel=False, max_iter=2000, rom_c=rom_c,
                                 theta=theta, eps_romsad=eps_rs)
        batch.sweep(rho, chk)
        torch.cuda.synchronize()
        return dict(n_sweep=float(np.mean([r["n_sweep"] for r in reps])),
                    converged=int(sum(r["converged"] for r in reps)),
                    residual_inf=float((rho - chk).abs().amax(1).mean().item()))

    dsa = run(rte.SA_DSA)
    for eps_pod in (1e-9, 1e-10, 1e-11):
        res = {"DSA": dsa}
        ranks = {}
        for w in (1, 3):
            rom_p, rom_c = rte.Rom.build(tb, eps_train=eps, window=w, rank_p=0, rank_c=0,
                                         eps_pod=eps_pod, max_iter=2000, dsa_rtol=1e-10)
            eps_rs = 0.1 * max(eps, eps_pod)  # Eq. (romsad_parameters) with the truncation tolerance
            ranks["r_p"] = rom_p.r
            ranks[f"r_c(w={w})"] = rom_c.r
            if w == 1:
                res["ROMIG"] = run(rte.SA_DSA, rom_p=rom_p)
            res[f"ROMSA-{w}"] = run(rte.SA_ROMSA, rom_c=rom_c)
            res[f"ROMSAD-{w},3"] = run(rte.SA_ROMSAD, rom_c=rom_c, theta=3, eps_rs=eps_rs)
        out[f"{eps_pod:g}"] = dict(ours=res, ranks=ranks, paper=PAPER_TABLES_1D[eps_pod])
    line = {
        "metric": METRIC, "value": None, "unit": "solves/s", "n_gpus": ws, "steps": 1, "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (the paper's 1D cross-regime problem, seeded test slopes)",
        "config": {"workload": "paper_1d_cross_regime_400_S16" + ("_cellwise" if a.cellwise_sigma else ""),
                   "note": "sweep counts and reduced dimensions vs the paper; sigma_s " +
                           ("at its cell averages" if a.cellwise_sigma else "linear in each cell "
                            "as in the paper (the 401 cell edges are the materials)"),
                   "wall_s": time.time() - t_all},
        "eps_pod": out,
        "two_material": run_two_material(rte, inputs, torch, local, rank),
    }
    return line


# ---- CPU oracle (baseline leg and the reference arm) ------------------------------------------
#
# The oracle as it stands (plain numpy/scipy FP64: a sparse LU per direction, the 2D DSA as a direct
# sparse solve) runs one parametric instance per process, in a pool of worker processes over all
# host cores (one BLAS thread each).  Each process peaks at ~7 GB at the 128^2 CL(16,4) size (64
# direction factorizations and the DSA factorization), so the pool is also capped by free memory.

_ORACLE_ROM = None   # the correction ROM in each worker of the test pool (set by the initializer)


def oracle_workers():
    """Processes for the oracle pool: every host core, unless free memory allows fewer."""
    cores = os.cpu_count() or 1
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        by_mem = max(1, int((avail - 16 * 2**30) // (8 * 2**30)))
    except (ValueError, OSError, AttributeError):
        by_mem = cores
    return max(1, min(cores, by_mem))


class _OraclePool:
    """A spawn-context process pool whose workers use one BLAS thread each."""

    def __init__(self, workers, initializer=None, initargs=()):
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        self.saved = {k: os.environ.get(k) for k in keys + ("CUDA_VISIBLE_DEVICES",)}
        for k in keys:
            os.environ[k] = "1"
        os.environ["CUDA_VISIBLE_DEVICES"] = ""
        self.ex = ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"),
                                      initializer=initializer, initargs=initargs)

    def __enter__(self):
        return self.ex

    def __exit__(self, *exc):
        self.ex.shutdown(wait=True)
        for k, v in self.saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _oracle_train(args):
    """Training solves of a share of the training instances (SI-DSA from zero to eps_train,
    absolute): the converged angular fluxes and the window's correction snapshots."""
    n, angles, seeds, eps_train, window = args
    from oracle.rom import training_snapshots
    from paper_2402_10488_gb300 import inputs
    F, dF, n_conv, _ = training_snapshots(inputs.lattice(n, angles, seeds, 4), eps_train, window)
    return F, dF, n_conv


def _oracle_set_rom(rom):
    global _ORACLE_ROM
    _ORACLE_ROM = rom


def _oracle_romsad(args):
    """One complete oracle ROMSAD solve (Alg. 2) of one test instance from rho = 0: set-up of its
    transport operators and DSA system, then the iterations to the relative stop tolerance."""
    n, angles, seed, eps, theta, eps_romsad = args
    from oracle.dsa import ConsistentDSA
    from oracle.sisa import sisa
    from oracle.transport import Transport
    from paper_2402_10488_gb300 import inputs
    t0 = time.perf_counter()
    tr = Transport(inputs.lattice(n, angles, [seed], 4), 0)
    res = sisa(tr, np.zeros(tr.n_dof), eps, 400, "romsad", dsa=ConsistentDSA(tr), rom_c=_ORACLE_ROM,
               theta=theta, eps_romsad=eps_romsad, tol_mode="rel")
    return dict(seconds=time.perf_counter() - t0, n_sweep=res["n_sweep"],
                n_romsa=res["sa"].count("romsa"), n_dsa=res["sa"].count("dsa"),
                converged=bool(res["converged"]))


def _oracle_dsa_iterations(args):
    """The oracle's set-up of one test instance and n iterations of Alg. 1 with DSA corrections."""
    n, angles, seed, n_iter = args
    from oracle.dsa import ConsistentDSA
    from oracle.sisa import sisa
    from oracle.transport import Transport
    from paper_2402_10488_gb300 import inputs
    t0 = time.perf_counter()
    tr = Transport(inputs.lattice(n, angles, [seed], 4), 0)
    sisa(tr, np.zeros(tr.n_dof), 0.0, n_iter, "dsa", dsa=ConsistentDSA(tr))
    return time.perf_counter() - t0


def oracle_offline(a, workers):
    """The oracle's offline stage for the workload (untimed, as in the paper's T_rel): the training
    SI-DSA solves spread over the pool by instance, the correction snapshot matrix (window 3), its
    thin SVD truncated to the workload's rank, and the correction ROM's reduced operators."""
    from oracle.rom import POD, ReducedModel
    from oracle.transport import Transport
    from paper_2402_10488_gb300 import inputs
    seeds = [inputs.TRAIN_SEED0 + k for k in range(a.ntrain)]
    # one training instance per task: a worker then holds one instance's factorizations at a time
    with _OraclePool(min(workers, len(seeds))) as ex:
        parts = list(ex.map(_oracle_train, [(a.n, a.angles, [sd], 1e-12, 3) for sd in seeds]))
    dF = np.concatenate([p[1] for p in parts], 1)
    pod_c = POD(dF, rank=a.rank)
    del dF, parts
    rom_c = ReducedModel(pod_c.U, Transport(inputs.lattice(a.n, a.angles, seeds[:1], 4), 0))
    rom_c.U = None   # the online stage reads only U^rho, U^iso and the reduced operators
    return rom_c, 0.1 * max(1e-12, pod_c.eps_equiv)


def run_reference(a, ws, rank):
    """The reference arm: the CPU oracle, unmodified, on the workload.  Untimed: the oracle's own
    offline stage.  Then W warm-up and K timed steps, one step = one complete oracle ROMSAD solve of
    one test instance (set-up + Alg. 2 iterations with the oracle's own counts and ROM); the steps
    run concurrently, one process per core, and the timed region is the pool's wall time for the K
    steps, so ms_per_step = wall / K."""
    if rank != 0:
        return None
    from paper_2402_10488_gb300 import inputs
    workers = oracle_workers()
    t0 = time.time()
    rom_c, eps_romsad = oracle_offline(a, workers)
    offline_s = time.time() - t0
    K = max(1, a.steps)
    # every core solves in the timed region (max(K, cores) instances); the region is split evenly
    # into the K steps
    n_solves = max(K, workers)
    seeds = [inputs.TEST_SEED0 + (k % a.batch) for k in range(n_solves)]
    job = lambda sd: (a.n, a.angles, sd, a.eps, 5, eps_romsad)
    with _OraclePool(workers, initializer=_oracle_set_rom, initargs=(rom_c,)) as ex:
        if a.warmup > 0:   # untimed warm-up solves
            list(ex.map(_oracle_romsad, [job(seeds[k]) for k in range(min(a.warmup, workers))]))
        t1 = time.perf_counter()
        out = list(ex.map(_oracle_romsad, [job(sd) for sd in seeds]))
        wall = time.perf_counter() - t1
    ok = sum(r["converged"] for r in out)
    v = ok / wall
    used = min(workers, n_solves)
    line = {"metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": ws, "steps": K,
            "warmup": a.warmup, "ms_per_step": 1e3 * wall / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"lattice{a.n}x{a.n}_CL({a.angles // 4},4)_ROMSAD",
                       "global_batch": n_solves, "stop": f"relative change < {a.eps:g}",
                       "n_train": a.ntrain, "rank": a.rank},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": used, "kind": "oracle",
                             "sample": (f"{n_solves} complete oracle ROMSAD solves in the K = {K} "
                                        f"steps' timed region (test instances "
                                        f"{seeds[0] - inputs.TEST_SEED0}..{seeds[-1] - inputs.TEST_SEED0}, "
                                        f"set-up + Alg. 2 with the oracle's own ROM, rank {a.rank} "
                                        f"from {a.ntrain} training solves, offline {offline_s:.0f} s "
                                        f"untimed), {used} processes on {os.cpu_count()} cores"),
                             "n_sweep_mean": float(np.mean([r["n_sweep"] for r in out])),
                             "n_romsa_mean": float(np.mean([r["n_romsa"] for r in out])),
                             "n_dsa_mean": float(np.mean([r["n_dsa"] for r in out])),
                             "seconds_per_solve_mean": float(np.mean([r["seconds"] for r in out])),
                             "offline_s": offline_s},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def cpu_baseline_leg(a, counts):
    """The oracle beside the GPU arm, bounded so the default run stays within minutes: its
    ROMSAD solves need its own offline stage (~45 CPU-minutes at this size; the reference arm runs
    it), so this leg times the rest of a ROMSAD solve -- the set-up and n iterations of Alg. 1, n
    this run's mean ROMSAD sweep count, with DSA corrections (ROMSAD's single ROMSA correction is a
    small dense solve, far cheaper in the oracle than the DSA one it stands in for) -- on one test
    instance per process, all processes at once."""
    from paper_2402_10488_gb300 import inputs
    workers = oracle_workers()
    n_iter = max(1, int(round(counts["n_sweep"])))
    jobs = [(a.n, a.angles, inputs.TEST_SEED0 + k, n_iter) for k in range(workers)]
    with _OraclePool(workers) as ex:
        t0 = time.perf_counter()
        secs = list(ex.map(_oracle_dsa_iterations, jobs))
        wall = time.perf_counter() - t0
    return {"value": workers / wall, "unit": "solves/s", "cores": workers, "kind": "oracle",
            "sample": (f"{workers} test instances at once, one process per core: the oracle's set-up "
                       f"and {n_iter} iterations of Alg. 1 with DSA (this run's mean ROMSAD sweep "
                       f"count {counts['n_sweep']:.2f}; the oracle's offline stage is not part of it)"),
            "wall_s": wall, "seconds_per_instance_mean": float(np.mean(secs))}


def main():
    a = parse()
    ws, rank, local = dist_init()
    if a.impl == "reference":
        line = run_reference(a, ws, rank)
        if rank == 0 and line is not None:
            print(json.dumps(line), flush=True)
        return
    if a.workload != "lattice":
        line = {"mixed": run_mixed, "serving": run_serving, "paper": run_paper,
                "paper1d": run_paper1d}[a.workload](
            a, ws, rank, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    line, counts = run_ours(a, ws, rank, local)
    if rank == 0:
        if ws == 1 and not a.no_cpu_baseline:
            try:
                line["cpu_baseline"] = cpu_baseline_leg(a, counts)
            except Exception as e:  # the baseline leg must not hide the GPU result
                line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 0,
                                        "kind": "oracle", "sample": f"failed: {e}"[:300]}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
