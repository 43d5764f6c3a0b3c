"""Thin ctypes binding of the C ABI in include/rte.h (argument marshalling only).

Device arrays are torch CUDA tensors (float64, contiguous) passed by ``data_ptr()``; streams
default to torch's current stream.  Every computation runs in the CUDA library; if the compiled
library is missing, ``lib()`` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librte_gb300.so")

RTE_OK, RTE_EINVAL, RTE_ENOMEM, RTE_ENOCONV, RTE_ETIMEOUT, RTE_ECUDA, RTE_ESTATE = 0, -1, -2, -3, -4, -5, -6
SA_NONE, SA_DSA, SA_ROMSA, SA_ROMSAD = 0, 1, 2, 3
SMOOTHER_GLOBAL, SMOOTHER_TILED, SMOOTHER_BLOCKED = 0, 1, 2
FAULT_LIFT_NO_MMA = 1

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# exported symbol -> (restype, argtypes); mirrors include/rte.h
SIGNATURES = {
    "rte_version": (_I, []),
    "rte_last_error": (ctypes.c_char_p, []),
    "rte_counters": (_I, [_P]),
    "rte_batch_timing": (_I, [_P, _I, _P]),
    "rte_batch_tune": (_I, [_P, _I]),
    "rte_batch_autotune": (_I, [_P, _P, _P, _P]),
    "rte_disc_create": (_I, [_P, _I, _P]),
    "rte_disc_destroy": (_I, [_P]),
    "rte_disc_info": (_I, [_P, _P]),
    "rte_disc_quadrature": (_I, [_P, _P, _P]),
    "rte_batch_create": (_I, [_P, _I, _P]),
    "rte_batch_destroy": (_I, [_P]),
    "rte_batch_set_params": (_I, [_P, _P, _P, _P, _P]),
    "rte_batch_set_params_device": (_I, [_P, _P, _P, _P, _P, _P]),
    "rte_batch_directions": (_I, [_P, _P]),
    "rte_sweep": (_I, [_P, _P, _P, _P, _I, _P, _P]),
    "rte_sweep_static": (_I, [_P, _P, _P, _I, _P]),
    "rte_residual": (_I, [_P, _P, _P, _P, _P, _P]),
    "rte_fma_peak": (_I, [_I, _I, _P, _P]),
    "rte_sweep_f32": (_I, [_P, _P, _P, _P, _P]),
    "rte_sweep_ff": (_I, [_P, _P, _P, _P, _P]),
    "rte_change_norm": (_I, [_P, _P, _P, _P, _P]),
    "rte_dsa_correction": (_I, [_P, _P, _P, _D, _I, _P, _P, _P]),
    "rte_correction_source": (_I, [_P, _P, _P, _P, _P]),
    "rte_rom_build": (_I, [_P, _P, _P, _P, _P]),
    "rte_rom_destroy": (_I, [_P]),
    "rte_rom_info": (_I, [_P, _P, _P]),
    "rte_rom_initial_guess": (_I, [_P, _P, _P, _P, _P]),
    "rte_romsa_correction": (_I, [_P, _P, _P, _P, _P, _P]),
    "rte_solve": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "rte_batch_set_slots": (_I, [_P, _I, _P, _P, _P, _P, _P, _P]),
    "rte_batch_info": (_I, [_P, _P]),
    "rte_rom_save": (_I, [_P, ctypes.c_char_p]),
    "rte_rom_load": (_I, [_P, ctypes.c_char_p, _P]),
    "rte_solve_many": (_I, [_I, _P, _P, _P, _P, _P, _P]),
    "rte_solve_lockstep": (_I, [_I, _P, _P, _P, _P, _P, _P]),
    "rte_solve_interleaved": (_I, [_I, _P, _P, _P, _P, _P, _P]),
    "rte_batch_tuned": (_I, [_P, _P, _P]),
    "rte_server_create": (_I, [_I, _P]),
    "rte_server_add_bucket": (_I, [_P, _P, _P, _P, _P, _P]),
    "rte_server_start": (_I, [_P]),
    "rte_server_submit": (_I, [_P, _I, _P, _P, _P, _P, _D, _P]),
    "rte_server_wait": (_I, [_P, ctypes.c_uint64, _D, _P, _P]),
    "rte_server_stats": (_I, [_P, _P]),
    "rte_server_destroy": (_I, [_P]),
    "rte_pgmres": (_I, [_P, _P, _P, _P, _P]),
    "rte_batch_dsa_smoothing": (_I, [_P, _I]),
    "rte_batch_dsa_smoother": (_I, [_P, _I]),
    "rte_pod_workspace_bytes": (_I, [_I, _I, _I, _P]),
    "rte_pod_project_bf16": (_I, [_P, _I, _I, _P, _I, _P, _P, _P, _P]),
    "rte_pod_lift_bf16": (_I, [_P, _I, _I, _P, _I, _P, _P, _P, _P]),
    "rte_fault_inject": (_I, [_I]),
}


def pod_workspace(r, n, B):
    """A zeroed device workspace for pod_project_bf16 / pod_lift_bf16 (a torch uint8 tensor)."""
    import torch
    nb = np.zeros(1, np.int64)
    check(lib().rte_pod_workspace_bytes(int(r), int(n), int(B), nb.ctypes.data_as(_P)))
    return torch.zeros(int(nb[0]), dtype=torch.uint8, device="cuda")


def pod_project_bf16(U, X, out, work, active=None, stream=None):
    """out[b][i] = sum_e U[i][e] X[b][e] on the tensor cores (BF16 operands, FP32 sums)."""
    r, n = U.shape
    check(lib().rte_pod_project_bf16(_ptr(U), int(r), int(n), _ptr(X), int(X.shape[0]),
                                     _ptr(active), _ptr(out), _ptr(work), _stream(stream)))


def pod_lift_bf16(U, C, Y, work, active=None, stream=None):
    """Y[b][e] = sum_i U[i][e] C[b][i] on the tensor cores (BF16 operands, FP32 sums)."""
    r, n = U.shape
    check(lib().rte_pod_lift_bf16(_ptr(U), int(r), int(n), _ptr(C), int(C.shape[0]),
                                  _ptr(active), _ptr(Y), _ptr(work), _stream(stream)))


def fma_peak(kind="fp64", device=0, stream=None):
    """Measured FMA throughput of the device in TFLOP/s (rte_fma_peak): kind "fp64" or "fp32"."""
    out = ctypes.c_double()
    check(lib().rte_fma_peak(int(device), 0 if kind == "fp64" else 1, ctypes.byref(out),
                             _stream(stream)))
    return float(out.value)


def fault_inject(what):
    """One-shot injected fault for tests of the failure path (rte_fault_inject)."""
    check(lib().rte_fault_inject(int(what)))


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    out = np.zeros(1, np.int64)
    check(lib().rte_counters(out.ctypes.data_as(_P)))
    return int(out[0])


class RTEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"RTE status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load the compiled library (no fallback: raises when it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2402_10488_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status, allow=()):
    if status != RTE_OK and status not in allow:
        raise RTEError(status, lib().rte_last_error().decode())
    return status


class _DiscDesc(ctypes.Structure):
    _fields_ = [("dim", _I), ("nx", _I), ("ny", _I), ("x0", _D), ("x1", _D), ("y0", _D),
                ("y1", _D), ("n_phi", _I), ("n_vz", _I), ("n_mat", _I), ("mat_id", _P),
                ("dx", _P), ("mat_id_right", _P)]


class _RomOpts(ctypes.Structure):
    _fields_ = [("eps_train", _D), ("window", _I), ("rank_p", _I), ("rank_c", _I),
                ("eps_pod", _D), ("max_iter", _I), ("dsa_rtol", _D), ("correction_start", _I)]


class _SolveOpts(ctypes.Structure):
    _fields_ = [("eps", _D), ("rel", _I), ("max_iter", _I), ("sa", _I), ("theta", _I),
                ("eps_romsad", _D), ("dsa_rtol", _D), ("dsa_max_it", _I), ("schedule", _P),
                ("fp32_switch", _D), ("refine_kappa", _D), ("refine_inner", _I),
                ("rom_bf16", _I), ("gang_wait", _I), ("verify", _I), ("sa_history", _P),
                ("outer_ff", _I)]


class SolveReport(ctypes.Structure):
    _fields_ = [("n_sweep", _I), ("converged", _I), ("n_romsa", _I), ("n_dsa", _I),
                ("dsa_iters", _I), ("last_change", _D), ("rho_inf", _D), ("n_sweep32", _I),
                ("pad", _I), ("r_inf", _D), ("balance_cell", _D), ("balance", _D)]


class _GmresOpts(ctypes.Structure):
    _fields_ = [("rtol", _D), ("restart", _I), ("max_iter", _I), ("precond", _I),
                ("dsa_rtol", _D), ("dsa_max_it", _I), ("zero_start", _I)]


class ServeReport(ctypes.Structure):
    _fields_ = [("solve", SolveReport), ("status", _I), ("bucket", _I), ("slot", _I), ("pad", _I),
                ("t_submit", _D), ("t_admit", _D), ("t_done", _D)]


def _report(r):
    return dict(n_sweep=r.n_sweep, converged=bool(r.converged), n_romsa=r.n_romsa, n_dsa=r.n_dsa,
                dsa_iters=r.dsa_iters, last_change=r.last_change, rho_inf=r.rho_inf,
                n_sweep32=r.n_sweep32, r_inf=r.r_inf, balance_cell=r.balance_cell,
                balance=r.balance)


def solve_opts(eps, sa=SA_DSA, rel=False, max_iter=1000, theta=0, eps_romsad=0.0, dsa_rtol=1e-10,
               dsa_max_it=500, schedule=None, fp32_switch=0.0, refine_kappa=0.0, refine_inner=0,
               gang_wait=0, rom_bf16=False, verify=False, sa_history=None, outer_ff=False):
    """rte_solve_opts; `schedule` (uint8 per iteration) and `sa_history` (a writable uint8 numpy
    array [B][max_iter]) are kept alive on the returned struct."""
    sched = None if schedule is None else _host(schedule, np.uint8)
    if sa_history is not None and (sa_history.dtype != np.uint8 or not sa_history.flags.c_contiguous):
        raise ValueError("sa_history must be a C-contiguous uint8 array")
    o = _SolveOpts(float(eps), 1 if rel else 0, int(max_iter), int(sa), int(theta),
                   float(eps_romsad), float(dsa_rtol), int(dsa_max_it),
                   None if sched is None else sched.ctypes.data_as(_P), float(fp32_switch),
                   float(refine_kappa), int(refine_inner), 1 if rom_bf16 else 0, int(gang_wait),
                   1 if verify else 0,
                   None if sa_history is None else sa_history.ctypes.data_as(_P),
                   1 if outer_ff else 0)
    o._sched = sched
    o._hist = sa_history
    return o


def _ptr(t):
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _host(a, dtype=np.float64):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


class Disc:
    """Discretisation handle: mesh, S_N rule, material map (rte_disc_create)."""

    def __init__(self, problem, device=0):
        L = lib()
        self._mat = _host(problem.mat_id, np.int32)
        dom = tuple(problem.domain) + ((0.0, 1.0) if problem.dim == 1 else ())
        edges = getattr(problem, "edges", None)
        self._dx = None if edges is None or problem.dim != 1 else _host(np.diff(edges))
        mat_r = getattr(problem, "mat_id_right", None)
        self._matr = None if mat_r is None else _host(mat_r, np.int32)
        d = _DiscDesc(problem.dim, problem.nx, problem.ny, dom[0], dom[1], dom[2], dom[3],
                      problem.n_phi, problem.n_vz, problem.n_mat,
                      self._mat.ctypes.data_as(_P),
                      None if self._dx is None else self._dx.ctypes.data_as(_P),
                      None if self._matr is None else self._matr.ctypes.data_as(_P))
        h = _P()
        check(L.rte_disc_create(ctypes.byref(d), device, ctypes.byref(h)))
        self.h = h
        self.device = device
        info = np.zeros(8, np.int64)
        check(L.rte_disc_info(h, info.ctypes.data_as(_P)))
        (self.n_cells, self.n_dof, self.P, self.n_angles, self.n_dirs, self.n_mat, self.dim,
         _) = (int(x) for x in info)

    def quadrature(self):
        v = np.zeros((self.n_angles, 3))
        w = np.zeros(self.n_angles)
        check(lib().rte_disc_quadrature(self.h, v.ctypes.data_as(_P), w.ctypes.data_as(_P)))
        return v, w

    def close(self):
        if self.h:
            lib().rte_disc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """B parametric instances on one discretisation (rte_batch_create / _set_params)."""

    def __init__(self, disc: Disc, B: int):
        h = _P()
        check(lib().rte_batch_create(disc.h, int(B), ctypes.byref(h)))
        self.h = h
        self.disc = disc
        self.B = int(B)

    @classmethod
    def from_problem(cls, problem, disc: Disc | None = None, device=0):
        disc = disc or Disc(problem, device)
        b = cls(disc, problem.batch)
        b.set_params(problem)
        return b

    def set_params(self, problem):
        st = _host(problem.sigma_t)
        ss = _host(problem.sigma_s)
        src = _host(problem.source)
        inf = _host(problem.inflow)
        check(lib().rte_batch_set_params(self.h, st.ctypes.data_as(_P), ss.ctypes.data_as(_P),
                                         src.ctypes.data_as(_P), inf.ctypes.data_as(_P)))

    def set_params_device(self, sigma_t, sigma_s, source, inflow, stream=None):
        """rte_batch_set_params_device: parameters from float64 device tensors [B][n_mat],
        [B][n_mat], [B][n_cells], [B][2*dim]; asynchronous on `stream`, validated on the device
        (an invalid value makes the next call that uses the parameters raise)."""
        for t, shape in ((sigma_t, (self.B, self.disc.n_mat)), (sigma_s, (self.B, self.disc.n_mat)),
                         (source, (self.B, self.disc.n_cells)), (inflow, (self.B, 2 * self.disc.dim))):
            if tuple(t.shape) != shape or str(t.dtype) != "torch.float64" or not t.is_cuda:
                raise ValueError(f"expected a float64 CUDA tensor of shape {shape}")
        check(lib().rte_batch_set_params_device(self.h, _ptr(sigma_t), _ptr(sigma_s), _ptr(source),
                                                _ptr(inflow), _stream(stream)))

    def set_slots(self, slots, sigma_t, sigma_s, source, inflow, stream=None):
        """Parameters of instances `slots` only (rte_batch_set_slots)."""
        sl = _host(slots, np.int32).reshape(-1)
        n = len(sl)
        st, ss = _host(sigma_t).reshape(n, -1), _host(sigma_s).reshape(n, -1)
        src, inf = _host(source).reshape(n, -1), _host(inflow).reshape(n, -1)
        check(lib().rte_batch_set_slots(self.h, n, sl.ctypes.data_as(_P), st.ctypes.data_as(_P),
                                        ss.ctypes.data_as(_P), src.ctypes.data_as(_P),
                                        inf.ctypes.data_as(_P), _stream(stream)))

    def dsa_smoothing(self, nu):
        """Red-black smoothing sweeps per multigrid level of the 2D DSA (rte_batch_dsa_smoothing)."""
        check(lib().rte_batch_dsa_smoothing(self.h, int(nu)))

    def dsa_smoother(self, kind):
        """Form of the 2D DSA multigrid smoother: SMOOTHER_GLOBAL / _TILED / _BLOCKED
        (rte_batch_dsa_smoother)."""
        check(lib().rte_batch_dsa_smoother(self.h, int(kind)))

    def info(self):
        out = np.zeros(6, np.int64)
        check(lib().rte_batch_info(self.h, out.ctypes.data_as(_P)))
        return dict(B=int(out[0]), bytes=int(out[1]), dirs_per_warp=int(out[2]),
                    min_dirs_per_warp=int(out[3]), dynamic=bool(out[4]), params_set=bool(out[5]))

    def tune(self, dirs_per_warp=0):
        """Directions swept per warp in 2D (1, 2, 4, 8; 0 = automatic)."""
        check(lib().rte_batch_tune(self.h, int(dirs_per_warp)))

    def autotune(self, stream=None):
        """Measured directions-per-warp per number of running instances (rte_batch_autotune).
        Returns [(count, dirs_per_warp), ...] ascending."""
        n = _I()
        table = np.zeros(64, np.int32)
        check(lib().rte_batch_autotune(self.h, _stream(stream), ctypes.byref(n),
                                       table.ctypes.data_as(_P)))
        return [(int(table[2 * k]), int(table[2 * k + 1])) for k in range(n.value)]

    def tuned(self):
        """rte_batch_tuned: [(count, dirs_per_warp, warps per direction group), ...] of the FP64
        sweep after autotune(), ascending; [] when not autotuned."""
        n = _I()
        table = np.zeros(96, np.int32)
        check(lib().rte_batch_tuned(self.h, ctypes.byref(n), table.ctypes.data_as(_P)))
        return [tuple(int(x) for x in table[3 * k:3 * k + 3]) for k in range(n.value)]

    def timing(self, enable):
        """enable=1 reset+start, 0 reset+stop, -1 read.  Returns a dict of phase times (ms) and
        counts: sweep (kernel only), dsa, rom, setup."""
        out = np.zeros(15)
        check(lib().rte_batch_timing(self.h, int(enable), out.ctypes.data_as(_P)))
        return dict(sweep_ms=float(out[0]), sweep_launches=int(out[1]), sweep_units=float(out[2]),
                    dsa_ms=float(out[3]), dsa_calls=int(out[4]), rom_ms=float(out[5]),
                    rom_calls=int(out[6]), setup_ms=float(out[7]), setup_calls=int(out[8]),
                    sweep32_ms=float(out[9]), sweep32_launches=int(out[10]),
                    sweep32_units=float(out[11]), sweepff_ms=float(out[12]),
                    sweepff_launches=int(out[13]), sweepff_units=float(out[14]))

    def directions(self):
        d = np.zeros((self.disc.n_dirs, 4))
        check(lib().rte_batch_directions(self.h, d.ctypes.data_as(_P)))
        return d

    def sweep(self, rho_in, rho_out, psi_out=None, with_source=True, active=None, stream=None):
        check(lib().rte_sweep(self.h, _ptr(rho_in), _ptr(rho_out), _ptr(psi_out),
                              1 if with_source else 0, _ptr(active), _stream(stream)))

    def sweep_f32(self, rho_in, rho_out, active=None, stream=None):
        """rte_sweep_f32: one FP32 sweep with source (2D), result in FP64."""
        check(lib().rte_sweep_f32(self.h, _ptr(rho_in), _ptr(rho_out), _ptr(active),
                                  _stream(stream)))

    def sweep_ff(self, rho_in, rho_out, active=None, stream=None):
        """rte_sweep_ff: one float-float sweep with source (2D), result in FP64."""
        check(lib().rte_sweep_ff(self.h, _ptr(rho_in), _ptr(rho_out), _ptr(active),
                                 _stream(stream)))

    def sweep_static(self, rho_in, rho_out, with_source=True, stream=None):
        """rte_sweep_static: the same sweep with the library's fixed scratch (no allocation)."""
        check(lib().rte_sweep_static(self.h, _ptr(rho_in), _ptr(rho_out), 1 if with_source else 0,
                                     _stream(stream)))

    def change_norm(self, rho_star, rho_prev, norms, stream=None):
        check(lib().rte_change_norm(self.h, _ptr(rho_star), _ptr(rho_prev), _ptr(norms),
                                    _stream(stream)))

    def correction_source(self, rho_star, rho_prev, R, stream=None):
        check(lib().rte_correction_source(self.h, _ptr(rho_star), _ptr(rho_prev), _ptr(R),
                                          _stream(stream)))

    def dsa_correction(self, R, drho, rtol=1e-10, max_it=500, active=None, stream=None):
        iters = np.zeros(self.B, np.int32)
        st = check(lib().rte_dsa_correction(self.h, _ptr(R), _ptr(drho), float(rtol), int(max_it),
                                            _ptr(active), iters.ctypes.data_as(_P),
                                            _stream(stream)), allow=(RTE_ENOCONV,))
        return iters, st

    def solve(self, rho, eps, sa=SA_DSA, rel=False, max_iter=1000, theta=0, eps_romsad=0.0,
              dsa_rtol=1e-10, dsa_max_it=500, rom_c=None, schedule=None, history=False,
              fp32_switch=0.0, refine_kappa=0.0, refine_inner=0, gang_wait=0, rom_bf16=False,
              verify=False, outer_ff=False, stream=None):
        """rte_solve.  Returns (reports, hist, status); with history=True, hist is the change per
        sweep [B][max_iter] and each report also carries "sa_history", the codes of
        rte_solve_opts.sa_history for its n_sweep sweeps."""
        sah = np.zeros((self.B, max_iter), np.uint8) if history else None
        opts = solve_opts(eps, sa, rel, max_iter, theta, eps_romsad, dsa_rtol, dsa_max_it, schedule,
                          fp32_switch, refine_kappa, refine_inner, gang_wait, rom_bf16, verify, sah,
                          outer_ff)
        reps = (SolveReport * self.B)()
        hist = np.zeros((self.B, max_iter)) if history else None
        st = check(lib().rte_solve(self.h, ctypes.byref(opts), None if rom_c is None else rom_c.h,
                                   _ptr(rho), reps,
                                   None if hist is None else hist.ctypes.data_as(_P),
                                   _stream(stream)), allow=(RTE_ENOCONV,))
        out = [_report(r) for r in reps]
        if history:
            for b, r in enumerate(out):
                r["sa_history"] = sah[b, : r["n_sweep"]].copy()
        return out, hist, st

    def residual(self, rho, out, cell_balance=None, active=None, stream=None):
        """rte_residual: out [B][4] = (||(I - L) rho - b-bar||_inf, max per-cell balance, global
        balance defect, int G), device tensors; cell_balance [B][n_cells] optional."""
        check(lib().rte_residual(self.h, _ptr(rho), _ptr(out), _ptr(cell_balance), _ptr(active),
                                 _stream(stream)))

    def pgmres(self, rho, rtol, restart=25, max_iter=500, precond=True, dsa_rtol=0.0,
               dsa_max_it=1, zero_start=True, stream=None):
        """DSA-preconditioned restarted GMRES on (I - L) rho = b-bar (rte_pgmres)."""
        o = _GmresOpts(float(rtol), int(restart), int(max_iter), 1 if precond else 0,
                       float(dsa_rtol), int(dsa_max_it), 1 if zero_start else 0)
        reps = (SolveReport * self.B)()
        st = check(lib().rte_pgmres(self.h, ctypes.byref(o), _ptr(rho), reps, _stream(stream)),
                   allow=(RTE_ENOCONV,))
        return [_report(r) for r in reps], st

    def close(self):
        if self.h:
            lib().rte_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_many(batches, rhos, opts, roms=None, streams=None, lockstep=False, interleaved=False):
    """rte_solve_many: batches[k] solved from rhos[k] (device tensors, overwritten) with opts[k]
    (rte_solve_opts from solve_opts()), optional roms[k] and streams[k].  lockstep=True runs
    rte_solve_lockstep instead (one sweep launch over all batches per iteration), interleaved=True
    rte_solve_interleaved (the sweeps one after another on a priority stream, each batch's
    corrections beside the next batch's sweep).  Returns per-batch report lists and the status."""
    if lockstep and interleaved:
        raise ValueError("lockstep and interleaved exclude each other")
    n = len(batches)
    bh = (_P * n)(*[b.h for b in batches])
    oa = (_SolveOpts * n)(*opts)
    rh = (_P * n)(*[_ptr(r) for r in rhos])
    reps = [(SolveReport * b.B)() for b in batches]
    rp = (_P * n)(*[ctypes.cast(r, _P) for r in reps])
    ro = None if roms is None else (_P * n)(*[None if r is None else r.h for r in roms])
    sa = None if streams is None else (_P * n)(*[_stream(s) for s in streams])
    fn = (lib().rte_solve_lockstep if lockstep else
          lib().rte_solve_interleaved if interleaved else lib().rte_solve_many)
    st = check(fn(n, bh, oa, ro, rh, rp, sa), allow=(RTE_ENOCONV,))
    return [[_report(r) for r in rr] for rr in reps], st


class Rom:
    """A POD reduced model built on the GPU (rte_rom_build) or loaded from a file."""

    def __init__(self, h, disc=None):
        self.h = h
        self.disc = disc  # keeps the discretisation alive as long as the model
        info = np.zeros(6)
        check(lib().rte_rom_info(h, info.ctypes.data_as(_P), None))
        self.r, self.n_snap = int(info[0]), int(info[1])
        self.eps_pod = float(info[2])
        sv = np.zeros(max(self.n_snap, 1))
        check(lib().rte_rom_info(h, info.ctypes.data_as(_P), sv.ctypes.data_as(_P)))
        self.sv = sv[: self.n_snap]

    @staticmethod
    def build(train: Batch, eps_train=1e-12, window=3, rank_p=20, rank_c=20, eps_pod=1e-9,
              max_iter=2000, dsa_rtol=1e-12, correction_start="zero", stream=None):
        """(rom_p, rom_c); correction_start="romig" takes the correction snapshots from training
        runs started at the ROMIG guess (for ROMIG followed by ROMSAD)."""
        o = _RomOpts(float(eps_train), int(window), int(rank_p), int(rank_c), float(eps_pod),
                     int(max_iter), float(dsa_rtol), 1 if correction_start == "romig" else 0)
        hp, hc = _P(), _P()
        check(lib().rte_rom_build(train.h, ctypes.byref(o), ctypes.byref(hp), ctypes.byref(hc),
                                  _stream(stream)))
        return Rom(hp, train.disc), Rom(hc, train.disc)

    def save(self, path):
        check(lib().rte_rom_save(self.h, os.fsencode(path)))

    @staticmethod
    def load(disc: Disc, path):
        h = _P()
        check(lib().rte_rom_load(disc.h, os.fsencode(path), ctypes.byref(h)))
        return Rom(h, disc)

    def initial_guess(self, batch: Batch, rho0, active=None, stream=None):
        check(lib().rte_rom_initial_guess(self.h, batch.h, _ptr(rho0), _ptr(active),
                                          _stream(stream)))

    def romsa_correction(self, batch: Batch, R, drho, active=None, stream=None):
        check(lib().rte_romsa_correction(self.h, batch.h, _ptr(R), _ptr(drho), _ptr(active),
                                         _stream(stream)))

    def close(self):
        if self.h:
            lib().rte_rom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (rte_server_*): buckets of slots, one worker thread."""

    def __init__(self, device=0):
        h = _P()
        check(lib().rte_server_create(int(device), ctypes.byref(h)))
        self.h = h
        self._keep = []
        self.buckets = []

    def add_bucket(self, batch: Batch, rom_p=None, rom_c=None, **opts):
        """Adds a bucket whose slots are `batch`'s instances; opts as solve_opts() (eps unused)."""
        o = solve_opts(opts.pop("eps", 0.0), **opts)
        k = _I()
        check(lib().rte_server_add_bucket(self.h, batch.h, None if rom_p is None else rom_p.h,
                                          None if rom_c is None else rom_c.h, ctypes.byref(o),
                                          ctypes.byref(k)))
        self._keep += [batch, rom_p, rom_c, o]
        self.buckets.append(batch)
        return int(k.value)

    def start(self):
        check(lib().rte_server_start(self.h))

    def submit(self, bucket, sigma_t, sigma_s, source, inflow, eps):
        st, ss, src, inf = _host(sigma_t), _host(sigma_s), _host(source), _host(inflow)
        t = ctypes.c_uint64()
        check(lib().rte_server_submit(self.h, int(bucket), st.ctypes.data_as(_P),
                                      ss.ctypes.data_as(_P), src.ctypes.data_as(_P),
                                      inf.ctypes.data_as(_P), float(eps), ctypes.byref(t)))
        return int(t.value)

    def wait(self, ticket, timeout=60.0, want_rho=True):
        """(rho, report) once the request finished, or None on timeout."""
        rep = ServeReport()
        rho = None
        if want_rho:
            # the bucket is only known from the report; allocate for the largest bucket
            rho = np.zeros(max(b.disc.n_dof for b in self.buckets))
        st = lib().rte_server_wait(self.h, ctypes.c_uint64(ticket), float(timeout),
                                   None if rho is None else rho.ctypes.data_as(_P), ctypes.byref(rep))
        if st == RTE_ETIMEOUT:
            return None
        check(st, allow=(RTE_ENOCONV,))
        r = _report(rep.solve)
        r.update(status=rep.status, bucket=rep.bucket, slot=rep.slot, t_submit=rep.t_submit,
                 t_admit=rep.t_admit, t_done=rep.t_done)
        if rho is not None:
            rho = rho[: self.buckets[rep.bucket].disc.n_dof]
        return rho, r

    def stats(self):
        out = np.zeros(8)
        check(lib().rte_server_stats(self.h, out.ctypes.data_as(_P)))
        keys = ("launches", "admitted", "completed", "queued", "max_queue", "max_running",
                "busy_s", "uptime_s")
        return dict(zip(keys, (float(x) for x in out)))

    def close(self):
        if self.h:
            lib().rte_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
