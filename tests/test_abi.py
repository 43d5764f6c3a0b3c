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
    assert L.rte_version() == 10900


def test_calls_without_gpu_fail_cleanly():
    """Without a device the calls return a status and a message; nothing crashes."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2402_10488_gb300 import inputs
    with pytest.raises(rte.RTEError) as e:
        rte.Disc(inputs.slab(4, 2, 1.0, 0.5))
    assert e.value.status in (rte.RTE_ECUDA, rte.RTE_EINVAL)


def test_boundary_rejects_bad_arguments_before_touching_the_device():
    """Argument checks of the C ABI run on the host before any CUDA call: each bad input returns
    RTE_EINVAL with a message (this runs with or without a GPU)."""
    import ctypes

    import numpy as np
    L = rte.lib()
    mat = np.zeros(4, np.int32)
    right_bad = np.array([0, 0, 1, 0], np.int32)     # material 1 with n_mat = 1

    def desc(**kw):
        base = dict(dim=1, nx=4, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, n_phi=4, n_vz=0, n_mat=1,
                    mat_id=mat.ctypes.data_as(ctypes.c_void_p))
        base.update(kw)
        return rte._DiscDesc(**base)

    bad = [desc(dim=3), desc(nx=0), desc(ny=2), desc(x1=0.0), desc(n_mat=0), desc(n_phi=3),
           desc(dim=2, ny=1, n_phi=5, n_vz=2), desc(dim=2, ny=1, n_phi=4, n_vz=0),
           desc(mat_id=None),
           # linear cross sections: right-end material out of range; a right-end map in 2D
           desc(mat_id_right=right_bad.ctypes.data_as(ctypes.c_void_p)),
           desc(dim=2, nx=2, ny=2, n_phi=4, n_vz=2, mat_id_right=mat.ctypes.data_as(ctypes.c_void_p))]
    for d in bad:
        h = ctypes.c_void_p()
        assert L.rte_disc_create(ctypes.byref(d), 0, ctypes.byref(h)) == rte.RTE_EINVAL
        assert L.rte_last_error()
        assert not h.value
    assert L.rte_disc_create(None, 0, None) == rte.RTE_EINVAL
    null = ctypes.c_void_p()
    assert L.rte_batch_create(None, 4, ctypes.byref(null)) == rte.RTE_EINVAL
    assert L.rte_solve(None, None, None, None, None, None, None) == rte.RTE_EINVAL
    assert L.rte_pgmres(None, None, None, None, None) == rte.RTE_EINVAL
    assert L.rte_server_submit(None, 0, None, None, None, None, 1e-6, None) == rte.RTE_EINVAL
    assert L.rte_server_wait(None, 1, 0.0, None, None) == rte.RTE_EINVAL
    assert L.rte_rom_load(None, b"/nonexistent", ctypes.byref(null)) == rte.RTE_EINVAL
    assert L.rte_batch_dsa_smoothing(None, 2) == rte.RTE_EINVAL
    assert L.rte_solve_many(0, None, None, None, None, None, None) == rte.RTE_EINVAL
    # destroying null handles is a no-op
    for fn in (L.rte_disc_destroy, L.rte_batch_destroy, L.rte_rom_destroy, L.rte_server_destroy):
        assert fn(None) == rte.RTE_OK


def test_server_create_and_destroy_without_buckets():
    """The serving loop's host object: created, refuses to start without a bucket, destroyed."""
    import ctypes
    L = rte.lib()
    h = ctypes.c_void_p()
    assert L.rte_server_create(0, ctypes.byref(h)) == rte.RTE_OK
    assert L.rte_server_start(h) == rte.RTE_ESTATE
    stats = (ctypes.c_double * 8)()
    assert L.rte_server_stats(h, stats) == rte.RTE_OK and stats[2] == 0
    assert L.rte_server_destroy(h) == rte.RTE_OK


def test_tensor_core_products_and_service_calls_check_arguments_on_the_host():
    """The BF16 POD products, the workspace query, the smoother choice and the fault hook reject bad
    arguments with RTE_EINVAL on the host, before any device memory is touched (the pointers below
    are never dereferenced)."""
    import ctypes

    import numpy as np
    L = rte.lib()
    out = np.zeros(1, np.int64)
    p_out = out.ctypes.data_as(ctypes.c_void_p)
    assert L.rte_pod_workspace_bytes(20, 65536, 152, p_out) == rte.RTE_OK and out[0] > 256
    small = int(out[0])
    assert L.rte_pod_workspace_bytes(20, 4096, 152, p_out) == rte.RTE_OK and 0 < out[0] <= small
    for r, n, B in ((33, 64, 2), (0, 64, 2), (20, 0, 2), (20, 64, 0)):
        assert L.rte_pod_workspace_bytes(r, n, B, p_out) == rte.RTE_EINVAL
    assert L.rte_pod_workspace_bytes(20, 64, 2, None) == rte.RTE_EINVAL
    fake = ctypes.c_void_p(0x10000)          # 16-byte aligned, never dereferenced
    odd = ctypes.c_void_p(0x10008)           # not 16-byte aligned
    assert L.rte_pod_project_bf16(None, 20, 64, fake, 2, None, fake, fake, None) == rte.RTE_EINVAL
    assert L.rte_pod_project_bf16(fake, 20, 64, fake, 2, None, fake, odd, None) == rte.RTE_EINVAL
    assert "aligned" in L.rte_last_error().decode()
    assert L.rte_pod_project_bf16(fake, 33, 64, fake, 2, None, fake, fake, None) == rte.RTE_EINVAL
    assert L.rte_pod_lift_bf16(fake, 0, 64, fake, 2, None, fake, fake, None) == rte.RTE_EINVAL
    assert L.rte_pod_lift_bf16(fake, 20, 64, fake, 0, None, fake, fake, None) == rte.RTE_EINVAL
    assert L.rte_pod_lift_bf16(fake, 20, 64, None, 2, None, fake, fake, None) == rte.RTE_EINVAL
    assert L.rte_batch_dsa_smoother(None, rte.SMOOTHER_GLOBAL) == rte.RTE_EINVAL
    assert L.rte_fault_inject(7) == rte.RTE_EINVAL
    assert L.rte_fault_inject(0) == rte.RTE_OK
