"""GPU parity of the POD ROM pipeline (Sec. 3): offline bases and singular values, ROMIG, ROMSA
and ROMSAD solves, against the CPU oracle on the same seeded training and test sets.

Tolerances, derived.  Training solves on both sides stop at an absolute change of 1e-13 with
DSA solved to 1e-13, so the snapshot matrices agree to delta ~ 1e-13 relative; the thin SVDs
(QR + one-sided Jacobi on the GPU, LAPACK in numpy) resolve singular values to a few ulps of
sigma_1, so they agree to ~delta sigma_1: checked at 1e-10 sigma_1.  A rank-r basis is the span of
the leading r singular vectors, which a perturbation of relative size delta moves by an angle of
at most delta sigma_1 / (sigma_r - sigma_{r+1}) (Wedin's bound); ROM outputs move by that angle
times the conditioning of the small reduced system.  The GPU-built models are therefore compared
at ranks that end at a wide gap of the oracle's spectrum (rank 4 of the parametric snapshots:
gap 6.8e-3 sigma_1; rank 4 of the correction snapshots: 1.8e-2 sigma_1), where the bound is
~1e-11, at 1e-10.  The online stage alone -- reduced-operator assembly and LU, projection, lift,
ROMIG, ROMSA and the Alg. 2 switch -- is compared with no SVD in between by loading the oracle's
own reduced model into the library through its ROM file format: 1e-12 for single ROM steps,
1e-11 for ROMSAD iterates, whose DSA steps are FGMRES solves to 1e-13 on the GPU and direct
solves in the oracle.  The GPU's own reduced operators are compared with the oracle's after
rotating one basis onto the other."""
import os
import struct

import numpy as np
import pytest

from oracle.dsa import ConsistentDSA
from oracle.rom import OfflineROMs
from oracle.sisa import sisa
from oracle.transport import Transport
from paper_2402_10488_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, NA, NVZ = 12, 8, 2
RP, RC = 4, 4          # ranks at wide gaps of the training spectra (see the header)


def _rte():
    from paper_2402_10488_gb300 import build, rte
    build.build()
    return rte


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module")
def roms():
    rte = _rte()
    train = inputs.lattice_train(N, NA, n_train=8, n_vz=NVZ)
    tb = rte.Batch.from_problem(train)
    rp, rc = rte.Rom.build(tb, eps_train=1e-13, window=3, rank_p=RP, rank_c=RC, max_iter=300,
                           dsa_rtol=1e-13)
    off = OfflineROMs(train, eps_train=1e-13, window=3, rank_p=RP, rank_c=RC)
    return rte, tb, rp, rc, off


# ---- the library's ROM file (rte_rom_save / rte_rom_load), written and read here ---------------
# layout: "RTEROM03", int32 {dim, nx, ny, n_phi, n_vz, n_mat, r, n_snap, n_cells, P}, double
# {x0, x1, y0, y1, eps_equiv}, int32 mat_id[n_cells] (1D: double dx[nx], int32 mat_right[nx]),
# double sv[n_snap], A0[r][r], Aa[n_mat][r][r], As[n_mat][r][r], a_side[4][r], U_rho[r][n_dof],
# U_iso[r][n_dof]

def _write_oracle_rom(path, problem, model, pod):
    """The oracle's reduced model (ReducedModel + its POD) in the library's file format."""
    assert problem.dim == 2
    tr = Transport(problem, 0)
    r = model.r
    Uj = model.U.reshape(model.Nv, model.N, r)
    a_side = np.zeros((4, r))
    for s in range(4):
        g = np.zeros(4)
        g[s] = 1.0
        a_side[s] = sum(Uj[j].T @ tr.dg.inflow_vector(tr.v[j], g) for j in range(model.Nv))
    with open(path, "wb") as f:
        f.write(b"RTEROM03")
        f.write(struct.pack("<10i", 2, problem.nx, problem.ny, problem.n_phi, problem.n_vz,
                            problem.n_mat, r, pod.sv.size, problem.n_cells, 4))
        f.write(struct.pack("<5d", *problem.domain, pod.eps_equiv))
        f.write(np.ascontiguousarray(problem.mat_id, np.int32).tobytes())
        for a in [pod.sv, model.A0, np.stack(model.Aa), np.stack(model.As), a_side,
                  model.U_rho.T, model.U_iso.T]:
            f.write(np.ascontiguousarray(a, np.float64).tobytes())


def _read_rom(path, n_mat, n_dof):
    with open(path, "rb") as f:
        assert f.read(8) == b"RTEROM03"
        hdr = struct.unpack("<10i", f.read(40))
        f.read(40)
        r, n_snap, n_cells = hdr[6], hdr[7], hdr[8]
        f.read(4 * n_cells)
        rd = lambda *shape: np.frombuffer(f.read(8 * int(np.prod(shape))), np.float64).reshape(shape)
        sv, A0, Aa, As, a_side = rd(n_snap), rd(r, r), rd(n_mat, r, r), rd(n_mat, r, r), rd(4, r)
        return dict(sv=sv, A0=A0, Aa=Aa, As=As, U_rho=rd(r, n_dof).T, U_iso=rd(r, n_dof).T)


def test_singular_values_match(roms):
    rte, _, rp, rc, off = roms
    assert rp.r == RP and rc.r == RC
    assert rp.n_snap == 8 and rc.n_snap == off.dF.shape[1]
    np.testing.assert_allclose(rp.sv, off.pod_p.sv, rtol=0, atol=1e-10 * off.pod_p.sv[0])
    np.testing.assert_allclose(rc.sv, off.pod_c.sv, rtol=0, atol=1e-10 * off.pod_c.sv[0])
    assert abs(rc.eps_pod - off.pod_c.eps_equiv) < 1e-10


def test_reduced_operators_match_after_basis_alignment(roms, tmp_path):
    """The GPU's U^rho, U^iso and affine reduced operators A_0r, A_{a,m,r}, A_{s,m,r} (Sec. 3.1.1)
    equal the oracle's in the oracle's basis rotated onto the GPU's: Q = argmin ||[U^rho; U^iso] Q
    - [U^rho; U^iso]_gpu|| is orthogonal to the subspace angle, and A_gpu = Q^T A Q."""
    rte, tb, rp, rc, off = roms
    for gpu, model in ((rp, off.rom_p), (rc, off.rom_c)):
        path = str(tmp_path / "gpu.rom")
        gpu.save(path)
        g = _read_rom(path, tb.disc.n_mat, tb.disc.n_dof)
        Xo = np.vstack([model.U_rho, model.U_iso])
        Xg = np.vstack([g["U_rho"], g["U_iso"]])
        Q = np.linalg.lstsq(Xo, Xg, rcond=None)[0]
        assert np.abs(Q.T @ Q - np.eye(gpu.r)).max() < 1e-10
        assert _rel(Xo @ Q, Xg) < 1e-10
        ops = [(g["A0"], model.A0)] + [(g["Aa"][m], model.Aa[m]) for m in range(tb.disc.n_mat)] + \
              [(g["As"][m], model.As[m]) for m in range(tb.disc.n_mat)]
        for Ag, Ao in ops:
            assert _rel(Ag, Q.T @ Ao @ Q) < 1e-10


def test_online_stage_with_the_oracle_rom(roms, tmp_path):
    """The oracle's rank-6 parametric and rank-8 correction models, loaded into the library: ROMIG
    guesses and ROMSA corrections at 1e-12 and ROMSAD iterates under a forced schedule at 1e-11
    of the oracle's (no SVD on either side, so nothing limits the agreement but rounding)."""
    rte, tb, _, _, _ = roms
    train = inputs.lattice_train(N, NA, n_train=8, n_vz=NVZ)
    off = OfflineROMs(train, eps_train=1e-13, window=3, rank_p=6, rank_c=8)
    paths = []
    for name, model, pod in (("p", off.rom_p, off.pod_p), ("c", off.rom_c, off.pod_c)):
        paths.append(str(tmp_path / f"oracle_{name}.rom"))
        _write_oracle_rom(paths[-1], train, model, pod)
    rp = rte.Rom.load(tb.disc, paths[0])
    rc = rte.Rom.load(tb.disc, paths[1])
    assert rp.r == 6 and rc.r == 8
    test = inputs.lattice_test(N, NA, 3, n_vz=NVZ)
    batch = rte.Batch(tb.disc, 3)
    batch.set_params(test)
    rho0 = torch.zeros((3, test.n_dof), dtype=torch.float64, device="cuda")
    rp.initial_guess(batch, rho0)
    R = np.random.default_rng(3).uniform(0, 1, (3, test.n_dof))
    d = torch.zeros((3, test.n_dof), dtype=torch.float64, device="cuda")
    rc.romsa_correction(batch, torch.tensor(R, device="cuda"), d)
    g0, gd = rho0.cpu().numpy(), d.cpu().numpy()
    for b in range(3):
        tr = Transport(test, b)
        assert _rel(g0[b], off.rom_p.initial_guess(tr)) < 1e-12
        assert _rel(gd[b], off.rom_c.romsa_correction(tr, R[b])) < 1e-12
    sched = np.array([1, 1, 0, 1, 0, 0, 0, 0], np.uint8)
    rho = torch.zeros((3, test.n_dof), dtype=torch.float64, device="cuda")
    rep, _, _ = batch.solve(rho, 0.0, sa=rte.SA_ROMSAD, max_iter=8, rom_c=rc, schedule=sched,
                            dsa_rtol=1e-13, dsa_max_it=3000, history=True)
    got = rho.cpu().numpy()
    names = ["romsa" if s else "dsa" for s in sched]
    for b in range(3):
        tr = Transport(test, b)
        ref = sisa(tr, np.zeros(tr.n_dof), 0.0, 8, "romsad", dsa=ConsistentDSA(tr), rom_c=off.rom_c,
                   schedule=names)
        assert _rel(got[b], ref["rho"]) < 1e-11
        assert list(rep[b]["sa_history"]) == [rte.SA_ROMSA if s else rte.SA_DSA for s in sched]


def test_romig_matches_oracle(roms):
    rte, tb, rp, rc, off = roms
    test = inputs.lattice_test(N, NA, 3, n_vz=NVZ)
    batch = rte.Batch(tb.disc, 3)
    batch.set_params(test)
    rho0 = torch.zeros((3, test.n_dof), dtype=torch.float64, device="cuda")
    rp.initial_guess(batch, rho0)
    got = rho0.cpu().numpy()
    for b in range(3):
        ref = off.rom_p.initial_guess(Transport(test, b))
        assert _rel(got[b], ref) < 1e-10, _rel(got[b], ref)


def test_romsa_correction_matches_oracle(roms):
    rte, tb, rp, rc, off = roms
    test = inputs.lattice_test(N, NA, 2, n_vz=NVZ)
    batch = rte.Batch(tb.disc, 2)
    batch.set_params(test)
    R = np.random.default_rng(3).uniform(0, 1, (2, test.n_dof))
    d = torch.zeros((2, test.n_dof), dtype=torch.float64, device="cuda")
    rc.romsa_correction(batch, torch.tensor(R, device="cuda"), d)
    got = d.cpu().numpy()
    for b in range(2):
        ref = off.rom_c.romsa_correction(Transport(test, b), R[b])
        assert _rel(got[b], ref) < 1e-10, _rel(got[b], ref)


def test_romsad_forced_schedule_iterates_and_converged(roms):
    rte, tb, rp, rc, off = roms
    test = inputs.lattice_test(N, NA, 2, n_vz=NVZ)
    batch = rte.Batch(tb.disc, 2)
    batch.set_params(test)
    sched = np.array([1, 1, 0, 1, 0, 0, 0, 0], np.uint8)
    rho = torch.zeros((2, test.n_dof), dtype=torch.float64, device="cuda")
    rep, hist, st = batch.solve(rho, 0.0, sa=rte.SA_ROMSAD, max_iter=8, rom_c=rc, schedule=sched,
                                dsa_rtol=1e-13, dsa_max_it=3000, history=True)
    got = rho.cpu().numpy()
    names = ["romsa" if s else "dsa" for s in sched]
    for b in range(2):
        tr = Transport(test, b)
        ref = sisa(tr, np.zeros(tr.n_dof), 0.0, 8, "romsad", dsa=ConsistentDSA(tr), rom_c=off.rom_c,
                   schedule=names)
        assert _rel(got[b], ref["rho"]) < 1e-10, _rel(got[b], ref["rho"])
        # a correction follows every one of the 8 sweeps: ROMSA after 1, 2, 4; DSA after the rest
        assert rep[b]["n_romsa"] == 3 and rep[b]["n_dsa"] == 5
    # Alg. 2 switch, converged answer equals SI-DSA's
    rho2 = torch.zeros((2, test.n_dof), dtype=torch.float64, device="cuda")
    rep2, hist2, st2 = batch.solve(rho2, 1e-12, sa=rte.SA_ROMSAD, rel=True, max_iter=300, rom_c=rc,
                                   theta=5, eps_romsad=0.1 * max(1e-13, rc.eps_pod), dsa_rtol=1e-2,
                                   history=True)
    assert st2 == 0
    for b in range(2):
        tr = Transport(test, b)
        ref = sisa(tr, np.zeros(tr.n_dof), 1e-14, 400, "dsa", dsa=ConsistentDSA(tr), tol_mode="rel")
        assert _rel(rho2.cpu().numpy()[b], ref["rho"]) < 1e-10
        h = hist2[b, : rep2[b]["n_sweep"]]
        eps_r = 0.1 * max(1e-13, rc.eps_pod)
        n_rom_expected = sum(1 for l, dl in enumerate(h[:-1], start=1) if l <= 5 and dl >= eps_r)
        assert rep2[b]["n_romsa"] == n_rom_expected
        # the recorded choice after every sweep is Alg. 2's on the recorded changes
        want = [rte.SA_ROMSA if (l <= 5 and dl >= eps_r) else rte.SA_DSA
                for l, dl in enumerate(h[:-1], start=1)] + [rte.SA_NONE]
        assert list(rep2[b]["sa_history"]) == want


def test_romig_started_correction_rom_matches_oracle():
    """Correction snapshots from ROMIG-started training runs (remark after Alg. 2): same snapshot
    count and leading singular values as the oracle, and ROMIG + ROMSAD on test instances under a
    forced schedule agrees iterate by iterate.  The ranks end at wide gaps of the spectra (rank 3 of
    the parametric snapshots: 2.1e-2 sigma_1; rank 6 of the ROMIG-started corrections: 1.1e-2
    sigma_1), so the ROMIG guesses that start the second training pass, and with them the
    correction snapshots, agree to ~1e-11: singular values and iterates are compared at 1e-10."""
    rte = _rte()
    train = inputs.lattice_train(N, NA, n_train=6, n_vz=NVZ)
    tb = rte.Batch.from_problem(train)
    kw = dict(eps_train=1e-13, window=2, rank_p=3, rank_c=6)
    rp, rc = rte.Rom.build(tb, max_iter=300, dsa_rtol=1e-13, correction_start="romig", **kw)
    off = OfflineROMs(train, correction_start="romig", **kw)
    assert rc.n_snap == off.dF.shape[1]
    np.testing.assert_allclose(rc.sv, off.pod_c.sv, rtol=0, atol=1e-10 * off.pod_c.sv[0])
    test = inputs.lattice_test(N, NA, 2, n_vz=NVZ)
    batch = rte.Batch(tb.disc, 2)
    batch.set_params(test)
    rho = torch.zeros((2, test.n_dof), dtype=torch.float64, device="cuda")
    rp.initial_guess(batch, rho)
    sched = np.array([1, 1, 0, 0, 0, 0], np.uint8)
    rep, _, _ = batch.solve(rho, 0.0, sa=rte.SA_ROMSAD, max_iter=6, rom_c=rc, schedule=sched,
                            dsa_rtol=1e-13, dsa_max_it=3000)
    got = rho.cpu().numpy()
    names = ["romsa" if s else "dsa" for s in sched]
    for b in range(2):
        tr = Transport(test, b)
        rho0 = off.rom_p.initial_guess(tr)
        ref = sisa(tr, rho0, 0.0, 6, "romsad", dsa=ConsistentDSA(tr), rom_c=off.rom_c,
                   schedule=names)
        assert _rel(got[b], ref["rho"]) < 1e-10, _rel(got[b], ref["rho"])
        assert rep[b]["n_romsa"] == 2 and rep[b]["n_dsa"] == 4


@pytest.mark.slow
def test_full_size_romsad_solution_is_a_fixed_point_of_the_oracle_operator():
    """The bench workload at full size in the bench's launch configuration (128^2 lattice,
    CL(16,4), 152 instances, measured sweep decomposition, one FP32 V-cycle per DSA): sampled
    instances of the GPU's ROMSAD solution are fixed points of the oracle's discrete operator,
    rho = L rho + b-bar (Eq. (rho_matrix_vec)), to within what the stop test at a relative change
    of 2e-7 allows: rho is the output of a sweep that changed its input by < 2e-7 ||rho||, so one
    more exact sweep changes it by at most ||L|| times that (||L||_inf is near 1 for these
    scattering ratios; the DG operator is not monotone, so 1e-6, the bench's error target, is
    the bound checked)."""
    rte = _rte()
    train = inputs.lattice_train(128, 64)
    tb = rte.Batch.from_problem(train)
    rp, rc = rte.Rom.build(tb, eps_train=1e-12, window=3, rank_p=20, rank_c=20, max_iter=500,
                           dsa_rtol=1e-8)
    test = inputs.lattice_test(128, 64, 152)
    batch = rte.Batch(tb.disc, 152)
    batch.set_params(test)
    batch.autotune()
    rho = torch.zeros((152, test.n_dof), dtype=torch.float64, device="cuda")
    reps, _, st = batch.solve(rho, 2e-7, sa=rte.SA_ROMSAD, rel=True, max_iter=400, rom_c=rc,
                              theta=5, eps_romsad=0.1 * max(1e-12, rc.eps_pod), dsa_rtol=0.0,
                              dsa_max_it=1)
    assert st == rte.RTE_OK and all(r["converged"] for r in reps)
    got = rho.cpu().numpy()
    for b in (0, 151):
        tr = Transport(test, b)
        fixed = tr.sweep(got[b])
        assert _rel(fixed, got[b]) < 1e-6


def test_more_snapshots_than_one_kernel_chunk():
    """Correction snapshot sets larger than one chunk of the device POD (60 training instances,
    window 3: up to 180 columns): snapshot count and leading singular values as numpy's SVD."""
    rte = _rte()
    train = inputs.lattice_train(8, 8, n_train=60, n_vz=2)
    tb = rte.Batch.from_problem(train)
    rp, rc = rte.Rom.build(tb, eps_train=1e-12, window=3, rank_p=10, rank_c=30, max_iter=300,
                           dsa_rtol=1e-13)
    off = OfflineROMs(train, eps_train=1e-12, window=3, rank_p=10, rank_c=30)
    assert rc.n_snap == off.dF.shape[1] and rc.n_snap > 128
    np.testing.assert_allclose(rc.sv[:30], off.pod_c.sv[:30], atol=1e-10 * off.pod_c.sv[0])
    np.testing.assert_allclose(rp.sv[:10], off.pod_p.sv[:10], atol=1e-10 * off.pod_p.sv[0])
