"""The oracle's offline stage against the reduced dimensions the paper prints for its 1D
cross-regime problem (Sec. 4.1.1; values and citation in tests/golden/cross_regime_ranks.json).

The training solves (SI-DSA from rho = 0 to the paper's absolute tolerance 1e-11), the snapshot
matrices F and delta F, the thin SVD and the truncation rule of Eq. (pod_truncation) together
decide r_p and r_c; a mistake in any of them (a wrong window, a correction snapshot of the wrong
sign or iterate, squared singular values in the rule) moves these ranks.

Which iterates form the window.  Sec. 3.2.1 takes delta f^(l) = f - f^(l) for l = 1..w_mu, f^(l) the
angular flux of sweep l, and the oracle follows it.  With it, r_p and r_c(window 1) equal the
printed table at every eps_POD, and r_c(window 3) is one above it (16/19/22 against 15/18/21).
Shifting the window by one iterate (l = 0..w_mu - 1, with f^(0) = 0 for the zero start, so that the
first correction snapshot is f itself) reproduces the whole printed table exactly, window 1 included:
that pins the training iterates f, f^(1), f^(2), the SVD and the rule to the paper's numbers.  The
shifted window is not the method, though: with it, ROMSA-1's correction basis is the parametric
basis, and ROMSA-1 then fails to converge, where the paper reports it converging (7.05 sweeps at
eps_POD = 1e-11) and the text's window converges in a few sweeps; both are checked below.  The 41
independent training solves run in a pool of worker processes (started with spawn) to keep the
test within about half a minute."""
import json
import os
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

import numpy as np
import pytest

from oracle.rom import POD, ReducedModel, pod_rank
from oracle.sisa import sisa
from oracle.transport import Transport
from paper_2402_10488_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def _snapshots(mu):
    from oracle.rom import training_snapshots
    F, dF, n_conv, _ = training_snapshots(inputs.cross_regime(mu), 1e-11, 3)
    return F, dF, n_conv


@pytest.fixture(scope="module")
def training():
    mus = inputs.cross_regime_train()
    chunks = np.array_split(mus, min(8, os.cpu_count() or 1))
    with ProcessPoolExecutor(len(chunks), mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_snapshots, chunks))
    F = np.concatenate([p[0] for p in parts], 1)
    dF3 = np.concatenate([p[1] for p in parts], 1)
    n_conv = [n for p in parts for n in p[2]]
    assert F.shape[1] == 41 and all(n >= 3 for n in n_conv)
    assert dF3.shape[1] == 3 * 41
    # columns of training solve k: dF3[:, 3k + l - 1] = f_k - f_k^(l), l = 1, 2, 3
    dF1 = dF3[:, 0::3]
    shifted3 = np.stack([F, dF3[:, 0::3], dF3[:, 1::3]], 2).reshape(F.shape[0], -1)   # l = 0, 1, 2
    return F, dF1, dF3, shifted3


def test_cross_regime_reduced_dimensions(training):
    F, dF1, dF3, shifted3 = training
    gold = json.load(open(os.path.join(HERE, "golden", "cross_regime_ranks.json")))
    sv_p, sv_c1, sv_c3, sv_s3 = (np.linalg.svd(S, compute_uv=False) for S in (F, dF1, dF3, shifted3))
    for k, eps in enumerate(gold["eps_pod"]):
        assert pod_rank(sv_p, eps) == gold["r_p"][k], eps
        assert pod_rank(sv_c1, eps) == gold["r_c_window1"][k], eps
        # the shifted window: the printed table exactly (its window 1 is F itself, r_p)
        assert pod_rank(sv_s3, eps) == gold["r_c_window3"][k], eps
        # the text's window 3 holds f - f^(3) where the shifted one holds f: one more dimension
        assert pod_rank(sv_c3, eps) == gold["r_c_window3"][k] + 1, eps


def test_shifted_window_makes_romsa1_diverge(training):
    """ROMSA-1 at eps_POD = 1e-11 (r_c = 7) on one test slope: the text's correction basis converges
    within a few sweeps (the paper: 7.05 on average); the basis of the shifted window (POD of F, the
    solutions, not corrections) does not converge within 40 sweeps."""
    F, dF1, _, _ = training
    mu = inputs.cross_regime_test(1)
    prob = inputs.cross_regime(mu)
    tr = Transport(prob, 0)
    tr0 = Transport(inputs.cross_regime(inputs.cross_regime_train()[:1]), 0)
    text = ReducedModel(POD(dF1, 1e-11).U, tr0)
    shifted = ReducedModel(POD(F, 1e-11).U, tr0)
    assert text.r == shifted.r == 7
    res_text = sisa(tr, np.zeros(tr.n_dof), 1e-11, 40, "romsa", rom_c=text)
    res_shift = sisa(tr, np.zeros(tr.n_dof), 1e-11, 40, "romsa", rom_c=shifted)
    assert res_text["converged"] and res_text["n_sweep"] <= 10
    assert not res_shift["converged"]
