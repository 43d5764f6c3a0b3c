"""The oracle's offline stage against the reduced dimensions the paper prints for its 1D
cross-regime problem (Sec. 4.1.1; values and citation in tests/golden/cross_regime_ranks.json).

The training solves (SI-DSA from rho = 0 to the paper's absolute tolerance 1e-11), the snapshot
matrices F and delta F (window 1 and 3), the thin SVD and the truncation rule of Eq.
(pod_truncation) together decide r_p and r_c; a mistake in any of them (a wrong window, a
correction snapshot of the wrong sign or iterate, squared singular values in the rule) moves
these ranks.  r_p and r_c with window 1 must equal the paper's at all three tolerances; with
window 3 the oracle (and the GPU library) find one more dimension than the paper at each
tolerance, so that column is checked to within one.  The 41 independent training solves run in
a pool of worker processes (started with spawn) to keep the test within about half a minute."""
import json
import os
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

import numpy as np

from oracle.rom import pod_rank
from paper_2402_10488_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def _snapshots(mu):
    from oracle.rom import training_snapshots
    F, dF, n_conv, _ = training_snapshots(inputs.cross_regime(mu), 1e-11, 3)
    return F, dF, n_conv


def test_cross_regime_reduced_dimensions_match_the_paper():
    gold = json.load(open(os.path.join(HERE, "golden", "cross_regime_ranks.json")))
    mus = inputs.cross_regime_train()
    chunks = np.array_split(mus, min(8, os.cpu_count() or 1))
    with ProcessPoolExecutor(len(chunks), mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_snapshots, chunks))
    F = np.concatenate([p[0] for p in parts], 1)
    dF3 = np.concatenate([p[1] for p in parts], 1)
    n_conv = [n for p in parts for n in p[2]]
    assert F.shape[1] == 41 and all(n >= 3 for n in n_conv)
    # window 1: the first correction snapshot of every training solve
    first = np.cumsum([0] + [min(n, 3) for n in n_conv[:-1]])
    dF1 = dF3[:, first]
    sv_p, sv_c1, sv_c3 = (np.linalg.svd(S, compute_uv=False) for S in (F, dF1, dF3))
    for k, eps in enumerate(gold["eps_pod"]):
        assert pod_rank(sv_p, eps) == gold["r_p"][k], eps
        assert pod_rank(sv_c1, eps) == gold["r_c_window1"][k], eps
        assert abs(pod_rank(sv_c3, eps) - gold["r_c_window3"][k]) <= 1, eps
