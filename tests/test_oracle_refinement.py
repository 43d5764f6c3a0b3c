"""Pins, on the CPU, for the mathematics behind the precision variant's FP64 outer residual
correction (not a method of the paper: a way of running its source iteration in low precision).

* The sweep is affine in rho: sweep(rho) = sweep(x0) + L (rho - x0) for any x0 (Eq.
  (rho_matrix_vec_def): sweep(rho) = L rho + b-bar).  The FP32 correction sweeps rely on exactly
  this: they add y0 = sweep(x0) in FP64 to a low-precision L applied to the small rho - x0.
* With the inner operator perturbed at low precision (here: every input and output of L rounded
  to 8 significant bits, BF16-like, so that the effect is large and visible), plain SI-DSA stalls
  at the perturbed operator's fixed point, far from the FP64 solution, while the outer loop --
  an FP64 residual r = sweep(x0) - x0, then low-precision SI-DSA iterations on (I - L) e = r, then
  x0 + e -- reaches the FP64 solution to the FP64 level.  The test implements that loop itself
  (this file is the only place it exists outside the CUDA library) and compares with the oracle's
  direct solve of (I - L) rho = b-bar.
"""
import numpy as np
import pytest

from oracle.dsa import ConsistentDSA
from oracle.transport import Transport
from paper_2402_10488_gb300 import inputs


def _round_bits(x, bits=8):
    """x rounded to `bits` significant bits (round to nearest), elementwise."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.round(m * 2.0 ** bits) / 2.0 ** bits, e)


def _problems():
    return [inputs.slab_random(24, 8, 3, seed=11, inflow=(0.7, 0.2)),
            inputs.random_2d(6, 4, 2, 2, seed=12, inflow=(0.4, 0.0, 1.1, 0.3))]


@pytest.mark.parametrize("k", [0, 1])
def test_sweep_is_affine_in_rho(k):
    tr = Transport(_problems()[k])
    rng = np.random.default_rng(3)
    x0, rho = rng.uniform(0, 1, tr.n_dof), rng.uniform(0, 1, tr.n_dof)
    lhs = tr.sweep(rho)
    rhs = tr.sweep(x0) + tr.L(rho - x0)
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(lhs).max()


@pytest.mark.parametrize("k", [0, 1])
def test_outer_residual_correction_reaches_the_fp64_solution_where_low_precision_si_stalls(k):
    tr = Transport(_problems()[k])
    dsa = ConsistentDSA(tr)
    exact = tr.solve_rho_direct()
    bbar = tr.bbar()
    L_lo = lambda v: _round_bits(tr.L(_round_bits(v)))   # the low-precision operator

    # plain SI-DSA with the low-precision operator throughout: stalls at its own fixed point
    rho = np.zeros(tr.n_dof)
    for _ in range(60):
        star = L_lo(rho) + _round_bits(bbar)
        rho = star + dsa.correction(tr.Ss @ (star - rho))
    err_lo = np.abs(rho - exact).max() / np.abs(exact).max()
    assert err_lo > 1e-5

    # outer loop: FP64 residual of x0, low-precision SI-DSA on (I - L) e = r, x0 += e
    x0 = np.zeros(tr.n_dof)
    outer = []
    for _ in range(12):
        r = tr.sweep(x0) - x0                     # FP64 sweep: the residual of (I - L) rho = b-bar
        outer.append(np.abs(r).max() / np.abs(x0 + r).max())
        if outer[-1] < 1e-14:
            break
        e = np.zeros(tr.n_dof)
        for _ in range(6):
            e_star = L_lo(e) + r
            e = e_star + dsa.correction(tr.Ss @ (e_star - e))
        x0 = x0 + e
    err = np.abs(x0 - exact).max() / np.abs(exact).max()
    assert err < 1e-12, (err, outer)
    # each outer step shrinks the FP64 residual by a large factor until round-off
    assert all(b < 0.1 * a for a, b in zip(outer, outer[1:]) if b > 1e-13)
