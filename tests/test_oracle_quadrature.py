"""Pins for the oracle's S_N rules (Sec. 2.1) against numpy's Gauss-Legendre, exactness on
monomials and closed-form node values."""
import json
import os

import numpy as np
import pytest

from oracle.quadrature import chebyshev_legendre, gauss_legendre

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8, 16, 20])
def test_gauss_legendre_matches_numpy_and_is_normalised(n):
    x, w = gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=2e-15)
    np.testing.assert_allclose(w, 0.5 * wr, atol=2e-15)
    assert abs(w.sum() - 1.0) < 1e-15


@pytest.mark.parametrize("n", [2, 5, 16])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 1.0 / (k + 1)     # (1/2) int_{-1}^{1} x^k dx
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    # degree 2n is not integrated exactly
    assert abs(np.dot(w, x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-12


def test_cl_golden_values():
    """CL(4,2): every component of every direction is +-1/sqrt(3), weights 1/8 (closed form:
    phi = pi/4 + k pi/2, v_z = +-1/sqrt(3), sqrt(1 - 1/3) cos(pi/4) = 1/sqrt(3))."""
    with open(os.path.join(GOLDEN, "cl_4_2.json")) as fh:
        g = json.load(fh)
    v, w = chebyshev_legendre(4, 2)
    np.testing.assert_allclose(v, np.array(g["v"]), atol=1e-15)
    np.testing.assert_allclose(w, np.array(g["w"]), atol=1e-15)


@pytest.mark.parametrize("nphi,nvz", [(4, 2), (8, 4), (16, 4), (30, 6), (32, 4)])
def test_cl_moments_and_symmetry(nphi, nvz):
    v, w = chebyshev_legendre(nphi, nvz)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)
    # second moments of the uniform measure on S^2: <v_d^2> = 1/3
    for d in range(3):
        assert abs(np.dot(w, v[:, d] ** 2) - 1.0 / 3.0) < 1e-15
    vx, vy, vz = v.T
    # odd moments dropped in the 2D DSA derivation vanish by the rule's reflection symmetry
    for q in (vx, vy, vx * vy, np.abs(vx) * vx, np.abs(vx) * vy, vx ** 2 * vy, vx * vy ** 2,
              vx * np.abs(vy), vx * np.abs(vx) * vy, vx * np.abs(vy) * vy, vz * np.abs(vx) * vz * vx):
        assert abs(np.dot(w, q)) < 1e-15
    # index order j = (j2-1) N_phi + j1: the first N_phi directions share the lowest v_z
    assert np.all(v[:nphi, 2] == v[0, 2]) and v[0, 2] < 0
