"""Pins for the oracle's DG matrices (Sec. 2.2, App. B): the printed App. B operators, the
upwind decomposition D_j = v (D_C - sign(v)/2 D_J), symmetry of D_J / skewness of D_C,
orthonormality, and a hand-derived closed form of the 1D cell matrix."""
import numpy as np
import pytest

from oracle.dg import DG1D, DG2D
from oracle.quadrature import chebyshev_legendre, gauss_legendre


def test_general_assembly_equals_appendix_b_operators_nonuniform():
    edges = np.array([0.0, 0.1, 0.35, 0.4, 1.0, 1.7, 2.0])
    dg = DG1D(edges)
    Dp, Dm = dg.appendix_b_D_plus_minus()
    # App. B: D_j = v D^- for v > 0 and v D^+ for v < 0
    for v in (0.3, 1.0, 0.97):
        np.testing.assert_allclose(dg.transport_matrix(v).toarray(), v * Dm, atol=1e-13)
        np.testing.assert_allclose(dg.transport_matrix(-v).toarray(), -v * Dp, atol=1e-13)


def test_1d_upwind_decomposition_and_symmetries():
    dg = DG1D.uniform(9, 0.0, 2.0)
    Dp, Dm = dg.appendix_b_D_plus_minus()
    DC, DJ = 0.5 * (Dp + Dm), Dp - Dm
    xi, _ = gauss_legendre(16)
    for v in xi:
        np.testing.assert_allclose(dg.transport_matrix(v).toarray(),
                                   v * (DC - np.sign(v) / 2 * DJ), atol=1e-12)
    np.testing.assert_allclose(DJ, DJ.T, atol=1e-13)
    assert np.max(np.linalg.eigvalsh(DJ)) < 1e-12            # negative semidefinite
    np.testing.assert_allclose(DC, -DC.T, atol=1e-13)         # skew


def test_1d_cell_matrix_closed_form():
    """Hand derivation for the orthonormal P^1 basis on a cell of width h, v > 0: the cell's
    block of D_j + sigma I is (v/h) [[1, sqrt3], [-sqrt3, 3]] + sigma I and its coupling to the
    upwind neighbour is -(v/h) [[1, sqrt3], [-sqrt3, -3]]."""
    h, v = 0.25, 0.7
    dg = DG1D.uniform(4, 0.0, 1.0)
    D = dg.transport_matrix(v).toarray()
    s3 = np.sqrt(3.0)
    np.testing.assert_allclose(D[2:4, 2:4], v / h * np.array([[1, s3], [-s3, 3]]), atol=1e-13)
    np.testing.assert_allclose(D[2:4, 0:2], -v / h * np.array([[1, s3], [-s3, -3]]), atol=1e-13)
    assert np.all(D[0:2, 2:] == 0)


def test_2d_upwind_decomposition_and_symmetries():
    dg = DG2D(5, 4, 0.0, 1.0, 0.0, 0.8)
    ops = dg.unit_direction_operators()
    DCx, DJx = 0.5 * (ops["x"][0] + ops["x"][1]), ops["x"][0] - ops["x"][1]
    DCy, DJy = 0.5 * (ops["y"][0] + ops["y"][1]), ops["y"][0] - ops["y"][1]
    v, _ = chebyshev_legendre(8, 2)
    for d in v:
        ref = d[0] * (DCx - np.sign(d[0]) / 2 * DJx) + d[1] * (DCy - np.sign(d[1]) / 2 * DJy)
        np.testing.assert_allclose(dg.transport_matrix(d).toarray(), ref.toarray(), atol=1e-12)
    for DC, DJ in ((DCx, DJx), (DCy, DJy)):
        DC, DJ = DC.toarray(), DJ.toarray()
        np.testing.assert_allclose(DJ, DJ.T, atol=1e-13)
        assert np.max(np.linalg.eigvalsh(DJ)) < 1e-12
        np.testing.assert_allclose(DC, -DC.T, atol=1e-13)


@pytest.mark.parametrize("dg", [DG1D(np.array([0.0, 0.2, 0.7, 1.0])), DG2D(3, 2, 0.0, 0.6, 0.0, 1.0)])
def test_orthonormal_basis(dg):
    n = dg.n_cells
    M = dg.mass_matrix(np.ones(n)).toarray()
    np.testing.assert_allclose(M, np.eye(dg.n_dof), atol=1e-14)
    area = dg.h if dg.dim == 1 else np.full(n, dg.hx * dg.hy)
    g = dg.source_vector(np.ones(n)).reshape(n, dg.P)
    np.testing.assert_allclose(g[:, 0], np.sqrt(area), atol=1e-15)
    np.testing.assert_allclose(g[:, 1:], 0.0, atol=1e-15)
