"""Angular quadrature rules of the S_N discretisation (paper Sec. 2.1).

Weights are normalised so that sum_j omega_j = 1, i.e. the rule approximates the normalised
integral (1/4pi) int_{S^2} f dv (2D) or (1/2) int_{-1}^{1} f dxi (1D slab, Eq. (2)).
"""
from __future__ import annotations

import numpy as np


def legendre_and_derivative(n: int, x: np.ndarray):
    """P_n(x) and P_n'(x) by the three-term recurrence (k+1)P_{k+1} = (2k+1)xP_k - kP_{k-1}."""
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    # derivative: (1 - x^2) P_n' = n (P_{n-1} - x P_n)
    dp = n * (p0 - x * p1) / (1.0 - x * x)
    return p1, dp


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1,1] normalised to sum 1 (Sec. 2.1: the 1D slab uses
    Gauss-Legendre points; normalised weights are half the textbook ones).

    Nodes: roots of P_n found by Newton's method from the Chebyshev-like initial guess
    cos(pi (i - 1/4) / (n + 1/2)); textbook weights 2 / ((1 - x^2) P_n'(x)^2).
    Returned in ascending order."""
    i = np.arange(1, n + 1)
    x = np.cos(np.pi * (i - 0.25) / (n + 0.5))
    for _ in range(100):
        p, dp = legendre_and_derivative(n, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p, dp = legendre_and_derivative(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], 0.5 * w[order]


def slab_rule(n: int):
    """1D slab S_N rule: directions xi_j (cosines) and weights omega_j, sum omega_j = 1."""
    return gauss_legendre(n)


def chebyshev_legendre(n_phi: int, n_vz: int):
    """CL(N_phi, N_vz) product rule on S^2 (Sec. 2.1):
        phi_{j1} = 2 j1 pi / N_phi - pi / N_phi,  omega^phi = 1 / N_phi,
        v_j = (cos(phi_{j1}) sqrt(1 - vz_{j2}^2), sin(phi_{j1}) sqrt(1 - vz_{j2}^2), vz_{j2}),
        omega_j = omega^phi_{j1} omega^{vz}_{j2},  j = (j2 - 1) N_phi + j1  (1-based).
    Returns v [N_phi*N_vz, 3] and omega [N_phi*N_vz] in that index order."""
    j1 = np.arange(1, n_phi + 1)
    phi = 2.0 * j1 * np.pi / n_phi - np.pi / n_phi
    vz, wz = gauss_legendre(n_vz)
    v = np.zeros((n_phi * n_vz, 3))
    w = np.zeros(n_phi * n_vz)
    for j2 in range(n_vz):
        s = np.sqrt(1.0 - vz[j2] ** 2)
        for a in range(n_phi):
            j = j2 * n_phi + a
            v[j] = (np.cos(phi[a]) * s, np.sin(phi[a]) * s, vz[j2])
            w[j] = (1.0 / n_phi) * wz[j2]
    return v, w


def rule_for(problem):
    """Directions and weights for a Problem description: 1D returns v[:,0] = xi."""
    if problem.dim == 1:
        xi, w = slab_rule(problem.n_phi)
        v = np.zeros((xi.size, 3))
        v[:, 0] = xi
        return v, w
    return chebyshev_legendre(problem.n_phi, problem.n_vz)
