"""Seeded synthetic workloads for the parametric radiative transfer equation.

This module is shared by the CPU oracle, the tests and ``bench.py``.  It only *describes*
problems: mesh sizes, the angular rule's name and sizes, a material map, per-instance cross
sections, a cellwise-constant isotropic source value and an isotropic inflow value per domain
side.  It holds none of the method's arithmetic (no quadrature nodes, no DG projections, no
matrices), so that the oracle and the CUDA path share inputs but no computation.

Problem statement: steady one-group RTE with isotropic scattering, isotropic source G and
isotropic inflow g (paper Sec. 2, Eq. (1); slab form Eq. (2)).  Cross sections are cellwise
constant: each cell carries a material id, each instance a table sigma_t[m], sigma_s[m].  In 1D a
second id per cell (``mat_id_right``) makes them linear across the cell, between the values of
the two materials at its ends.

Layout conventions (an interface, used identically by every consumer):
  * cell index ``c = j * nx + i`` (i along x, j along y; ny = 1 in 1D);
  * ``inflow`` sides are ordered (x-, x+, y-, y+) -- the value of g on the side where the
    particles enter the domain.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Sequence

import numpy as np

# Seeds: training and test parameter sets are disjoint (paper Sec. 4 requires
# P_train and P_test to be disjoint).
TRAIN_SEED0 = 1000
TEST_SEED0 = 2000
BATCH_SEED = 3000
SERVE_SEED = 5000


@dataclass
class Problem:
    """A batch of B parametric instances sharing mesh, angular rule and material map."""

    dim: int                      # 1 (slab) or 2 (X-Y geometry)
    nx: int
    ny: int                       # 1 when dim == 1
    domain: tuple                 # (x0, x1) in 1D, (x0, x1, y0, y1) in 2D
    quad: str                     # 'gl' (1D Gauss-Legendre) or 'cl' (2D Chebyshev-Legendre)
    n_phi: int                    # number of GL points (1D) or Chebyshev points N_phi (2D)
    n_vz: int                     # number of GL points in v_z (2D); 0 in 1D
    mat_id: np.ndarray            # int32 [n_cells]
    sigma_t: np.ndarray           # float64 [B, n_mat]
    sigma_s: np.ndarray           # float64 [B, n_mat]
    source: np.ndarray            # float64 [B, n_cells], cellwise-constant G
    inflow: np.ndarray            # float64 [B, 2*dim], isotropic inflow per side
    params: np.ndarray = field(default=None)  # float64 [B, p], the mu that made each instance
    name: str = ""
    edges: np.ndarray = field(default=None)   # 1D only: cell edges x_0 < ... < x_N (None: uniform)
    # 1D only: material at each cell's right end (None: mat_id).  Cross sections are then linear
    # across every cell, from the value of material mat_id[c] at its left end to that of
    # mat_id_right[c] at its right end.
    mat_id_right: np.ndarray = field(default=None)

    # ---- sizes -------------------------------------------------------------------------
    @property
    def n_cells(self) -> int:
        return self.nx * self.ny

    @property
    def n_mat(self) -> int:
        return int(self.sigma_t.shape[1])

    @property
    def batch(self) -> int:
        return int(self.sigma_t.shape[0])

    @property
    def n_angles(self) -> int:
        return self.n_phi if self.dim == 1 else self.n_phi * self.n_vz

    @property
    def dofs_per_cell(self) -> int:
        return 2 if self.dim == 1 else 4

    @property
    def n_dof(self) -> int:
        return self.n_cells * self.dofs_per_cell

    def instance(self, b: int) -> "Problem":
        """The b-th instance as a batch of one."""
        return self.subset([b])

    def subset(self, idx: Sequence[int]) -> "Problem":
        idx = list(idx)
        return replace(
            self,
            sigma_t=self.sigma_t[idx].copy(),
            sigma_s=self.sigma_s[idx].copy(),
            source=self.source[idx].copy(),
            inflow=self.inflow[idx].copy(),
            params=None if self.params is None else self.params[idx].copy(),
        )

    def validate(self) -> None:
        assert self.dim in (1, 2)
        assert self.mat_id.shape == (self.n_cells,)
        assert self.mat_id.min() >= 0 and self.mat_id.max() < self.n_mat
        if self.mat_id_right is not None:
            assert self.dim == 1 and self.mat_id_right.shape == (self.n_cells,)
            assert self.mat_id_right.min() >= 0 and self.mat_id_right.max() < self.n_mat
        B = self.batch
        assert self.sigma_s.shape == self.sigma_t.shape
        assert self.source.shape == (B, self.n_cells)
        assert self.inflow.shape == (B, 2 * self.dim)
        assert np.all(self.sigma_t > 0) and np.all(self.sigma_s >= 0)
        assert np.all(self.sigma_s <= self.sigma_t)


def _stack(rows) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(rows, dtype=np.float64))


# ---- 1D slab workloads ---------------------------------------------------------------------

def slab(n_cells: int, n_angles: int, sigma_t, sigma_s, G=1.0, inflow=(0.0, 0.0),
         domain=(0.0, 1.0), name="slab") -> Problem:
    """Homogeneous slab, one material; sigma_t/sigma_s may be sequences (one per instance)."""
    st = np.atleast_1d(np.asarray(sigma_t, dtype=np.float64))
    ss = np.atleast_1d(np.asarray(sigma_s, dtype=np.float64))
    B = max(st.size, ss.size)
    st = np.broadcast_to(st, (B,)).copy()
    ss = np.broadcast_to(ss, (B,)).copy()
    return Problem(
        dim=1, nx=n_cells, ny=1, domain=tuple(domain), quad="gl", n_phi=n_angles, n_vz=0,
        mat_id=np.zeros(n_cells, np.int32),
        sigma_t=st[:, None].copy(), sigma_s=ss[:, None].copy(),
        source=np.full((B, n_cells), float(G)),
        inflow=np.tile(_stack(inflow), (B, 1)),
        params=np.stack([st, ss], 1), name=name,
    )


def slab_diffusive(n_cells: int = 128, n_angles: int = 16, eps: float = 0.01) -> Problem:
    """Diffusive slab on [0,1]: sigma_t = 1/eps, sigma_a = eps, G = 1, vacuum inflow."""
    st = 1.0 / eps
    return slab(n_cells, n_angles, st, st - eps, G=1.0, name=f"slab{n_cells}_S{n_angles}_eps{eps}")


def slab_random(n_cells: int, n_angles: int, n_mat: int, seed: int, B: int = 1,
                inflow=(0.0, 0.0), linear: bool = False) -> Problem:
    """Slab with random per-cell materials (for parity tests): c = sigma_s/sigma_t in [0, 0.99].
    linear: a second random material per cell for its right end (cross sections linear across
    the cell; c stays in [0, 0.99] everywhere since both ends satisfy it)."""
    rng = np.random.default_rng(seed)
    mat = rng.integers(0, n_mat, n_cells).astype(np.int32)
    st = rng.uniform(0.5, 20.0, (B, n_mat))
    ss = st * rng.uniform(0.0, 0.99, (B, n_mat))
    G = rng.uniform(0.0, 2.0, (B, n_cells))
    mat_r = rng.integers(0, n_mat, n_cells).astype(np.int32) if linear else None
    return Problem(1, n_cells, 1, (0.0, 1.0), "gl", n_angles, 0, mat, st, ss, G,
                   np.tile(_stack(inflow), (B, 1)), None,
                   f"slab_random{seed}" + ("_linear" if linear else ""), mat_id_right=mat_r)


# ---- 2D lattice-cell workloads -------------------------------------------------------------

def lattice_map(n: int) -> np.ndarray:
    """Material id per cell of an n x n mesh of [0,1]^2: 1 inside the centred square inclusion
    of side 0.4, else 0.  A cell is inside iff its centre satisfies |x-0.5| < 0.2 and
    |y-0.5| < 0.2, decided in integers: 6n < 20i+10 < 14n (same for j)."""
    i = np.arange(n)
    inside_1d = (6 * n < 20 * i + 10) & (20 * i + 10 < 14 * n)
    inside = inside_1d[None, :] & inside_1d[:, None]  # [j, i]
    return inside.astype(np.int32).reshape(-1)


def lattice_params(seeds: Sequence[int]) -> np.ndarray:
    """mu = (mu_in, mu_out, mu_a): sigma_s ~ U[1,100] in the inclusion, U[0.1,1] outside,
    sigma_a ~ U[0.01,0.1] everywhere; one numpy Generator per seed."""
    out = []
    for s in seeds:
        rng = np.random.default_rng(int(s))
        out.append((rng.uniform(1.0, 100.0), rng.uniform(0.1, 1.0), rng.uniform(0.01, 0.1)))
    return _stack(out)


def lattice_from_params(n: int, n_phi: int, n_vz: int, mu: np.ndarray, G: float = 1.0,
                        name: str = "") -> Problem:
    mu = np.atleast_2d(np.asarray(mu, dtype=np.float64))
    B = mu.shape[0]
    mu_in, mu_out, mu_a = mu[:, 0], mu[:, 1], mu[:, 2]
    sigma_s = np.stack([mu_out, mu_in], 1)          # material 0 = outside, 1 = inclusion
    sigma_t = sigma_s + mu_a[:, None]
    return Problem(
        dim=2, nx=n, ny=n, domain=(0.0, 1.0, 0.0, 1.0), quad="cl", n_phi=n_phi, n_vz=n_vz,
        mat_id=lattice_map(n), sigma_t=sigma_t, sigma_s=sigma_s,
        source=np.full((B, n * n), float(G)), inflow=np.zeros((B, 4)), params=mu.copy(),
        name=name or f"lattice{n}_CL({n_phi},{n_vz})",
    )


def lattice(n: int, n_angles: int, seeds: Sequence[int], n_vz: int = 4) -> Problem:
    """Two-material lattice cell on [0,1]^2 with CL(n_angles/n_vz, n_vz), vacuum inflow, G=1."""
    assert n_angles % n_vz == 0
    return lattice_from_params(n, n_angles // n_vz, n_vz, lattice_params(seeds))


def lattice_train(n: int, n_angles: int, n_train: int = 32, n_vz: int = 4) -> Problem:
    return lattice(n, n_angles, [TRAIN_SEED0 + k for k in range(n_train)], n_vz)


def lattice_test(n: int, n_angles: int, n_test: int = 10, n_vz: int = 4, first: int = 0) -> Problem:
    return lattice(n, n_angles, [TEST_SEED0 + first + k for k in range(n_test)], n_vz)


def random_2d(n: int, n_phi: int, n_vz: int, n_mat: int, seed: int, B: int = 1,
              inflow=(0.0, 0.0, 0.0, 0.0), ny: int | None = None) -> Problem:
    """Random material map and cross sections on [0,1]^2 (for parity tests); c in [0, 0.99]."""
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    mat = rng.integers(0, n_mat, n * ny).astype(np.int32)
    st = rng.uniform(0.5, 60.0, (B, n_mat))
    ss = st * rng.uniform(0.0, 0.99, (B, n_mat))
    G = rng.uniform(0.0, 2.0, (B, n * ny))
    return Problem(2, n, ny, (0.0, 1.0, 0.0, 1.0), "cl", n_phi, n_vz, mat, st, ss, G,
                   np.tile(_stack(inflow), (B, 1)), None, f"random2d_{n}x{ny}_{seed}")


# ---- batched / serving workloads ------------------------------------------------------------

MESH_SIDES_BATCH = (64, 96, 128, 192)
ANGLES_BATCH = (32, 64, 128)


def mixed_batch_spec(n_instances: int = 256, seed: int = BATCH_SEED):
    """Per-instance (mesh side, angle count, mu) for the batched workload: side from
    {64,96,128,192}, angles from {32,64,128}, mu as in the lattice workload."""
    rng = np.random.default_rng(seed)
    sides = rng.choice(MESH_SIDES_BATCH, n_instances)
    angles = rng.choice(ANGLES_BATCH, n_instances)
    mu = np.stack([rng.uniform(1.0, 100.0, n_instances), rng.uniform(0.1, 1.0, n_instances),
                   rng.uniform(0.01, 0.1, n_instances)], 1)
    return [(int(s), int(a), mu[k]) for k, (s, a) in enumerate(zip(sides, angles))]


MESH_SIDES_SERVE = (64, 96, 128, 192, 256)
ANGLES_SERVE = (32, 64, 128, 256)
TOLS_SERVE = (1e-6, 1e-8)


def serving_requests(n_requests: int, rate: float = 2000.0, seed: int = SERVE_SEED):
    """Request stream of the serving workload: Poisson arrivals (exponential gaps, mean 1/rate
    seconds), mesh side from {64,...,256}, angles from {32,...,256}, mu as in the lattice
    workload, relative tolerance 1e-6 or 1e-8, all uniform.  Returns (t_arrival, side, angles,
    mu, tol) per request."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    sides = rng.choice(MESH_SIDES_SERVE, n_requests)
    angles = rng.choice(ANGLES_SERVE, n_requests)
    tols = rng.choice(TOLS_SERVE, n_requests)
    mu = np.stack([rng.uniform(1.0, 100.0, n_requests), rng.uniform(0.1, 1.0, n_requests),
                   rng.uniform(0.01, 0.1, n_requests)], 1)
    return [(float(t[k]), int(sides[k]), int(angles[k]), mu[k], float(tols[k]))
            for k in range(n_requests)]


# ---- the paper's 2D test problems (Sec. 4.2.1 homogeneous medium, Sec. 4.2.3 pin cell) --------

def cell_average(fn, nx: int, ny: int, domain, order: int = 4) -> np.ndarray:
    """Cell averages of a function on a uniform nx x ny mesh (cell index c = j*nx + i) by an
    order x order tensor Gauss-Legendre rule per cell (numpy's nodes)."""
    x0, x1, y0, y1 = domain
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    t, w = np.polynomial.legendre.leggauss(order)
    xs = x0 + hx * (np.arange(nx)[:, None] + 0.5 + 0.5 * t[None, :])   # [nx, order]
    ys = y0 + hy * (np.arange(ny)[:, None] + 0.5 + 0.5 * t[None, :])
    X = xs[None, :, None, :]
    Y = ys[:, None, :, None]
    vals = fn(X, Y)                                                       # [ny, nx, order, order]
    avg = 0.25 * np.einsum("jiab,a,b->ji", vals, w, w)
    return avg.reshape(-1)


def homogeneous_medium(mu_s, n: int = 80, n_phi: int = 30, n_vz: int = 6) -> Problem:
    """Sec. 4.2.1: [0,1]^2, sigma_a = 0, sigma_s = mu_s (one material), zero inflow,
    G = exp(-100((x-0.5)^2 + (y-0.5)^2)) taken cellwise constant (cell averages)."""
    mu_s = np.atleast_1d(np.asarray(mu_s, dtype=np.float64))
    B = mu_s.size
    dom = (0.0, 1.0, 0.0, 1.0)
    G = cell_average(lambda x, y: np.exp(-100.0 * ((x - 0.5) ** 2 + (y - 0.5) ** 2)), n, n, dom)
    return Problem(2, n, n, dom, "cl", n_phi, n_vz, np.zeros(n * n, np.int32), mu_s[:, None].copy(),
                   mu_s[:, None].copy(), np.tile(G, (B, 1)), np.zeros((B, 4)), mu_s[:, None].copy(),
                   f"homogeneous{n}_CL({n_phi},{n_vz})")


def homogeneous_train():
    """21 training values mu_s = 0.9 + m/200, m = 0..20 (Sec. 4.2.1)."""
    return 0.9 + np.arange(21) / 200.0


def homogeneous_test(n_test: int = 10, seed: int = TEST_SEED0):
    return np.random.default_rng(seed).uniform(0.9, 1.1, n_test)


def pin_cell_map(n: int) -> np.ndarray:
    """Material id on an n x n mesh of [-1,1]^2: 1 inside |x| <= 0.5 and |y| <= 0.5 (cell centre
    inside; mesh-aligned when n is a multiple of 4), else 0."""
    i = np.arange(n)
    c = -1.0 + (i + 0.5) * 2.0 / n
    inside = np.abs(c) <= 0.5
    return (inside[None, :] & inside[:, None]).astype(np.int32).reshape(-1)


def pin_cell(mu, n: int = 80, n_phi: int = 30, n_vz: int = 6) -> Problem:
    """Sec. 4.2.3: [-1,1]^2, zero inflow, G = exp(-100(x^2 + y^2)) (cell averages); inside the
    centre square sigma_a = mu_a, sigma_s = mu_s; outside sigma_a = 0, sigma_s = 100."""
    mu = np.atleast_2d(np.asarray(mu, dtype=np.float64))   # rows (mu_a, mu_s)
    B = mu.shape[0]
    dom = (-1.0, 1.0, -1.0, 1.0)
    G = cell_average(lambda x, y: np.exp(-100.0 * (x ** 2 + y ** 2)), n, n, dom)
    sigma_s = np.stack([np.full(B, 100.0), mu[:, 1]], 1)    # material 0 = outside, 1 = pin
    sigma_t = sigma_s + np.stack([np.zeros(B), mu[:, 0]], 1)
    return Problem(2, n, n, dom, "cl", n_phi, n_vz, pin_cell_map(n), sigma_t, sigma_s,
                   np.tile(G, (B, 1)), np.zeros((B, 4)), mu.copy(), f"pincell{n}_CL({n_phi},{n_vz})")


def pin_cell_train():
    """25 training pairs (mu_a, mu_s) = (0.05 i, 0.05 j), i, j = 1..5 (Sec. 4.2.3)."""
    return np.array([(0.05 * i, 0.05 * j) for i in range(1, 6) for j in range(1, 6)])


def pin_cell_test(n_test: int = 10, seed: int = TEST_SEED0):
    return np.random.default_rng(seed).uniform(0.05, 0.5, (n_test, 2))


# ---- the paper's 1D cross-regime problem (Sec. 4.1.1) -----------------------------------------

def cross_regime(mu_s, n: int = 400, n_angles: int = 16, linear: bool = True) -> Problem:
    """Sec. 4.1.1: slab [0,10], sigma_a = 0, sigma_s(x) = 0.1 + mu_s x, G = 0.01, vacuum inflow,
    n uniform cells, S_16.  linear: sigma_s is linear inside the cells as in the paper; the n + 1
    cell edges are the materials (material m holds sigma_s(x_m)) and cell c runs from material c
    to material c + 1.  Otherwise sigma_s is taken cellwise constant at its cell average (the
    value at the cell centre), every cell its own material."""
    mu_s = np.atleast_1d(np.asarray(mu_s, dtype=np.float64))
    B = mu_s.size
    name = f"cross_regime{n}_S{n_angles}"
    if linear:
        xe = np.arange(n + 1) * 10.0 / n
        sig = 0.1 + mu_s[:, None] * xe[None, :]
        return Problem(1, n, 1, (0.0, 10.0), "gl", n_angles, 0, np.arange(n, dtype=np.int32),
                       sig.copy(), sig.copy(), np.full((B, n), 0.01), np.zeros((B, 2)),
                       mu_s[:, None].copy(), name + "_linear",
                       mat_id_right=np.arange(1, n + 1, dtype=np.int32))
    xc = (np.arange(n) + 0.5) * 10.0 / n
    sig = 0.1 + mu_s[:, None] * xc[None, :]
    return Problem(1, n, 1, (0.0, 10.0), "gl", n_angles, 0, np.arange(n, dtype=np.int32), sig.copy(),
                   sig.copy(), np.full((B, n), 0.01), np.zeros((B, 2)), mu_s[:, None].copy(), name)


def cross_regime_train():
    """41 training slopes mu_s = 10 + j/4, j = 0..40 (Sec. 4.1.1)."""
    return 10.0 + np.arange(41) / 4.0


def cross_regime_test(n_test: int = 20, seed: int = TEST_SEED0):
    return np.random.default_rng(seed).uniform(10.0, 20.0, n_test)



# ---- the paper's 1D two-material problem (Sec. 4.1.2) -----------------------------------------

def two_material_edges():
    """Non-uniform mesh of Sec. 4.1.2: width 1/100 on [0,1], 1/10 on [1,11] (200 cells)."""
    return np.concatenate([np.arange(101) / 100.0, 1.0 + np.arange(1, 101) / 10.0])


def two_material(mu, n_angles: int = 16) -> Problem:
    """Sec. 4.1.2: slab [0,11]; on [0,1] sigma_a = mu_a, sigma_s = 0; on [1,11] sigma_a = 0,
    sigma_s = mu_s; G = 0; isotropic inflow 5 at x = 0 and 0 at x = 11; S_16."""
    mu = np.atleast_2d(np.asarray(mu, dtype=np.float64))   # rows (mu_a, mu_s)
    B = mu.shape[0]
    edges = two_material_edges()
    n = edges.size - 1
    mat = (edges[:-1] >= 1.0 - 1e-12).astype(np.int32)       # 0 absorber, 1 scatterer
    sigma_s = np.stack([np.zeros(B), mu[:, 1]], 1)
    sigma_t = sigma_s + np.stack([mu[:, 0], np.zeros(B)], 1)
    inflow = np.tile(np.array([5.0, 0.0]), (B, 1))
    return Problem(1, n, 1, (0.0, 11.0), "gl", n_angles, 0, mat, sigma_t, sigma_s,
                   np.zeros((B, n)), inflow, mu.copy(), f"two_material{n}_S{n_angles}", edges)


def two_material_train():
    """451 training pairs (mu_a, mu_s) = (0.5 + 0.1 m, 10 + n), m = 0..10, n = 0..40."""
    return np.array([(0.5 + 0.1 * m, 10.0 + k) for m in range(11) for k in range(41)])


def two_material_test(n_test: int = 20, seed: int = TEST_SEED0):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0.5, 1.5, n_test), rng.uniform(10.0, 50.0, n_test)], 1)


# ---- the paper's variable-scattering problem (Sec. 4.2.4) -----------------------------------

def variable_scattering_map(n: int = 80, levels: int = 64):
    """Material map and level values for sigma_s = mu_s f(x, y) + 0.1 on [-1,1]^2 with
    f = r^4 (2 - r^2)^2 for r <= 1 and 1 outside: f is averaged over each cell (4x4 Gauss rule) and
    the cell averages are grouped into `levels` equal-width bins of [0, 1] (f = 1 exactly, i.e.
    cells entirely outside the unit disc, gets a material of its own); each bin is a material whose
    f is the mean of its cells' averages."""
    dom = (-1.0, 1.0, -1.0, 1.0)

    def f(x, y):
        r2 = x * x + y * y
        return np.where(r2 <= 1.0, r2 * r2 * (2.0 - r2) ** 2, 1.0)

    avg = cell_average(f, n, n, dom)
    raw = np.where(avg >= 1.0 - 1e-15, levels, np.minimum((avg * levels).astype(int), levels - 1))
    used = np.unique(raw)
    mat = np.searchsorted(used, raw).astype(np.int32)
    fval = np.array([avg[raw == u].mean() for u in used])
    return mat, fval


def variable_scattering(mu_s, n: int = 80, n_phi: int = 30, n_vz: int = 6, levels: int = 64) -> Problem:
    """Sec. 4.2.4: [-1,1]^2, zero inflow, sigma_a = 0, sigma_s = mu_s f + 0.1 (levels of f as in
    variable_scattering_map), G = (10 / pi) exp(-100 (x^2 + y^2)) (cell averages)."""
    mu_s = np.atleast_1d(np.asarray(mu_s, dtype=np.float64))
    B = mu_s.size
    dom = (-1.0, 1.0, -1.0, 1.0)
    mat, fval = variable_scattering_map(n, levels)
    sig = mu_s[:, None] * fval[None, :] + 0.1
    G = cell_average(lambda x, y: 10.0 / np.pi * np.exp(-100.0 * (x ** 2 + y ** 2)), n, n, dom)
    return Problem(2, n, n, dom, "cl", n_phi, n_vz, mat, sig.copy(), sig.copy(), np.tile(G, (B, 1)),
                   np.zeros((B, 4)), mu_s[:, None].copy(), f"variable_scattering{n}_CL({n_phi},{n_vz})")


def variable_scattering_train():
    """50 training values uniformly spread over [49.9, 99.9] (Sec. 4.2.4)."""
    return np.linspace(49.9, 99.9, 50)


def variable_scattering_test(n_test: int = 10, seed: int = TEST_SEED0):
    return np.random.default_rng(seed).uniform(49.9, 99.9, n_test)
