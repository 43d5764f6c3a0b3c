"""Upwind discontinuous Galerkin matrices (paper Sec. 2.2 and App. B).

Discrete space: Q^K on each rectangle (Eq. (discrete_space)), K = 1 in all of the paper's tests
(Sec. 4), with an orthonormal basis on every cell (Sec. 2.2, "orthonormal basis").  Reading
taken for the basis: the scaled tensor Legendre polynomials
    phi_a(x) = sqrt((2a+1)/h) P_a(xi),  xi = 2 (x - x_c) / h,  a in {0, 1},
and in 2D phi_k(x, y) = phi^x_a(x) phi^y_b(y) with local index k = a + 2 b.

Global DOF index of local function k in cell c is c * P + k (P = 2 in 1D, 4 in 2D), cell index
c = j * nx + i.

Every matrix entry is computed from its integral definition by Gauss quadrature: the volume term
-int (v . grad phi_k) phi_l, the face term int H(v, phi_l, n) phi_k with the upwind flux
    H(v, f, n) = (v.n)/2 (f^+ + f^-) + |v.n|/2 (f^- - f^+)          (Eq. (upwind)),
the mass matrices int sigma phi_k phi_l, the source int G phi_k and the inflow term
-int g phi_k (v.n) over inflow boundary edges (Eq. (dg_matrix_vec) and the definitions under it).

Reading of the edge sum in Eq. (DG): the test function is discontinuous, so the sum over edges
is taken cell by cell -- each cell T^- integrates H(v, f, n) phi_k|_{T^-} over each of its own
edges with its own outward normal, skipping edges that lie on the inflow boundary.  In 1D this
reproduces App. B's D^+ and D^- exactly (checked by a test).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# textbook 3-point Gauss-Legendre on [-1, 1]; exact for polynomials of degree <= 5, which covers
# every product of two Q^1 functions (and their derivatives) per coordinate direction.
_GX = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
_GW = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])


def basis_1d(h: float, xi: np.ndarray):
    """Values and x-derivatives of the orthonormal P^1 basis on a cell of width h at local
    coordinates xi in [-1, 1].  Returns (vals[len(xi), 2], dvals[len(xi), 2])."""
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    s0 = np.sqrt(1.0 / h)
    s1 = np.sqrt(3.0 / h)
    vals = np.stack([s0 * np.ones_like(xi), s1 * xi], 1)
    dvals = np.stack([np.zeros_like(xi), s1 * np.ones_like(xi) * (2.0 / h)], 1)
    return vals, dvals


class DG1D:
    """Upwind DG-P^1 on a slab partition x_0 < x_1 < ... < x_N (App. B uses this setting)."""

    dim = 1
    P = 2

    def __init__(self, edges: np.ndarray):
        self.edges = np.asarray(edges, dtype=np.float64)
        self.nx = self.edges.size - 1
        self.ny = 1
        self.n_cells = self.nx
        self.n_dof = self.P * self.n_cells
        self.h = np.diff(self.edges)

    @classmethod
    def uniform(cls, n, x0=0.0, x1=1.0):
        return cls(np.linspace(x0, x1, n + 1))

    # -- local integrals ------------------------------------------------------------------
    def _vol_deriv(self, c):
        """int_{T_c} phi_k' phi_l dx, [k, l]."""
        h = self.h[c]
        vals, dvals = basis_1d(h, _GX)
        return (h / 2.0) * np.einsum("q,qk,ql->kl", _GW, dvals, vals)

    def _mass(self, c):
        h = self.h[c]
        vals, _ = basis_1d(h, _GX)
        return (h / 2.0) * np.einsum("q,qk,ql->kl", _GW, vals, vals)

    def _int_phi(self, c):
        h = self.h[c]
        vals, _ = basis_1d(h, _GX)
        return (h / 2.0) * np.einsum("q,qk->k", _GW, vals)

    def trace(self, c, side):
        """Values of cell c's basis at its left (side=-1) or right (side=+1) end."""
        return basis_1d(self.h[c], np.array([float(side)]))[0][0]

    # -- matrices -------------------------------------------------------------------------
    def transport_matrix(self, v) -> sp.csr_matrix:
        """D_j for direction cosine v (Eq. (dg_matrix_vec) definition of (D_j)_{kl})."""
        v = float(np.atleast_1d(v)[0])
        P, N = self.P, self.n_cells
        rows, cols, vals = [], [], []

        def add(ci, cj, blk):
            r = ci * P + np.arange(P)
            cc = cj * P + np.arange(P)
            rows.append(np.repeat(r, P))
            cols.append(np.tile(cc, P))
            vals.append(np.asarray(blk).reshape(-1))

        for c in range(N):
            add(c, c, -v * self._vol_deriv(c))
            for side in (-1, +1):              # left edge (n = -1), right edge (n = +1)
                vn = v * side
                nb = c + side
                boundary = nb < 0 or nb >= N
                own = self.trace(c, side)
                if boundary:
                    if vn < 0:                 # inflow boundary edge: moved to the right side
                        continue
                    add(c, c, (0.5 * vn + 0.5 * abs(vn)) * np.outer(own, own))
                    continue
                other = self.trace(nb, -side)  # neighbour's trace at the shared edge
                add(c, c, (0.5 * vn + 0.5 * abs(vn)) * np.outer(own, own))
                add(c, nb, (0.5 * vn - 0.5 * abs(vn)) * np.outer(own, other))
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n_dof, self.n_dof))
        return A.tocsr()

    def mass_matrix(self, sigma_cell, sigma_right=None) -> sp.csr_matrix:
        """int sigma phi_k phi_l (Sigma_t, Sigma_s).  sigma cellwise constant, or -- with
        sigma_right -- linear on every cell from sigma_cell[c] at its left end to sigma_right[c] at
        its right end (the paper's cross-regime problem has sigma_s linear in x, Sec. 4.1.1)."""
        if sigma_right is None:
            blocks = [sp.csr_matrix(float(sigma_cell[c]) * self._mass(c)) for c in range(self.n_cells)]
            return sp.csr_matrix(sp.block_diag(blocks, format="csr"))
        blocks = []
        for c in range(self.n_cells):
            h = self.h[c]
            vals, _ = basis_1d(h, _GX)
            sig = float(sigma_cell[c]) * 0.5 * (1.0 - _GX) + float(sigma_right[c]) * 0.5 * (1.0 + _GX)
            blocks.append(sp.csr_matrix((h / 2.0) * np.einsum("q,q,qk,ql->kl", _GW, sig, vals, vals)))
        return sp.csr_matrix(sp.block_diag(blocks, format="csr"))

    def source_vector(self, G_cell) -> np.ndarray:
        """(G)_k = int G phi_k with cellwise-constant G."""
        return np.concatenate([float(G_cell[c]) * self._int_phi(c) for c in range(self.n_cells)])

    def inflow_vector(self, v, g_sides) -> np.ndarray:
        """(g^bc_j)_k = -sum over inflow boundary edges of g phi_k (v . n); g_sides = (g(x_0), g(x_N))."""
        v = float(np.atleast_1d(v)[0])
        out = np.zeros(self.n_dof)
        if v > 0:   # enters at the left end, n = -1
            out[0:2] += -float(g_sides[0]) * self.trace(0, -1) * (v * -1.0)
        elif v < 0:  # enters at the right end, n = +1
            c = self.n_cells - 1
            out[2 * c:2 * c + 2] += -float(g_sides[1]) * self.trace(c, +1) * (v * 1.0)
        return out

    def net_upwind_outflow(self, v, f, g_sides) -> np.ndarray:
        """Per cell: sum over its two ends of (v.n) f_hat, f_hat the upwind point value (own
        trace where v.n > 0, the neighbour's where v.n < 0, g at an inflow end)."""
        v = float(np.atleast_1d(v)[0])
        N = self.n_cells
        fc = np.asarray(f).reshape(N, 2)
        out = np.zeros(N)
        for c in range(N):
            for side in (-1, +1):
                vn = v * side
                nb = c + side
                if vn > 0:
                    up = self.trace(c, side) @ fc[c]
                elif 0 <= nb < N:
                    up = self.trace(nb, -side) @ fc[nb]
                else:
                    up = float(g_sides[0] if side < 0 else g_sides[1])
                out[c] += vn * up
        return out

    # -- App. B operators, transcribed from their definitions -------------------------------
    def appendix_b_D_plus_minus(self):
        """(D^+)_{kl} = -sum_i int_{T_i} phi_k' phi_l + sum_{i=1}^{N-1} phi_l(x^+_{i+1/2}) phi_k(x^-_{i+1/2})
                        - sum_{i=1}^{N} phi_l(x^+_{i-1/2}) phi_k(x^+_{i-1/2}),
           (D^-)_{kl} = -sum_i int_{T_i} phi_k' phi_l + sum_{i=1}^{N} phi_l(x^-_{i+1/2}) phi_k(x^-_{i+1/2})
                        - sum_{i=2}^{N} phi_l(x^-_{i-1/2}) phi_k(x^+_{i-1/2})          (App. B).
        phi(x^-_{i+1/2}) is the trace of cell i at its right end, phi(x^+_{i-1/2}) the trace of
        cell i at its left end (1-based cell i, 0-based c = i - 1)."""
        N, P = self.n_cells, self.P
        Dp = np.zeros((self.n_dof, self.n_dof))
        Dm = np.zeros((self.n_dof, self.n_dof))

        def right_end(i):   # global vector of all basis values at x^-_{i+1/2}: cell i's right end
            g = np.zeros(self.n_dof)
            g[(i - 1) * P:(i - 1) * P + P] = self.trace(i - 1, +1)
            return g

        def left_end(i):    # values at x^+_{i-1/2}: cell i's left end
            g = np.zeros(self.n_dof)
            g[(i - 1) * P:(i - 1) * P + P] = self.trace(i - 1, -1)
            return g

        vol = sp.block_diag([sp.csr_matrix(self._vol_deriv(c)) for c in range(N)]).toarray()
        Dp -= vol
        Dm -= vol
        for i in range(1, N):          # x^+_{i+1/2} is cell (i+1)'s left end
            Dp += np.outer(right_end(i), left_end(i + 1))   # [k, l] = phi_k(x^-) phi_l(x^+)
        for i in range(1, N + 1):
            Dp -= np.outer(left_end(i), left_end(i))
            Dm += np.outer(right_end(i), right_end(i))
        for i in range(2, N + 1):      # x^-_{i-1/2} is cell (i-1)'s right end
            Dm -= np.outer(left_end(i), right_end(i - 1))   # [k, l] = phi_k(x^+) phi_l(x^-)
        return Dp, Dm


class DG2D:
    """Upwind DG-Q^1 on a uniform nx x ny Cartesian mesh of [x0,x1] x [y0,y1]."""

    dim = 2
    P = 4

    # faces: name, outward normal, neighbour offset (di, dj), own local coord on the face,
    # neighbour local coord on the face, index of the coordinate that varies along the face
    _FACES = (
        ("W", (-1.0, 0.0), (-1, 0), ("xi", -1.0), ("xi", +1.0)),
        ("E", (+1.0, 0.0), (+1, 0), ("xi", +1.0), ("xi", -1.0)),
        ("S", (0.0, -1.0), (0, -1), ("eta", -1.0), ("eta", +1.0)),
        ("N", (0.0, +1.0), (0, +1), ("eta", +1.0), ("eta", -1.0)),
    )

    def __init__(self, nx, ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0):
        self.nx, self.ny = nx, ny
        self.x0, self.x1, self.y0, self.y1 = x0, x1, y0, y1
        self.hx = (x1 - x0) / nx
        self.hy = (y1 - y0) / ny
        self.n_cells = nx * ny
        self.n_dof = self.P * self.n_cells
        self._local()

    def _phi(self, xi, eta):
        """phi_k at local points (xi[q], eta[q]); k = a + 2b.  Returns vals, d/dx, d/dy [q, 4]."""
        vx, dx = basis_1d(self.hx, xi)
        vy, dy = basis_1d(self.hy, eta)
        vals = np.zeros((xi.size, 4))
        ddx = np.zeros((xi.size, 4))
        ddy = np.zeros((xi.size, 4))
        for b in range(2):
            for a in range(2):
                k = a + 2 * b
                vals[:, k] = vx[:, a] * vy[:, b]
                ddx[:, k] = dx[:, a] * vy[:, b]
                ddy[:, k] = vx[:, a] * dy[:, b]
        return vals, ddx, ddy

    def _local(self):
        """Reference-cell integrals (all cells of a uniform mesh share them)."""
        XI, ETA = np.meshgrid(_GX, _GX, indexing="ij")
        W = np.outer(_GW, _GW).reshape(-1) * (self.hx / 2.0) * (self.hy / 2.0)
        vals, ddx, ddy = self._phi(XI.reshape(-1), ETA.reshape(-1))
        self.mass_local = np.einsum("q,qk,ql->kl", W, vals, vals)
        self.int_phi = np.einsum("q,qk->k", W, vals)
        self.vol_x = np.einsum("q,qk,ql->kl", W, ddx, vals)  # int d_x phi_k phi_l
        self.vol_y = np.einsum("q,qk,ql->kl", W, ddy, vals)
        self.face = {}
        for name, n, off, own, oth in self._FACES:
            if own[0] == "xi":            # vertical edge, points vary in eta (y)
                wq = _GW * self.hy / 2.0
                ov, _, _ = self._phi(np.full(3, own[1]), _GX)
                nv, _, _ = self._phi(np.full(3, oth[1]), _GX)
            else:                         # horizontal edge, points vary in xi (x)
                wq = _GW * self.hx / 2.0
                ov, _, _ = self._phi(_GX, np.full(3, own[1]))
                nv, _, _ = self._phi(_GX, np.full(3, oth[1]))
            self.face[name] = dict(
                normal=np.array(n), off=off, wq=wq, own_vals=ov, nb_vals=nv,
                own_own=np.einsum("q,qk,ql->kl", wq, ov, ov),
                own_nb=np.einsum("q,qk,ql->kl", wq, ov, nv),
                int_own=np.einsum("q,qk->k", wq, ov),
            )

    def _cells(self):
        j, i = np.divmod(np.arange(self.n_cells), self.nx)
        return i, j

    def _assemble(self, blocks):
        """blocks: list of (row_cells[array], col_cells[array], 4x4 block or [n,4,4])."""
        P = self.P
        rows, cols, vals = [], [], []
        kk, ll = np.meshgrid(np.arange(P), np.arange(P), indexing="ij")
        for rc, cc, blk in blocks:
            rc = np.asarray(rc)
            cc = np.asarray(cc)
            b = np.broadcast_to(blk, (rc.size, P, P))
            rows.append((rc[:, None, None] * P + kk[None]).reshape(-1))
            cols.append((cc[:, None, None] * P + ll[None]).reshape(-1))
            vals.append(b.reshape(-1))
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n_dof, self.n_dof))
        return A.tocsr()

    def transport_matrix(self, v) -> sp.csr_matrix:
        """D_j for direction v = (v_x, v_y[, v_z]) (Eq. (dg_matrix_vec) definition of (D_j)_{kl})."""
        vx, vy = float(v[0]), float(v[1])
        i, j = self._cells()
        c = np.arange(self.n_cells)
        blocks = [(c, c, -(vx * self.vol_x + vy * self.vol_y))]
        for name, _, off, _, _ in self._FACES:
            f = self.face[name]
            vn = vx * f["normal"][0] + vy * f["normal"][1]
            ni, nj = i + off[0], j + off[1]
            interior = (ni >= 0) & (ni < self.nx) & (nj >= 0) & (nj < self.ny)
            own_coef = 0.5 * vn + 0.5 * abs(vn)
            nb_coef = 0.5 * vn - 0.5 * abs(vn)
            ci = c[interior]
            blocks.append((ci, ci, own_coef * f["own_own"]))
            blocks.append((ci, nj[interior] * self.nx + ni[interior], nb_coef * f["own_nb"]))
            if vn >= 0:                   # boundary edge that is not an inflow edge
                cb = c[~interior]
                blocks.append((cb, cb, own_coef * f["own_own"]))
        return self._assemble(blocks)

    def mass_matrix(self, sigma_cell) -> sp.csr_matrix:
        c = np.arange(self.n_cells)
        blk = np.asarray(sigma_cell, dtype=np.float64)[:, None, None] * self.mass_local[None]
        return self._assemble([(c, c, blk)])

    def source_vector(self, G_cell) -> np.ndarray:
        return (np.asarray(G_cell, dtype=np.float64)[:, None] * self.int_phi[None]).reshape(-1)

    def inflow_vector(self, v, g_sides) -> np.ndarray:
        """(g^bc_j)_k = -sum_{inflow boundary edges} int g phi_k (v . n); g per side (x-, x+, y-, y+)."""
        vx, vy = float(v[0]), float(v[1])
        i, j = self._cells()
        out = np.zeros((self.n_cells, 4))
        side_of = {"W": 0, "E": 1, "S": 2, "N": 3}
        for name, _, off, _, _ in self._FACES:
            f = self.face[name]
            vn = vx * f["normal"][0] + vy * f["normal"][1]
            if vn >= 0:
                continue
            ni, nj = i + off[0], j + off[1]
            bnd = ~((ni >= 0) & (ni < self.nx) & (nj >= 0) & (nj < self.ny))
            out[bnd] += -float(g_sides[side_of[name]]) * vn * f["int_own"][None]
        return out.reshape(-1)

    def net_upwind_outflow(self, v, f, g_sides) -> np.ndarray:
        """Per cell: int_{dT} (v.n) f_hat over its four edges, f_hat the upwind trace (own trace
        where v.n > 0, the neighbour's where v.n < 0, the inflow value g on inflow boundary
        edges).  Evaluated from traces at edge Gauss points, independently of D_j."""
        vx, vy = float(v[0]), float(v[1])
        i, j = self._cells()
        fc = np.asarray(f).reshape(self.n_cells, 4)
        out = np.zeros(self.n_cells)
        side_of = {"W": 0, "E": 1, "S": 2, "N": 3}
        for name, _, off, _, _ in self._FACES:
            fa = self.face[name]
            vn = vx * fa["normal"][0] + vy * fa["normal"][1]
            ni, nj = i + off[0], j + off[1]
            interior = (ni >= 0) & (ni < self.nx) & (nj >= 0) & (nj < self.ny)
            own_tr = fc @ fa["own_vals"].T                      # [cell, q]
            nb_idx = np.where(interior, nj * self.nx + ni, 0)
            nb_tr = fc[nb_idx] @ fa["nb_vals"].T
            if vn > 0:
                up = own_tr
            else:
                up = np.where(interior[:, None], nb_tr, float(g_sides[side_of[name]]))
            out += vn * (up @ fa["wq"])
        return out

    def unit_direction_operators(self):
        """2D analogues of App. B's D^+ and D^-, one pair per axis, from the general assembly:
        D^-_d = D(v = e_d) (upwind from the low side), D^+_d = -D(v = -e_d), so that
        D_j = v_d D^-_d for v_d > 0 and v_d D^+_d for v_d < 0 on each axis's terms, as in 1D."""
        out = {}
        for d, e in (("x", (1.0, 0.0)), ("y", (0.0, 1.0))):
            Dm = self.transport_matrix(e)
            Dp = -self.transport_matrix((-e[0], -e[1]))
            out[d] = (Dp, Dm)
        return out


def make_dg(problem):
    """DG object for a Problem description (paper's meshes are uniform; 1D may be non-uniform)."""
    if problem.dim == 1:
        if getattr(problem, "edges", None) is not None:
            return DG1D(problem.edges)
        x0, x1 = problem.domain[:2]
        return DG1D.uniform(problem.nx, x0, x1)
    x0, x1, y0, y1 = problem.domain
    return DG2D(problem.nx, problem.ny, x0, x1, y0, y1)
