"""Consistent diffusion synthetic acceleration (paper App. B, used as stated in Sec. 4.1.1).

DSA replaces the kinetic correction equation (Eq. (discrete_correction)) by the system obtained
from the P1 ansatz delta f(x, v) = delta rho(x) + 3 v . delta J(x), substituted into the upwind
DG discretisation of the correction equation and integrated numerically against 1 and v over
the quadrature (App. B).  The oracle solves the resulting (rho, J) system with a sparse direct
solver, so its delta rho is the exact DSA correction.

1D (App. B, printed):
    D_C dJ - c1 D_J drho + Sigma_a drho = R,                 c1 = sum_{v_j>0} omega_j v_j
    c2 D_C drho + (Sigma_t - 3 c3 D_J) dJ = 0,               c2 = sum_j omega_j v_j^2,
                                                             c3 = sum_{v_j>0} omega_j v_j^3
with R = Sigma_s (rho^{(l,*)} - rho^{(l-1)}), D_C = (D^+ + D^-)/2, D_J = D^+ - D^-.

2D (not printed in the paper; the same steps applied to X-Y geometry).  Per axis d in {x, y},
D_j = sum_d v_d (D_{C,d} - sign(v_d)/2 D_{J,d}) with D_{C,d}, D_{J,d} built from the unit-
direction operators.  Taking the 0th and the v_x, v_y moments of
    (sum_d [v_d D_{C,d} - |v_d|/2 D_{J,d}] + Sigma_t)(drho + 3 v_x dJ_x + 3 v_y dJ_y)
        = Sigma_s drho + R
over a rule that is symmetric under v_x -> -v_x and v_y -> -v_y (CL with even N_phi) gives
    [Sigma_a - 1/2 <|v_x|> D_{J,x} - 1/2 <|v_y|> D_{J,y}] drho
        + 3<v_x^2> D_{C,x} dJ_x + 3<v_y^2> D_{C,y} dJ_y = R
    <v_x^2> D_{C,x} drho + [3<v_x^2> Sigma_t - 3/2 <|v_x|^3> D_{J,x} - 3/2 <v_x^2 |v_y|> D_{J,y}] dJ_x = 0
    <v_y^2> D_{C,y} drho + [3<v_y^2> Sigma_t - 3/2 <|v_y|^3> D_{J,y} - 3/2 <v_y^2 |v_x|> D_{J,x}] dJ_y = 0
where <.> = sum_j omega_j (.).  The v_z component of J decouples and vanishes.  All moments that
vanish by the rule's symmetry (<v_x>, <v_x v_y>, <v_x|v_x|>, ...) are dropped; a test checks
they are zero to rounding.  In 1D (v_y = 0) these equations are App. B's, with 3<v^2> = 1.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .transport import Transport


def moments_1d(v, w):
    xi = v[:, 0] if v.ndim == 2 else v
    pos = xi > 0
    c1 = float(np.sum(w[pos] * xi[pos]))
    c2 = float(np.sum(w * xi ** 2))
    c3 = float(np.sum(w[pos] * xi[pos] ** 3))
    return c1, c2, c3


def moments_2d(v, w):
    vx, vy = v[:, 0], v[:, 1]
    return dict(
        abs_x=float(np.sum(w * np.abs(vx))), abs_y=float(np.sum(w * np.abs(vy))),
        xx=float(np.sum(w * vx ** 2)), yy=float(np.sum(w * vy ** 2)),
        abs3_x=float(np.sum(w * np.abs(vx) ** 3)), abs3_y=float(np.sum(w * np.abs(vy) ** 3)),
        xx_absy=float(np.sum(w * vx ** 2 * np.abs(vy))),
        yy_absx=float(np.sum(w * vy ** 2 * np.abs(vx))),
    )


class ConsistentDSA:
    """delta rho = DSA correction for a given R = Sigma_s (rho* - rho_prev)."""

    def __init__(self, tr: Transport):
        self.tr = tr
        dg = tr.dg
        if tr.dim == 1:
            Dp, Dm = dg.appendix_b_D_plus_minus()
            Dp, Dm = sp.csr_matrix(Dp), sp.csr_matrix(Dm)
            DC = 0.5 * (Dp + Dm)
            DJ = Dp - Dm
            c1, c2, c3 = moments_1d(tr.v, tr.w)
            self.consts = (c1, c2, c3)
            M = sp.bmat([[tr.Sa - c1 * DJ, DC],
                         [c2 * DC, tr.St - 3.0 * c3 * DJ]], format="csc")
            self.n_fields = 2
        else:
            ops = dg.unit_direction_operators()
            DCx = 0.5 * (ops["x"][0] + ops["x"][1])
            DJx = ops["x"][0] - ops["x"][1]
            DCy = 0.5 * (ops["y"][0] + ops["y"][1])
            DJy = ops["y"][0] - ops["y"][1]
            m = moments_2d(tr.v, tr.w)
            self.consts = m
            self.ops = (DCx, DJx, DCy, DJy)
            A = tr.Sa - 0.5 * m["abs_x"] * DJx - 0.5 * m["abs_y"] * DJy
            Bx = 3.0 * m["xx"] * tr.St - 1.5 * m["abs3_x"] * DJx - 1.5 * m["xx_absy"] * DJy
            By = 3.0 * m["yy"] * tr.St - 1.5 * m["abs3_y"] * DJy - 1.5 * m["yy_absx"] * DJx
            M = sp.bmat([[A, 3.0 * m["xx"] * DCx, 3.0 * m["yy"] * DCy],
                         [m["xx"] * DCx, Bx, None],
                         [m["yy"] * DCy, None, By]], format="csc")
            self.n_fields = 3
        self.M = M
        self._lu = None

    def system(self):
        return self.M

    def solve_fields(self, R):
        """All fields (drho, dJ...) of the DSA system with right-hand side (R, 0, ...)."""
        if self._lu is None:
            self._lu = spla.splu(self.M)
        N = self.tr.n_dof
        rhs = np.zeros(self.n_fields * N)
        rhs[:N] = R
        return self._lu.solve(rhs)

    def correction(self, R):
        return self.solve_fields(R)[: self.tr.n_dof]
