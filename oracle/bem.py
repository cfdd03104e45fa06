"""The BEM-coupled FMM preconditioner z = M^-1 r (oracle, FP64).

Paper Sec. 5.2-5.3.  Green's representation, Eq. (bem); with u = 0 on the
boundary (reading S2) the boundary equation Eq. (ubound) becomes
  int_Gamma (du/dn) G dGamma = - int_Omega f G dOmega    on Gamma,
and the interior representation Eq. (uinter) becomes
  u = int_Gamma (du/dn) G dGamma + int_Omega f G dOmega  in Omega.
The preconditioner treats the residual r as f (reading S1: -Lap u - k^2 u = f,
so the volume term enters with a plus sign).  Discretised (Sec. 5.3; readings
B1 constant panels with a one-point rule off the diagonal, B2 midpoint volume
weights h^3, B3 singular diagonals by integration, B4 unpreconditioned inner
GMRES):

  Pass A   g = G_{Gamma Omega} w,            w = h^3 r
  inner    V q = -g,  V_ij = h^2 G(y_i, y_j) (i != j), V_ii = s_Gamma
  Pass C   z = G_{Omega Omega} w + G_{Omega Gamma} (h^2 q) + s_Omega r

Every G-sum is an FMM (Sec. 5.3: the FMM accelerates all the mat-vecs).
"""
from __future__ import annotations

import numpy as np

from . import geometry
from .fmm import FMM, direct_sum, self_panel, self_volume
from .gmres import fgmres


class Problem:
    """Interior nodes, boundary panels, tree and self terms for one (n, k)."""

    def __init__(self, n, k, p, leaf, theta):
        self.n, self.k, self.p, self.leaf, self.theta = n, k, p, leaf, theta
        self.h = 1.0 / (n + 1)
        self.x_vol = geometry.interior_nodes(n)
        self.x_bnd, self.n_bnd_normals = geometry.boundary_panels(n)
        self.NO = len(self.x_vol)
        self.NG = len(self.x_bnd)
        self.points = np.vstack([self.x_vol, self.x_bnd])
        self.vol = np.zeros(self.NO + self.NG, dtype=bool)
        self.vol[:self.NO] = True
        self.bnd = ~self.vol
        self.s_vol = self_volume(self.h, k)
        self.s_bnd = self_panel(self.h, k)
        h = self.h
        self.sigma = np.concatenate([np.full(self.NO, self.s_vol / h ** 3),
                                     np.full(self.NG, self.s_bnd / h ** 2)])
        self.fmm = FMM(self.points, self.NO, leaf, theta, k, p)

    def green(self, q_all, src, tgt, method):
        """G-sum over point weights q_all (length N_Omega + N_Gamma)."""
        if method == "fmm":
            return self.fmm.apply(q_all, src, tgt, self.sigma)
        return direct_sum(self.points, q_all, src, tgt, self.k, self.sigma)

    def precond(self, r, inner_rtol=1e-12, inner_maxit=200, inner_m=50,
                method="fmm", inner="gmres"):
        """z = M^-1 r for a residual r on the interior nodes.  Returns
        (z, inner_iterations)."""
        h = self.h
        NO = self.NO
        qa = np.zeros(NO + self.NG, dtype=np.complex128)
        qa[:NO] = h ** 3 * np.asarray(r)
        g = self.green(qa, self.vol, self.bnd, method)[NO:]          # Pass A

        def V(qb):                                                     # Pass B
            qq = np.zeros(NO + self.NG, dtype=np.complex128)
            qq[NO:] = h ** 2 * qb
            return self.green(qq, self.bnd, self.bnd, method)[NO:]

        if inner == "dense":
            Vm = np.stack([V(e) for e in np.eye(self.NG)], axis=1)
            q = np.linalg.solve(Vm, -g)
            its = 0
        else:
            q, info = fgmres(V, -g, None, m=inner_m, rtol=inner_rtol, maxit=inner_maxit)
            its = info["iters"]
        qa[NO:] = h ** 2 * q
        z = self.green(qa, self.vol | self.bnd, self.vol, method)[:NO]   # Pass C
        return z, its
