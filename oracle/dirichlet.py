"""Inhomogeneous Dirichlet data: the double-layer term (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package header): only tests/ use it.

Paper Sec. 5.2, Green's representation Eq. (bem) for -Lap u - k^2 u = f
(reading S1), with eta = 1 in Omega and 1/2 on the (flat part of the)
boundary, and its two uses for Dirichlet data u = u_Gamma:

  Eq. (ubound)  int_Gamma (du/dn) G = int_Gamma u (delta/2 + dG/dn) - int_Omega f G   on Gamma
  Eq. (uinter)  u = int_Gamma (du/dn) G - int_Gamma u dG/dn + int_Omega f G             in Omega

The paper's third model problem (Sec. 6) is the 2D instance with
inhomogeneous Dirichlet data.  The normal derivative of the 3D kernel (Sec.
5.2) is taken with the factor dr/dn_y that the 2D form keeps (reading S3):

  dG/dn_y (x, y) = (i k r - 1) e^{i k r} / (4 pi r^2) * (y - x).n_y / r,   r = |x - y|,

n_y the outward unit normal at the source point y.

Discretisation (Sec. 5.3; readings B1, B2): constant panels of area h^2 at
the boundary grid nodes off the edges, one-point rule off the diagonal,
midpoint volume weights h^3.  The double-layer matrix is
  D_ij = h^2 dG/dn_y(x_i, y_j)  (i != j),   D_ii = 0,
the diagonal being zero because (y - x).n_y vanishes over a point's own flat
panel (the principal value; the jump is the separate delta/2 term).  With
q = du/dn on the panels and V, N the single-layer and volume G-sums of the
homogeneous preconditioner (module bem):

  boundary    V q = u_Gamma / 2 + D_{Gamma Gamma} u_Gamma - N_{Gamma Omega} f
  interior    u   = V_{Omega Gamma} q - D_{Omega Gamma} u_Gamma + N_{Omega Omega} f

The dipole sums are also evaluated by the FMM flow of Sec. 5.1.2 (every G-sum
is an FMM, Sec. 5.3): only P2M and P2P change.  A dipole of strength mu at y
with normal n has the multipole coefficients
  M_a = sum_j mu_j n_j . grad_y conj(R_a(y_j - c)),
the normal derivative of the monopole P2M of Sec. 5.1.2 (special.regular_grad_all);
M2M, M2L, L2L and L2P are those of module fmm.

On the finite-difference side the Dirichlet values enter the right-hand side:
for the 7-point operator with u = u_Gamma at the boundary nodes,
  A_h u = f + lift(u_Gamma),  lift_i = (1/h^2) sum of u_Gamma over the boundary
neighbours of interior node i; those neighbours are exactly the panel
centres (face nodes off the edges), in the panel order of module geometry.
"""
from __future__ import annotations

from math import pi

import numpy as np

from . import special as S
from .bem import Problem
from .fmm import FMM
from .gmres import fgmres
from .tree import centres, flat


def dgreen_dn(x: np.ndarray, y: np.ndarray, ny: np.ndarray, k: float) -> np.ndarray:
    """dG/dn_y (x_i, y_j) for all pairs: shape (len x, len y) (Sec. 5.2, reading S3)."""
    d = y[None, :, :] - x[:, None, :]
    r = np.sqrt(np.sum(d * d, axis=-1))
    rn = np.sum(d * ny[None, :, :], axis=-1) / r          # dr/dn_y
    return (1j * k * r - 1.0) * np.exp(1j * k * r) / (4 * pi * r * r) * rn


def double_layer_direct(points, mu, normals, src_mask, tgt_mask, k, block=512):
    """phi_i = sum_{j src, j != i} mu_j dG/dn_y(x_i, y_j) at every target i,
    the O(N^2) definition (zero at non-targets; the own-panel term is zero).
    `normals` has a row per point (only the source rows are read)."""
    points = np.asarray(points)
    src = np.flatnonzero(src_mask)
    tgt = np.flatnonzero(tgt_mask)
    phi = np.zeros(len(points), dtype=np.complex128)
    ys, ns, ms = points[src], normals[src], mu[src]
    for b0 in range(0, len(tgt), block):
        ti = tgt[b0:b0 + block]
        same = ti[:, None] == src[None, :]
        xt = points[ti]
        # keep r > 0 on the excluded diagonal before evaluating the kernel
        d = ys[None, :, :] - xt[:, None, :]
        r = np.sqrt(np.sum(d * d, axis=-1))
        r = np.where(same, 1.0, r)
        rn = np.sum(d * ns[None, :, :], axis=-1) / r
        g = (1j * k * r - 1.0) * np.exp(1j * k * r) / (4 * pi * r * r) * rn
        g = np.where(same, 0.0, g)
        phi[ti] = g @ ms
    return phi


def p2m_dipole(fmm: FMM, mu, normals, src_mask):
    """Dipole P2M: M_a(c) = sum_j mu_j n_j . grad_y conj(R_a(y_j - c)) over the
    sources of each leaf (the normal derivative of the monopole P2M)."""
    L = fmm.L
    M = np.zeros((8 ** L, fmm.P), dtype=np.complex128)
    j = np.flatnonzero(src_mask)
    if len(j) == 0:
        return M
    leaf = fmm.tree.leaf[j]
    c = centres(L)[leaf]
    G = S.regular_grad_all(fmm.p, fmm.k, fmm.tree.points[j] - c)   # (3, P, nj)
    dR = np.einsum("xaj,jx->aj", np.conj(G), normals[j])            # n . grad conj(R)
    np.add.at(M, leaf, (mu[j][None, :] * dR).T)
    return M


def p2p_dipole(fmm: FMM, mu, normals, src_mask, tgt_mask):
    """Dipole P2P: the direct double-layer sum over the leaves that are not
    separated from the target's leaf (reading T4), j != i."""
    tr = fmm.tree
    L = fmm.L
    s = 2 ** L
    phi = np.zeros(len(tr.points), dtype=np.complex128)
    src = np.flatnonzero(src_mask)
    tgt = np.flatnonzero(tgt_mask)
    src_by_leaf, tgt_by_leaf = {}, {}
    for j, lf in zip(src, tr.leaf[src]):
        src_by_leaf.setdefault(int(lf), []).append(j)
    for i, lf in zip(tgt, tr.leaf[tgt]):
        tgt_by_leaf.setdefault(int(lf), []).append(i)
    near = np.array(tr.near)
    for lf, ti in tgt_by_leaf.items():
        ti = np.array(ti)
        c = tr.leaf_c[ti[0]]
        nb = c + near
        ok = np.all((nb >= 0) & (nb < s), axis=1)
        sj = [src_by_leaf.get(int(f), []) for f in flat(nb[ok], L)]
        sj = np.array([j for lst in sj for j in lst], dtype=np.int64)
        if len(sj) == 0:
            continue
        m = np.zeros(len(tr.points), dtype=bool)
        m[sj] = True
        t = np.zeros(len(tr.points), dtype=bool)
        t[ti] = True
        phi[ti] = double_layer_direct(tr.points, mu, normals, m, t, fmm.k)[ti]
    return phi


def double_layer_fmm(fmm: FMM, mu, normals, src_mask, tgt_mask):
    """The double-layer sum by the FMM flow of Sec. 5.1.2 with dipole P2M and
    P2P (M2M, M2L, L2L, L2P unchanged)."""
    L = fmm.L
    M = {L: p2m_dipole(fmm, mu, normals, src_mask)}
    for l in range(L - 1, 1, -1):
        M[l] = fmm.m2m(M[l + 1], l)
    Lc = {l: fmm.m2l(M[l], l) for l in range(2, L + 1)}
    for l in range(2, L):
        Lc[l + 1] = fmm.l2l(Lc[l], Lc[l + 1], l)
    phi = fmm.l2p(Lc[L], tgt_mask)
    phi += p2p_dipole(fmm, mu, normals, src_mask, tgt_mask)
    return phi


def panel_of_neighbour(n: int):
    """For every interior node (lexicographic, x fastest) and each of its six
    neighbours (-x, +x, -y, +y, -z, +z): the panel index of that neighbour when
    it is a boundary node, else -1.  Shape (n^3, 6)."""
    g = np.arange(1, n + 1)
    L, J, I = np.meshgrid(g, g, g, indexing="ij")
    I, J, L = I.ravel(), J.ravel(), L.ravel()
    idx3 = (I, J, L)
    out = np.full((n ** 3, 6), -1, dtype=np.int64)
    for axis in range(3):
        free = [a for a in range(3) if a != axis]
        a, b = idx3[free[0]], idx3[free[1]]
        for side in (0, 1):
            face = 2 * axis + side
            on = idx3[axis] == (1 if side == 0 else n)
            out[on, face] = face * n * n + (b[on] - 1) * n + (a[on] - 1)
    return out


def dirichlet_lift(n: int, u_bnd) -> np.ndarray:
    """lift_i = (1/h^2) sum of u_Gamma over the boundary neighbours of interior
    node i, so that A_h u = f + lift for u = u_Gamma on the boundary nodes."""
    h = 1.0 / (n + 1)
    nb = panel_of_neighbour(n)
    ub = np.asarray(u_bnd, dtype=np.complex128)
    vals = np.where(nb >= 0, ub[np.maximum(nb, 0)], 0.0)
    return vals.sum(axis=1) / (h * h)


class DirichletProblem(Problem):
    """The homogeneous problem of module bem plus the panel normals and the
    double-layer sums for Dirichlet data."""

    def __init__(self, n, k, p, leaf, theta):
        super().__init__(n, k, p, leaf, theta)
        self.normals = np.zeros((self.NO + self.NG, 3))
        self.normals[self.NO:] = self.n_bnd_normals

    def dense_V(self):
        """The single-layer matrix by its definition (readings B1, B3):
        V_ij = h^2 G(y_i, y_j) for i != j, V_ii = s_Gamma."""
        Y = self.x_bnd
        d = Y[:, None, :] - Y[None, :, :]
        r = np.sqrt(np.sum(d * d, axis=-1))
        np.fill_diagonal(r, 1.0)
        Vm = self.h ** 2 * np.exp(1j * self.k * r) / (4 * pi * r)
        np.fill_diagonal(Vm, self.s_bnd)
        return Vm

    def double_layer(self, u_bnd, tgt, method):
        """D u_Gamma = sum_j h^2 u_j dG/dn_y(x_i, y_j) at the targets `tgt`
        (a point mask over volume + boundary points); full-length result."""
        mu = np.zeros(self.NO + self.NG, dtype=np.complex128)
        mu[self.NO:] = self.h ** 2 * np.asarray(u_bnd)
        if method == "fmm":
            return double_layer_fmm(self.fmm, mu, self.normals, self.bnd, tgt)
        return double_layer_direct(self.points, mu, self.normals, self.bnd, tgt, self.k)

    def bem_solve(self, f, u_bnd, inner_rtol=1e-12, inner_maxit=200, inner_m=50,
                  method="fmm", inner="gmres"):
        """u on the interior nodes from Eq. (ubound) then Eq. (uinter) with
        volume data f and Dirichlet data u_Gamma.  Returns (u, q, inner_iterations),
        q = du/dn on the panels."""
        h = self.h
        NO = self.NO
        u_bnd = np.asarray(u_bnd, dtype=np.complex128)
        qa = np.zeros(NO + self.NG, dtype=np.complex128)
        qa[:NO] = h ** 3 * np.asarray(f)
        nf = self.green(qa, self.vol, self.bnd, method)[NO:]             # N_{Gamma Omega} f
        du = self.double_layer(u_bnd, self.bnd, method)[NO:]             # D_{Gamma Gamma} u
        rhs = 0.5 * u_bnd + du - nf

        def V(qb):
            qq = np.zeros(NO + self.NG, dtype=np.complex128)
            qq[NO:] = h ** 2 * qb
            return self.green(qq, self.bnd, self.bnd, method)[NO:]

        if inner == "dense":
            q = np.linalg.solve(self.dense_V(), rhs)
            its = 0
        else:
            q, info = fgmres(V, rhs, None, m=inner_m, rtol=inner_rtol, maxit=inner_maxit)
            its = info["iters"]
        qa[NO:] = h ** 2 * q
        u = self.green(qa, self.vol | self.bnd, self.vol, method)[:NO]     # V q + N f
        u -= self.double_layer(u_bnd, self.vol, method)[:NO]               # - D u
        return u, q, its
