"""Fast multipole evaluation of the 3D Helmholtz potential (oracle, FP64).

Paper Sec. 5.1: the N-body sum f(y_j) = sum_i w_i K(y_j, x_i) with the 3D
Helmholtz kernel K = G = exp(i k r) / (4 pi r) of Sec. 5.2, evaluated by the
FMM flow of Sec. 5.1.2: P2M, M2M, M2L, L2L, L2P and P2P.

Expansions (reading F1), from the addition theorem
G(x, y) = i k sum_a S_a(x - c) conj(R_a(y - c)),  |y - c| < |x - c|:
  multipole about c:  phi(x) = i k sum_a M_a S_a(x - c),
                      M_a = sum_j q_j conj(R_a(y_j - c));
  local about c:      phi(x) = i k sum_a L_a R_a(x - c).
Degrees n = 0..p-1 (reading F2); centres are geometric cell centres.

The potential returned at every target i is
  phi_i = sum_{j in sources, j != i} q_j G(x_i, x_j) + [i is a source] sigma_i q_i
where sigma_i q_i is the singular self term (reading B3): the integral of G
over the point's own cell (volume node) or panel (boundary element) divided by
its quadrature weight.
"""
from __future__ import annotations

from math import pi

import numpy as np

from . import special as S
from . import translations as TT
from .tree import Tree, centres, flat


def green(x: np.ndarray, y: np.ndarray, k: float) -> np.ndarray:
    """G(x, y) = exp(i k |x - y|) / (4 pi |x - y|) for all pairs: (len x, len y)."""
    d = x[:, None, :] - y[None, :, :]
    r = np.sqrt(np.sum(d * d, axis=-1))
    return np.exp(1j * k * r) / (4 * pi * r)


# ---------------------------------------------------------------- self terms

def _gauss(n: int, a: float, b: float):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def self_volume(h: float, k: float, nq: int = 28) -> complex:
    """Integral of G(0, y) over the cube [-h/2, h/2]^3 (reading B3).

    The cube is the union of six pyramids with apex at the centre; in each,
    y = s P with P on the face x = h/2 and s in [0, 1], dV = s^2 (h/2) ds dA.
    Every pyramid gives the same value, so the integral is
      6 (h/2) int_face int_0^1 s^2 G(s |P|) ds dA
    with Gauss-Legendre rules in s and in both face coordinates."""
    u, wu = _gauss(nq, -h / 2, h / 2)
    s, ws = _gauss(nq, 0.0, 1.0)
    U, V = np.meshgrid(u, u, indexing="ij")
    W2 = np.outer(wu, wu)
    R = np.sqrt(h * h / 4 + U * U + V * V)
    total = 0.0 + 0.0j
    for si, wsi in zip(s, ws):
        r = si * R
        total += wsi * np.sum(W2 * si * si * np.exp(1j * k * r) / (4 * pi * r))
    return 6 * (h / 2) * total


def self_panel(h: float, k: float, nq: int = 28) -> complex:
    """Integral of G(0, y) over the square panel [-h/2, h/2]^2 (reading B3).

    Four triangles with apex at the centre: y = s P with P on the edge
    x = h/2, dA = s (h/2) ds du; the integral is
      4 (h/2) int_edge int_0^1 s G(s |P|) ds du."""
    u, wu = _gauss(nq, -h / 2, h / 2)
    s, ws = _gauss(nq, 0.0, 1.0)
    R = np.sqrt(h * h / 4 + u * u)
    total = 0.0 + 0.0j
    for si, wsi in zip(s, ws):
        r = si * R
        total += wsi * np.sum(wu * si * np.exp(1j * k * r) / (4 * pi * r))
    return 4 * (h / 2) * total


# ---------------------------------------------------------------- direct sum

def direct_sum(points, q, src_mask, tgt_mask, k, sigma, block=512):
    """phi_i = sum_{j src, j != i} q_j G(x_i, x_j) + [i src] sigma_i q_i for
    every target i (paper Sec. 5.1: all pairs, O(N^2)).  Returns phi over all
    points (zero at non-targets)."""
    points = np.asarray(points)
    src = np.flatnonzero(src_mask)
    tgt = np.flatnonzero(tgt_mask)
    phi = np.zeros(len(points), dtype=np.complex128)
    ys, qs = points[src], q[src]
    for b0 in range(0, len(tgt), block):
        ti = tgt[b0:b0 + block]
        d = points[ti][:, None, :] - ys[None, :, :]
        r = np.sqrt(np.sum(d * d, axis=-1))
        same = ti[:, None] == src[None, :]
        r = np.where(same, 1.0, r)
        g = np.where(same, 0.0, np.exp(1j * k * r) / (4 * pi * r))
        phi[ti] = g @ qs
    phi[tgt] += np.where(src_mask[tgt], sigma[tgt] * q[tgt], 0.0)
    return phi


# ---------------------------------------------------------------- FMM stages

class FMM:
    """FMM over a fixed point set (reading T1-T4 tree, F1-F3 expansions)."""

    def __init__(self, points, n_vol, leaf, theta, k, p):
        self.tree = Tree(points, n_vol, leaf, theta)
        self.k = k
        self.p = p
        self.P = p * p
        self.L = self.tree.L
        self._m2l_cache = {}
        self._ops = {}

    # width of a cell at level l
    def w(self, l):
        return 1.0 / 2 ** l

    def p2m(self, q, src_mask):
        """P2M (Sec. 5.1.2): M_a(c) = sum_j q_j conj(R_a(y_j - c)) over the
        sources of each leaf."""
        L = self.L
        M = np.zeros((8 ** L, self.P), dtype=np.complex128)
        j = np.flatnonzero(src_mask)
        if len(j) == 0:
            return M
        leaf = self.tree.leaf[j]
        c = centres(L)[leaf]
        R = S.regular_all(self.p, self.k, self.tree.points[j] - c)   # (P, nj)
        np.add.at(M, leaf, (q[j][None, :] * np.conj(R)).T)
        return M

    def m2m(self, Mchild, l):
        """M2M (Sec. 5.1.2): multipoles of level l+1 to level l."""
        s = 2 ** l
        Mpar = np.zeros((8 ** l, self.P), dtype=np.complex128)
        g = np.arange(s)
        iz, iy, ix = np.meshgrid(g, g, g, indexing="ij")
        I = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
        wc = self.w(l + 1)
        for o in np.ndindex(2, 2, 2):
            o = np.array(o)
            t = (0.5 - o) * wc                      # c_parent - c_child
            key = ("m2m", l, tuple(o))
            if key not in self._ops:
                self._ops[key] = TT.m2m_op(self.p, self.k, t)
            T = self._ops[key]
            child = flat(2 * I + o, l + 1)
            Mpar += Mchild[child] @ T.T
        return Mpar

    def m2l(self, M, l):
        """M2L (Sec. 5.1.2): L_T += sum_{S in list(T)} T(c_T - c_S) M_S."""
        Lc = np.zeros((8 ** l, self.P), dtype=np.complex128)
        for v, (t_idx, s_idx) in self.tree.m2l_pairs(l).items():
            key = (l, v)
            if key not in self._m2l_cache:
                t = -np.array(v, dtype=np.float64) * self.w(l)   # c_T - c_S
                self._m2l_cache[key] = TT.m2l_op(self.p, self.k, t)
            T = self._m2l_cache[key]
            # each target appears once per offset, so a plain indexed add is
            # the sum over the list
            Lc[t_idx] += M[s_idx] @ T.T
        return Lc

    def l2l(self, Lpar, Lchild, l):
        """L2L (Sec. 5.1.2): locals of level l to level l+1 (added in)."""
        s = 2 ** l
        g = np.arange(s)
        iz, iy, ix = np.meshgrid(g, g, g, indexing="ij")
        I = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
        wc = self.w(l + 1)
        for o in np.ndindex(2, 2, 2):
            o = np.array(o)
            t = (o - 0.5) * wc                      # c_child - c_parent
            key = ("l2l", l, tuple(o))
            if key not in self._ops:
                self._ops[key] = TT.l2l_op(self.p, self.k, t)
            T = self._ops[key]
            child = flat(2 * I + o, l + 1)
            Lchild[child] += Lpar[flat(I, l)] @ T.T
        return Lchild

    def l2p(self, Lleaf, tgt_mask):
        """L2P (Sec. 5.1.2): phi_i = i k sum_a L_a R_a(x_i - c)."""
        phi = np.zeros(len(self.tree.points), dtype=np.complex128)
        i = np.flatnonzero(tgt_mask)
        if len(i) == 0:
            return phi
        leaf = self.tree.leaf[i]
        c = centres(self.L)[leaf]
        R = S.regular_all(self.p, self.k, self.tree.points[i] - c)   # (P, ni)
        phi[i] = 1j * self.k * np.sum(Lleaf[leaf].T * R, axis=0)
        return phi

    def p2p(self, q, src_mask, tgt_mask):
        """P2P (Sec. 5.1.2): direct sum over the leaves that are not separated
        from the target's leaf, the leaf itself included, j != i (reading T4)."""
        tr = self.tree
        L = self.L
        s = 2 ** L
        phi = np.zeros(len(tr.points), dtype=np.complex128)
        src = np.flatnonzero(src_mask)
        tgt = np.flatnonzero(tgt_mask)
        src_by_leaf = {}
        for j, lf in zip(src, tr.leaf[src]):
            src_by_leaf.setdefault(int(lf), []).append(j)
        tgt_by_leaf = {}
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
            d = tr.points[ti][:, None, :] - tr.points[sj][None, :, :]
            r = np.sqrt(np.sum(d * d, axis=-1))
            same = ti[:, None] == sj[None, :]
            r = np.where(same, 1.0, r)
            g = np.where(same, 0.0, np.exp(1j * self.k * r) / (4 * pi * r))
            phi[ti] = g @ q[sj]
        return phi

    def apply(self, q, src_mask, tgt_mask, sigma):
        """Full FMM: phi at targets (zero elsewhere), self term included."""
        L = self.L
        M = {L: self.p2m(q, src_mask)}
        for l in range(L - 1, 1, -1):
            M[l] = self.m2m(M[l + 1], l)
        Lc = {l: self.m2l(M[l], l) for l in range(2, L + 1)}
        for l in range(2, L):
            Lc[l + 1] = self.l2l(Lc[l], Lc[l + 1], l)
        phi = self.l2p(Lc[L], tgt_mask)
        phi += self.p2p(q, src_mask, tgt_mask)
        phi[tgt_mask] += np.where(src_mask[tgt_mask], sigma[tgt_mask] * q[tgt_mask], 0.0)
        return phi
