"""Uniform octree and interaction lists (oracle).

Paper Sec. 5.1.1 (hierarchical domain decomposition: the cube is subdivided
recursively into eight cells down to a leaf level) and Sec. 7 (theta = 0.4).
Readings taken where the paper is silent:

T1  depth L = max(2, ceil(log8(N_vol / leaf))), i.e. the smallest L >= 2 with
    leaf * 8^L >= N_vol; every leaf is at level L.
T2  root box [0,1]^3; a point x lies in cell floor(x 2^l), clamped to 2^l - 1.
T3  two cells of one level with centre offset d (in cell widths) are
    separated iff theta * |d| > 1, i.e. theta |c_T - c_S| > r_T + r_S with r
    the half width; evaluated in exact rational arithmetic.
T4  M2L at level l >= 2 for separated pairs whose parents are not separated;
    P2P for leaf pairs that are not separated (the leaf itself included).

Cells are addressed by integer coordinates (ix, iy, iz); the flat index is
ix + iy 2^l + iz 4^l.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import product

import numpy as np


def depth(n_vol: int, leaf: int) -> int:
    L = 2
    while leaf * 8 ** L < n_vol:
        L += 1
    return L


def _theta_sq(theta: float) -> Fraction:
    t = Fraction(theta).limit_denominator(10000)
    return t * t


def separated(d2: int, theta: float) -> bool:
    """T3 with d2 = |d|^2 in cell widths squared."""
    return _theta_sq(theta) * d2 > 1


def near_offsets(theta: float):
    """Offsets v (cell units) of cells that are NOT separated from a cell."""
    r = int(np.floor(1.0 / theta)) + 1
    out = []
    for v in product(range(-r, r + 1), repeat=3):
        if not separated(v[0] ** 2 + v[1] ** 2 + v[2] ** 2, theta):
            out.append(v)
    return out


def m2l_offsets(theta: float, parity):
    """M2L offsets for a cell whose coordinates have parity bits `parity`
    (each 0 or 1): v = 2u + c - parity over non-separated parent offsets u and
    child positions c, kept if v itself is separated (T4)."""
    b = np.array(parity)
    out = set()
    for u in near_offsets(theta):
        for c in product((0, 1), repeat=3):
            v = 2 * np.array(u) + np.array(c) - b
            if separated(int(v @ v), theta):
                out.add(tuple(int(t) for t in v))
    return sorted(out)


def cell_of(x: np.ndarray, level: int) -> np.ndarray:
    """T2: integer cell coordinates of points x (N, 3) at `level`."""
    s = 2 ** level
    return np.minimum(np.floor(x * s).astype(np.int64), s - 1)


def flat(c: np.ndarray, level: int) -> np.ndarray:
    s = 2 ** level
    return c[..., 0] + s * c[..., 1] + s * s * c[..., 2]


def centres(level: int) -> np.ndarray:
    """Centres of all cells of a level, indexed by flat index: (8^level, 3)."""
    s = 2 ** level
    g = (np.arange(s) + 0.5) / s
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


class Tree:
    """Uniform octree over a set of points (all points in [0,1]^3)."""

    def __init__(self, points: np.ndarray, n_vol: int, leaf: int, theta: float):
        self.L = depth(n_vol, leaf)
        self.theta = theta
        self.points = np.asarray(points, dtype=np.float64)
        self.leaf_c = cell_of(self.points, self.L)
        self.leaf = flat(self.leaf_c, self.L)
        self.near = near_offsets(theta)
        self.m2l = {b: m2l_offsets(theta, b) for b in product((0, 1), repeat=3)}
        self._pairs = {}

    def m2l_pairs(self, level: int):
        """All (target, source) flat-index pairs of level `level` with their
        offset: dict v -> (targets, sources) arrays."""
        if level in self._pairs:
            return self._pairs[level]
        s = 2 ** level
        g = np.arange(s)
        iz, iy, ix = np.meshgrid(g, g, g, indexing="ij")
        T = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
        par = T % 2
        out = {}
        for b, offs in self.m2l.items():
            sel = np.all(par == np.array(b), axis=1)
            Tb = T[sel]
            for v in offs:
                S = Tb + np.array(v)
                ok = np.all((S >= 0) & (S < s), axis=1)
                if not np.any(ok):
                    continue
                t_idx = flat(Tb[ok], level)
                s_idx = flat(S[ok], level)
                if v in out:
                    out[v] = (np.concatenate([out[v][0], t_idx]),
                              np.concatenate([out[v][1], s_idx]))
                else:
                    out[v] = (t_idx, s_idx)
        self._pairs[level] = out
        return out
