"""Pins for the oracle's tree, FMM and self terms."""
from itertools import product
from math import log, pi, sqrt

import numpy as np
import pytest

from oracle import fmm as F
from oracle import geometry, tree


def test_offset_counts():
    # theta = 0.4: |d|^2 <= 6 is near (6.25 bound); theta = 0.35: |d|^2 <= 8
    assert len(tree.near_offsets(0.4)) == 81
    assert len(tree.near_offsets(0.35)) == 93
    for b in product((0, 1), repeat=3):
        assert len(tree.m2l_offsets(0.4, b)) == 567
        assert len(tree.m2l_offsets(0.35, b)) == 651


@pytest.mark.parametrize("theta", [0.4, 0.35])
def test_lists_cover_every_leaf_pair_once(theta):
    """Brute force at L = 3: each ordered leaf pair is handled exactly once,
    either by P2P at the leaf level or by M2L at exactly one level."""
    L = 3
    s = 2 ** L
    t = tree.Tree(np.zeros((1, 3)), 8 ** L, 1, theta)
    assert t.L == L
    count = np.zeros((8 ** L, 8 ** L), dtype=np.int64)
    for l in range(2, L + 1):
        sh = L - l
        for v, (ti, si) in t.m2l_pairs(l).items():
            # expand each level-l pair to all leaf pairs below it
            sl = 2 ** l
            tc = np.stack([ti % sl, (ti // sl) % sl, ti // (sl * sl)], 1)
            sc = np.stack([si % sl, (si // sl) % sl, si // (sl * sl)], 1)
            for a in product(range(2 ** sh), repeat=3):
                for b in product(range(2 ** sh), repeat=3):
                    lt = tree.flat(tc * 2 ** sh + np.array(a), L)
                    ls = tree.flat(sc * 2 ** sh + np.array(b), L)
                    np.add.at(count, (lt, ls), 1)
    g = np.arange(s)
    iz, iy, ix = np.meshgrid(g, g, g, indexing="ij")
    C = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], 1)
    for i in range(8 ** L):
        for v in t.near:
            c = C[i] + np.array(v)
            if np.all((c >= 0) & (c < s)):
                count[i, tree.flat(c, L)] += 1
    assert np.all(count == 1)


def test_depth_rule():
    assert tree.depth(16 ** 3, 32) == 3
    assert tree.depth(64 ** 3, 64) == 4
    assert tree.depth(128 ** 3, 64) == 5
    assert tree.depth(24 ** 3, 64) == 3
    assert tree.depth(96 ** 3, 64) == 5
    assert tree.depth(10, 64) == 2


def test_single_source_closed_form():
    # one source: the potential is the free-space Green's function (Sec. 5.2)
    k = 7.0
    pts = np.array([[0.3, 0.4, 0.5], [0.9, 0.1, 0.2], [0.35, 0.42, 0.47]])
    q = np.array([2.0 - 1.0j, 0, 0])
    src = np.array([True, False, False])
    phi = F.direct_sum(pts, q, src, ~src, k, np.zeros(3))
    for i in (1, 2):
        r = np.linalg.norm(pts[i] - pts[0])
        assert abs(phi[i] - q[0] * np.exp(1j * k * r) / (4 * pi * r)) < 1e-15


def _random_problem(N, seed):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0, 1, (N, 3))
    q = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return pts, q


def test_fmm_converges_to_direct_sum():
    """Error of the FMM against the O(N^2) sum falls geometrically with p."""
    pts, q = _random_problem(600, 1)
    allm = np.ones(len(pts), bool)
    sig = np.zeros(len(pts))
    k = 6.0
    d = F.direct_sum(pts, q, allm, allm, k, sig)
    errs = []
    for p in (2, 4, 6, 8, 10):
        f = F.FMM(pts, len(pts), 4, 0.4, k, p).apply(q, allm, allm, sig)
        errs.append(np.linalg.norm(f - d) / np.linalg.norm(d))
    assert all(errs[i + 1] < 0.3 * errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-6


def test_fmm_high_order_matches_direct():
    pts, q = _random_problem(250, 2)
    allm = np.ones(len(pts), bool)
    sig = np.zeros(len(pts))
    k = 3.0
    d = F.direct_sum(pts, q, allm, allm, k, sig)
    f = F.FMM(pts, len(pts), 2, 0.4, k, 16).apply(q, allm, allm, sig)
    assert np.linalg.norm(f - d) / np.linalg.norm(d) < 1e-10


def test_fmm_low_frequency_limit():
    """k -> 0: exp(ikr)/(4 pi r) = 1/(4 pi r) + ik/(4 pi) + O(k^2 r)."""
    pts, q = _random_problem(300, 3)
    allm = np.ones(len(pts), bool)
    sig = np.zeros(len(pts))
    k = 1e-4
    f = F.FMM(pts, len(pts), 4, 0.4, k, 12).apply(q, allm, allm, sig)
    d = pts[:, None, :] - pts[None, :, :]
    r = np.sqrt(np.sum(d * d, -1))
    np.fill_diagonal(r, np.inf)
    lap = (1 / (4 * pi * r)) @ q + 1j * k / (4 * pi) * (q.sum() - q)
    assert np.linalg.norm(f - lap) / np.linalg.norm(lap) < 1e-7


def test_fmm_linear_and_set_masks():
    pts, q = _random_problem(300, 4)
    rng = np.random.default_rng(5)
    src = rng.uniform(size=300) < 0.5
    tgt = rng.uniform(size=300) < 0.6
    sig = rng.standard_normal(300)
    k = 5.0
    m = F.FMM(pts, 300, 4, 0.4, k, 8)
    f = m.apply(q, src, tgt, sig)
    d = F.direct_sum(pts, q, src, tgt, k, sig)
    assert np.all(f[~tgt] == 0)
    assert np.linalg.norm(f - d) / np.linalg.norm(d) < 1e-5
    f2 = m.apply(2.5j * q, src, tgt, sig)
    assert np.allclose(f2, 2.5j * f, rtol=1e-13, atol=1e-13)


def test_self_terms_static_closed_forms():
    """k = 0: cube integral of 1/(4 pi r) is h^2 C3/(4 pi) with
    C3 = 3 ln((sqrt3+1)/(sqrt3-1)) - pi/2; square panel gives
    h 4 ln(1 + sqrt2)/(4 pi)."""
    h = 0.037
    C3 = 3 * log((sqrt(3) + 1) / (sqrt(3) - 1)) - pi / 2
    assert abs(C3 - 2.380077363979554) < 1e-14
    assert abs(F.self_volume(h, 0.0) - h * h * C3 / (4 * pi)) < 1e-15 * h * h
    assert abs(F.self_panel(h, 0.0) - h * 4 * log(1 + sqrt(2)) / (4 * pi)) < 1e-15 * h


@pytest.mark.parametrize("k", [4.0, 16.0, 32.0])
def test_self_terms_against_octant_quadrature(k):
    """k > 0: compare with tensor Gauss-Legendre over each octant (quadrant)
    of the singular part's complement plus the exact static part."""
    h = 1.0 / 17
    x, w = np.polynomial.legendre.leggauss(40)
    x = 0.25 * h * (x + 1)             # [0, h/2]
    w = 0.25 * h * w
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    R = np.sqrt(X * X + Y * Y + Z * Z)
    smooth = 8 * np.sum(W * (np.exp(1j * k * R) - 1) / (4 * pi * R))
    C3 = 3 * log((sqrt(3) + 1) / (sqrt(3) - 1)) - pi / 2
    ref = h * h * C3 / (4 * pi) + smooth
    assert abs(F.self_volume(h, k) - ref) < 1e-9 * abs(ref)
    X2, Y2 = np.meshgrid(x, x, indexing="ij")
    W2 = w[:, None] * w[None, :]
    R2 = np.sqrt(X2 * X2 + Y2 * Y2)
    smooth2 = 4 * np.sum(W2 * (np.exp(1j * k * R2) - 1) / (4 * pi * R2))
    ref2 = h * 4 * log(1 + sqrt(2)) / (4 * pi) + smooth2
    assert abs(F.self_panel(h, k) - ref2) < 1e-9 * abs(ref2)


def test_geometry_counts_and_placement():
    n = 5
    x = geometry.interior_nodes(n)
    assert x.shape == (125, 3)
    h = 1 / 6
    assert np.allclose(x[1], [2 * h, h, h]) and np.allclose(x[5], [h, 2 * h, h])
    c, nr = geometry.boundary_panels(n)
    assert c.shape == (150, 3)
    # no panel on an edge or a corner; every panel on exactly one face
    on = (np.isclose(c, 0) | np.isclose(c, 1)).sum(1)
    assert np.all(on == 1)
    assert np.allclose(np.abs(nr).sum(1), 1)
    assert np.allclose(c[0], [0, h, h]) and np.allclose(c[1], [0, 2 * h, h])
    assert np.allclose(c[25], [1, h, h]) and np.allclose(c[50], [h, 0, h])
