"""Pins for the oracle's special functions and translation operators.

Each check compares against something other than the oracle itself: closed
forms, arbitrary-precision mpmath, exact rational Gaunt coefficients (sympy),
and the addition theorems evaluated pointwise with a much larger truncation.
"""
import math

import numpy as np
import pytest

from oracle import special as S
from oracle import translations as TT

mpmath = pytest.importorskip("mpmath")


def test_bessel_closed_forms():
    x = np.linspace(0.05, 40.0, 301)
    np.testing.assert_allclose(S.sph_jn(0, x), np.sin(x) / x, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(S.sph_jn(1, x), np.sin(x) / x ** 2 - np.cos(x) / x,
                               rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(S.sph_yn(0, x), -np.cos(x) / x, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(S.sph_yn(1, x), -np.cos(x) / x ** 2 - np.sin(x) / x,
                               rtol=1e-11, atol=1e-15)
    # h_0 = -i e^{ix} / x
    np.testing.assert_allclose(S.sph_hn(0, x), -1j * np.exp(1j * x) / x, rtol=1e-13)


def test_bessel_wronskian():
    # j_n y_{n-1} - j_{n-1} y_n = 1 / x^2
    x = np.linspace(0.3, 30.0, 97)
    for n in range(1, 16):
        w = S.sph_jn(n, x) * S.sph_yn(n - 1, x) - S.sph_jn(n - 1, x) * S.sph_yn(n, x)
        np.testing.assert_allclose(w * x * x, 1.0, rtol=1e-10)


@pytest.mark.parametrize("n", [0, 3, 7, 11, 15, 20])
def test_bessel_mpmath(n):
    # range of arguments the FMM uses: k rho in leaves up to k |t| at level 2
    for x in [1e-3, 0.07, 0.5, 1.3, 2.9, 6.0, 11.0, 23.0, 47.0]:
        jr = float(mpmath.sqrt(mpmath.pi / (2 * x)) * mpmath.besselj(n + 0.5, x))
        yr = float(mpmath.sqrt(mpmath.pi / (2 * x)) * mpmath.bessely(n + 0.5, x))
        assert abs(S.sph_jn(n, x) - jr) <= 1e-13 * abs(jr) + 1e-300
        assert abs(S.sph_yn(n, x) - yr) <= 1e-13 * abs(yr)


def test_ylm_closed_forms():
    th = np.array([0.1, 0.7, 1.9, 2.8])
    ph = np.array([0.3, -1.2, 2.5, 0.0])
    np.testing.assert_allclose(S.ylm(0, 0, th, ph), 0.5 / np.sqrt(np.pi))
    np.testing.assert_allclose(S.ylm(1, 0, th, ph), np.sqrt(3 / (4 * np.pi)) * np.cos(th))
    np.testing.assert_allclose(S.ylm(1, 1, th, ph),
                               -np.sqrt(3 / (8 * np.pi)) * np.sin(th) * np.exp(1j * ph))
    np.testing.assert_allclose(S.ylm(1, -1, th, ph),
                               np.sqrt(3 / (8 * np.pi)) * np.sin(th) * np.exp(-1j * ph))
    np.testing.assert_allclose(S.ylm(2, 2, th, ph),
                               0.25 * np.sqrt(15 / (2 * np.pi)) * np.sin(th) ** 2
                               * np.exp(2j * ph))


def test_ylm_orthonormal():
    p = 7
    xg, wg = np.polynomial.legendre.leggauss(16)
    nph = 32
    TH, PH = np.meshgrid(np.arccos(xg), 2 * np.pi * np.arange(nph) / nph, indexing="ij")
    W = (wg[:, None] * np.full(nph, 2 * np.pi / nph)[None, :]).ravel()
    Y = S.ylm_all(p, TH.ravel(), PH.ravel())
    gram = (Y * W) @ np.conj(Y).T
    np.testing.assert_allclose(gram, np.eye(p * p), atol=1e-13)


def test_ylm_addition_theorem():
    # sum_m Y_n^m(a) conj(Y_n^m(b)) = (2n+1)/(4 pi) P_n(a . b)
    rng = np.random.default_rng(3)
    a = rng.standard_normal(3); a /= np.linalg.norm(a)
    b = rng.standard_normal(3); b /= np.linalg.norm(b)
    _, ta, pa = S.cart2sph(a[None])
    _, tb, pb = S.cart2sph(b[None])
    for n in range(9):
        s = sum(S.ylm(n, m, ta, pa) * np.conj(S.ylm(n, m, tb, pb)) for m in range(-n, n + 1))
        ref = (2 * n + 1) / (4 * np.pi) * np.polynomial.legendre.legval(a @ b, [0] * n + [1])
        assert abs(s[0] - ref) < 1e-13


def test_gaunt_vs_sympy_exact():
    from sympy.physics.wigner import gaunt
    p = 4
    gt = S.gaunt_table(p)
    ns, ms = S.nm_of(p * p)
    worst = 0.0
    for a in range(p * p):
        for b in range(p * p):
            mu = int(ms[a] - ms[b])
            for l in range(abs(mu), 2 * p - 1):
                # conj(Y_n^m) = (-1)^m Y_n^{-m}
                ref = float(gaunt(int(ns[a]), int(ns[b]), l, int(ms[a]), -int(ms[b]), -mu))
                ref *= (-1) ** (int(ms[b]) + mu)
                worst = max(worst, abs(ref - gt[a, b, l]))
    assert worst < 1e-14


def test_greens_function_expansion():
    # G(x, y) = i k sum_a S_a(x) conj(R_a(y)) for |y| < |x| (reading F1)
    k = 5.0
    x = np.array([0.7, -0.2, 0.45])
    y = np.array([0.1, 0.12, -0.05])
    r = np.linalg.norm(x - y)
    G = np.exp(1j * k * r) / (4 * np.pi * r)
    s = 1j * k * np.sum(S.singular_all(30, k, x[None])[:, 0]
                        * np.conj(S.regular_all(30, k, y[None])[:, 0]))
    assert abs(s - G) < 1e-14 * abs(G) + 1e-15


@pytest.mark.parametrize("k", [0.7, 4.0, 16.0])
def test_translation_addition_theorems(k):
    """(S|R), (R|R) and (S|S)=(R|R) against pointwise evaluation of the
    untranslated basis with a large output truncation."""
    p, pbig = 5, 18
    rng = np.random.default_rng(int(k * 10))
    for _ in range(3):
        t = rng.uniform(-1, 1, 3); t *= 0.9 / np.linalg.norm(t)
        r = rng.uniform(-1, 1, 3); r *= 0.1 / np.linalg.norm(r)
        # S(r + t) = sum (S|R)(t) R(r), |r| < |t|
        lhs = S.singular_all(p, k, (r + t)[None])[:, 0]
        T = TT._op("SR", pbig, k, t)[:, :p * p]
        rhs = T.T @ S.regular_all(pbig, k, r[None])[:, 0]
        assert np.max(np.abs(lhs - rhs)) < 1e-10 * np.max(np.abs(lhs))
        # R(r + t) = sum (R|R)(t) R(r)
        lhs = S.regular_all(p, k, (r + t)[None])[:, 0]
        T = TT._op("RR", pbig, k, t)[:, :p * p]
        rhs = T.T @ S.regular_all(pbig, k, r[None])[:, 0]
        assert np.max(np.abs(lhs - rhs)) < 1e-12 * max(1e-3, np.max(np.abs(lhs)))
        # S(r + t) = sum (R|R)(t) S(r), |r| > |t| (swap the roles)
        lhs = S.singular_all(p, k, (t + r)[None])[:, 0]
        T = TT._op("RR", pbig, k, r)[:, :p * p]
        rhs = T.T @ S.singular_all(pbig, k, t[None])[:, 0]
        assert np.max(np.abs(lhs - rhs)) < 1e-10 * np.max(np.abs(lhs))


def test_translation_truncation_converges():
    # M2L of a single multipole coefficient: error of the truncated local
    # expansion falls geometrically with its order
    k = 3.0
    t = np.array([0.0, 0.0, 1.0])
    r = np.array([0.15, -0.1, 0.2])
    lhs = S.singular_all(3, k, (r + t)[None])[:, 0]
    errs = []
    for po in (6, 10, 14, 18):
        T = TT._op("SR", po, k, t)[:, :9]
        rhs = T.T @ S.regular_all(po, k, r[None])[:, 0]
        errs.append(np.max(np.abs(lhs - rhs)))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[-1] < 1e-9 * np.max(np.abs(lhs))
