"""Translation operators between spherical-wave expansions (oracle).

Paper Sec. 5.1.2 names the M2M, M2L and L2L kernels but gives no formulas.
Reading F3: each translation is the exact re-expansion of the truncated input
expansion about the new centre, truncated to degrees n' < p.  With
R_n^m(v) = j_n(k|v|) Y_n^m(v/|v|) and S_n^m(v) = h_n(k|v|) Y_n^m(v/|v|) the
Helmholtz addition theorem gives (finite Gaunt sums in l)

  R_a(r + t) = sum_a' (R|R)_{a' a}(t) R_a'(r)                 all r
  S_a(r + t) = sum_a' (R|R)_{a' a}(t) S_a'(r)                 |r| > |t|
  S_a(r + t) = sum_a' (S|R)_{a' a}(t) R_a'(r)                 |r| < |t|

  (F|R)_{a' a}(t) = 4 pi sum_l i^(n' + l - n) F_{l, m - m'}(t)
                      * integral Y_a conj(Y_a') conj(Y_{l, m - m'})

with F = R for (R|R) and F = S for (S|R), a = (n, m), a' = (n', m').
The matrices below map input coefficients (index a) to output ones (a'):
out = T @ in.
"""
from __future__ import annotations

from functools import lru_cache
from math import pi

import numpy as np

from .special import gaunt_table, nm_of, regular_all, singular_all


@lru_cache(maxsize=None)
def _pattern(p: int):
    """Nonzero terms of the Gaunt sum: for every (a', a, l) with a nonzero
    Gaunt integral, the flat index of F_{l, m - m'} and the factor
    4 pi i^(n' + l - n) * integral Y_a conj(Y_a') conj(Y_{l, m - m'})."""
    P = p * p
    lmax = 2 * p - 1
    gt = gaunt_table(p)
    ns, ms = nm_of(P)
    AP, A, L = np.meshgrid(np.arange(P), np.arange(P), np.arange(lmax), indexing="ij")
    g = gt[A, AP, L]                      # integral Y_a conj(Y_a') conj(Y_{l, m - m'})
    keep = g != 0.0
    AP, A, L, g = AP[keep], A[keep], L[keep], g[keep]
    mu = ms[A] - ms[AP]
    FI = L * L + L + mu
    phase = (1j) ** ((ns[AP] + L - ns[A]) % 4)
    return AP, A, FI, 4 * pi * phase * g


def _op(kind: str, p: int, k: float, t) -> np.ndarray:
    P = p * p
    lmax = 2 * p - 1
    t = np.asarray(t, dtype=np.float64).reshape(1, 3)
    if kind == "RR":
        F = regular_all(lmax, k, t)[:, 0]
    else:
        F = singular_all(lmax, k, t)[:, 0]
    AP, A, FI, C = _pattern(p)
    T = np.zeros((P, P), dtype=np.complex128)
    np.add.at(T, (AP, A), C * F[FI])
    return T


def m2m_op(p: int, k: float, t) -> np.ndarray:
    """Multipole at a child centre c' to multipole at the parent centre c;
    t = c - c' (the S -> S re-expansion uses (R|R)(t))."""
    return _op("RR", p, k, t)


def m2l_op(p: int, k: float, t) -> np.ndarray:
    """Multipole at a source centre c_S to local at a target centre c_T;
    t = c_T - c_S."""
    return _op("SR", p, k, t)


def l2l_op(p: int, k: float, t) -> np.ndarray:
    """Local at a parent centre c to local at a child centre c'; t = c' - c."""
    return _op("RR", p, k, t)
