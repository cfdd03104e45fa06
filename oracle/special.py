"""Special functions for the 3D Helmholtz kernel (oracle, FP64).

Paper Sec. 5.2: the 3D Green's function is G(P,Q) = exp(i k r) / (4 pi r).
Its expansion uses spherical Bessel j_n, y_n and Hankel h_n = j_n + i y_n
functions and orthonormal spherical harmonics Y_n^m (reading F1).

Coefficient index: a = n*n + n + m for degree n, order m in [-n, n].
"""
from __future__ import annotations

from functools import lru_cache
from math import factorial, pi, sqrt

import numpy as np
from scipy import special as sp


def sph_jn(n, x):
    """Spherical Bessel function of the first kind (scipy)."""
    return sp.spherical_jn(n, x)


def sph_yn(n, x):
    """Spherical Bessel function of the second kind (scipy)."""
    return sp.spherical_yn(n, x)


def sph_hn(n, x):
    """Spherical Hankel function of the first kind, h_n = j_n + i y_n."""
    return sp.spherical_jn(n, x) + 1j * sp.spherical_yn(n, x)


def idx(n: int, m: int) -> int:
    return n * n + n + m


def nm_of(P: int):
    """Arrays (n, m) for every coefficient index a < P."""
    ns, ms = [], []
    n = 0
    while n * n < P:
        for m in range(-n, n + 1):
            ns.append(n)
            ms.append(m)
        n += 1
    return np.array(ns[:P]), np.array(ms[:P])


def ylm(n: int, m: int, theta, phi):
    """Orthonormal spherical harmonic with the Condon-Shortley phase:
    Y_n^m = sqrt((2n+1)/(4 pi) (n-|m|)!/(n+|m|)!) P_n^|m|(cos theta) e^{i |m| phi},
    Y_n^{-m} = (-1)^m conj(Y_n^m).  scipy's lpmv carries the (-1)^m phase."""
    am = abs(m)
    norm = sqrt((2 * n + 1) / (4 * pi) * factorial(n - am) / factorial(n + am))
    y = norm * sp.lpmv(am, n, np.cos(theta)) * np.exp(1j * am * np.asarray(phi))
    if m < 0:
        y = (-1) ** am * np.conj(y)
    return y


def ylm_all(nmax: int, theta, phi):
    """All Y_n^m for n < nmax at the given angles: shape (nmax^2, *theta.shape)."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    out = np.empty((nmax * nmax,) + theta.shape, dtype=np.complex128)
    for n in range(nmax):
        for m in range(-n, n + 1):
            out[idx(n, m)] = ylm(n, m, theta, phi)
    return out


def cart2sph(v):
    """(r, theta, phi) of vectors v[..., 3]; theta polar from +z, phi azimuth."""
    v = np.asarray(v, dtype=np.float64)
    r = np.sqrt(np.sum(v * v, axis=-1))
    rho = np.hypot(v[..., 0], v[..., 1])
    theta = np.arctan2(rho, v[..., 2])
    phi = np.arctan2(v[..., 1], v[..., 0])
    return r, theta, phi


def regular_all(p: int, k: float, v):
    """R_n^m(v) = j_n(k|v|) Y_n^m(v/|v|) for n < p: shape (p^2, npts)."""
    r, th, ph = cart2sph(v)
    Y = ylm_all(p, th, ph)
    ns, _ = nm_of(p * p)
    J = sph_jn(ns[:, None], k * r[None, :])
    return J * Y


def singular_all(p: int, k: float, v):
    """S_n^m(v) = h_n(k|v|) Y_n^m(v/|v|) for n < p: shape (p^2, npts)."""
    r, th, ph = cart2sph(v)
    Y = ylm_all(p, th, ph)
    ns, _ = nm_of(p * p)
    H = sph_hn(ns[:, None], k * r[None, :])
    return H * Y


@lru_cache(maxsize=None)
def gaunt_table(p: int):
    """Gaunt integrals gt[a, b, l] = integral over the unit sphere of
    Y_a conj(Y_b) conj(Y_{l, m_a - m_b}) for a, b < p^2 and l < 2p - 1
    (zero where |m_a - m_b| > l).

    Computed by tensor quadrature on the sphere: Gauss-Legendre in cos(theta)
    and the trapezoidal rule in phi, both exact for the polynomial degrees
    involved (at most 4p - 4 in cos theta, 4p - 4 in the azimuthal frequency).
    """
    P = p * p
    lmax = 2 * p - 1
    nth = 2 * p + 2
    nph = 4 * p + 2
    xg, wg = np.polynomial.legendre.leggauss(nth)
    theta = np.arccos(xg)
    phi = 2 * pi * np.arange(nph) / nph
    TH, PH = np.meshgrid(theta, phi, indexing="ij")
    W = (wg[:, None] * np.full(nph, 2 * pi / nph)[None, :]).ravel()
    Yall = ylm_all(lmax, TH.ravel(), PH.ravel())  # (lmax^2, nq)
    ns, ms = nm_of(P)
    gt = np.zeros((P, P, lmax), dtype=np.float64)
    for a in range(P):
        for b in range(P):
            mu = ms[a] - ms[b]
            # selection rules of the integral (|mu| <= l, triangle, parity):
            # the quadrature would leave rounding noise there, so skip them
            ls = np.arange(max(abs(mu), abs(ns[a] - ns[b])), min(ns[a] + ns[b], lmax - 1) + 1)
            ls = ls[(ns[a] + ns[b] + ls) % 2 == 0]
            if len(ls) == 0:
                continue
            f = W * Yall[a] * np.conj(Yall[b])
            vals = np.conj(Yall[ls * ls + ls + mu]) @ f
            gt[a, b, ls] = vals.real
    return gt


def regular_grad_all(p: int, k: float, v):
    """Cartesian gradient of R_n^m(v) = j_n(k|v|) Y_n^m(v/|v|) for n < p:
    shape (3, p^2, npts).  Used for dipole sources (the normal derivative of
    the source-side expansion, paper Sec. 5.2, Eq. (bem) second term).

    The gradient of a regular wave function is exact in the neighbouring
    degrees (the addition theorem's differentiation rule; from the Bessel
    recurrences j_n' -+ (n+1 or -n)/x j_n = j_{n-1} or -j_{n+1} and the
    recurrences of Y_n^m in cos(theta) and sin(theta) e^{+-i phi}):
      d/dz R_n^m       = k (A R_{n-1}^m - B R_{n+1}^m)
      (d/dx + i d/dy) R_n^m = k (C R_{n-1}^{m+1} + D R_{n+1}^{m+1})
      (d/dx - i d/dy) R_n^m = -k (E R_{n-1}^{m-1} + F R_{n+1}^{m-1})
    A = sqrt((n^2 - m^2) / ((2n-1)(2n+1))),  B = sqrt(((n+1)^2 - m^2) / ((2n+1)(2n+3))),
    C = sqrt((n-m)(n-m-1) / ((2n-1)(2n+1))), D = sqrt((n+m+1)(n+m+2) / ((2n+1)(2n+3))),
    E = sqrt((n+m)(n+m-1) / ((2n-1)(2n+1))), F = sqrt((n-m+1)(n-m+2) / ((2n+1)(2n+3))),
    with R of order |m| > n taken as zero.  Orthonormal Y with the
    Condon-Shortley phase (function ylm).  Needs R up to degree p; regular on
    the polar axis and at the centre."""
    v = np.atleast_2d(np.asarray(v, dtype=np.float64))
    Rall = regular_all(p + 1, k, v)                       # degrees n <= p
    npts = v.shape[0]
    zero = np.zeros(npts, dtype=np.complex128)

    def R(n, m):
        return Rall[idx(n, m)] if 0 <= n and abs(m) <= n else zero

    out = np.zeros((3, p * p, npts), dtype=np.complex128)
    for n in range(p):
        lo = (2 * n - 1) * (2 * n + 1)
        hi = (2 * n + 1) * (2 * n + 3)
        for m in range(-n, n + 1):
            A = sqrt((n * n - m * m) / lo) if n > 0 else 0.0
            B = sqrt(((n + 1) ** 2 - m * m) / hi)
            C = sqrt((n - m) * (n - m - 1) / lo) if n > 0 else 0.0
            D = sqrt((n + m + 1) * (n + m + 2) / hi)
            E = sqrt((n + m) * (n + m - 1) / lo) if n > 0 else 0.0
            F = sqrt((n - m + 1) * (n - m + 2) / hi)
            dz = k * (A * R(n - 1, m) - B * R(n + 1, m))
            dplus = k * (C * R(n - 1, m + 1) + D * R(n + 1, m + 1))
            dminus = -k * (E * R(n - 1, m - 1) + F * R(n + 1, m - 1))
            a = idx(n, m)
            out[0, a] = 0.5 * (dplus + dminus)
            out[1, a] = (dplus - dminus) / 2j
            out[2, a] = dz
    return out
