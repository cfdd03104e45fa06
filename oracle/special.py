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

    Chain rule in spherical coordinates,
      grad R = rho^ dR/drho + theta^ (1/rho) dR/dtheta + phi^ (1/(rho sin theta)) dR/dphi,
    with dR/drho = k j_n'(k rho) Y (scipy's derivative), dY/dphi = i m Y and,
    for Y ~ P_n^|m|(cos theta), the Legendre identity
      (1 - x^2) dP_n^m/dx = (n + m) P_{n-1}^m - n x P_n^m,  x = cos theta,
    so dP_n^m(cos theta)/dtheta = -((n + m) P_{n-1}^m - n x P_n^m) / sin theta.
    Points on the polar axis (sin theta = 0) or at the centre are refused."""
    v = np.atleast_2d(np.asarray(v, dtype=np.float64))
    r, th, ph = cart2sph(v)
    st, ct = np.sin(th), np.cos(th)
    if np.any(r <= 0) or np.any(np.abs(st) < 1e-12):
        raise ValueError("regular_grad_all: point at the centre or on the polar axis")
    P = p * p
    ns, ms = nm_of(P)
    jn = sph_jn(ns[:, None], k * r[None, :])
    djn = sp.spherical_jn(ns[:, None], k * r[None, :], derivative=True)
    Y = ylm_all(p, th, ph)
    dY = np.empty_like(Y)
    for n in range(p):
        for m in range(-n, n + 1):
            am = abs(m)
            norm = sqrt((2 * n + 1) / (4 * pi) * factorial(n - am) / factorial(n + am))
            pn = sp.lpmv(am, n, ct)
            pn1 = sp.lpmv(am, n - 1, ct) if n >= 1 and am <= n - 1 else 0.0 * ct
            dp = -((n + am) * pn1 - n * ct * pn) / st
            d = norm * dp * np.exp(1j * am * ph)
            if m < 0:
                d = (-1) ** am * np.conj(d)
            dY[idx(n, m)] = d
    dR_drho = k * djn * Y
    dR_dth = jn * dY / r[None, :]
    dR_dph = jn * (1j * ms[:, None]) * Y / (r * st)[None, :]
    e_r = np.stack([st * np.cos(ph), st * np.sin(ph), ct])
    e_t = np.stack([ct * np.cos(ph), ct * np.sin(ph), -st])
    e_p = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)])
    return (e_r[:, None, :] * dR_drho[None] + e_t[:, None, :] * dR_dth[None]
            + e_p[:, None, :] * dR_dph[None])
