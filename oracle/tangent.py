"""Tangent (d/dk) and adjoint of the truncated FMM (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package header): only tests/ use it.

The differentiation form of the build asks for dphi/dk and for the adjoint
(conjugate transpose) of the FMM apply of Sec. 5.1.2 (Helmholtz kernel of
Sec. 5.2), checked against the oracle.  The truncated FMM is a fixed sequence
of linear stages whose coefficients depend on k.  Its adjoint takes every
stage conjugate-transposed in reverse order (apply_adjoint); its exact
k-derivative follows every stage by the product rule, in the order of the
forward pass (readings F1-F3 for the expansions):

  P2M    M_a   = sum_j q_j conj(R_a(y_j - c)),      dM_a = sum_j q_j conj(dR_a/dk)
  M2M    M_par = T M_ch,                            dM_par = dT M_ch + T dM_ch
  M2L    L_T   = sum_S T_v M_S,                     dL_T = sum_S (dT_v M_S + T_v dM_S)
  L2L    L_ch += T L_par,                           dL_ch += dT L_par + T dL_par
  L2P    phi_i = i k sum_a L_a R_a(x_i - c),        dphi_i = i sum_a L_a R_a
                                                           + i k sum_a (dL_a R_a + L_a dR_a/dk)
  P2P    G = e^{ikr}/(4 pi r),                      dG/dk = i e^{ikr}/(4 pi)
  self   sigma_i q_i,                               dsigma_i q_i

with dR_a/dk(v) = |v| j_n'(k|v|) Y_a(v^) and, in the translation operators'
Gaunt sums (module translations), F = R or S replaced by its k-derivative
|t| j_l'(k|t|) Y or |t| h_l'(k|t|) Y.  The self terms' derivatives are the
integrals of dG/dk over the point's own cell or panel divided by its weight.
"""
from __future__ import annotations

from math import pi

import numpy as np

from . import special as S
from . import translations as TT
from .fmm import FMM, _gauss
from .tree import centres, flat


def regular_dk_all(p: int, k: float, v):
    """dR_a/dk (v) = |v| j_n'(k|v|) Y_a(v^) for a < p^2: shape (p^2, npts)."""
    r, th, ph = S.cart2sph(v)
    Y = S.ylm_all(p, th, ph)
    ns, _ = S.nm_of(p * p)
    dj = S.sp.spherical_jn(ns[:, None], k * r[None, :], derivative=True)
    return r[None, :] * dj * Y


def _op_dk(kind: str, p: int, k: float, t) -> np.ndarray:
    """d/dk of translations._op: the Gaunt sum with F replaced by dF/dk."""
    P = p * p
    lmax = 2 * p - 1
    t = np.asarray(t, dtype=np.float64).reshape(1, 3)
    r, th, ph = S.cart2sph(t)
    Y = S.ylm_all(lmax, th, ph)[:, 0]
    ls, _ = S.nm_of(lmax * lmax)
    x = k * r[0]
    dj = S.sp.spherical_jn(ls, x, derivative=True)
    if kind == "RR":
        dF = r[0] * dj * Y
    else:
        dy = S.sp.spherical_yn(ls, x, derivative=True)
        dF = r[0] * (dj + 1j * dy) * Y
    AP, A, FI, C = TT._pattern(p)
    T = np.zeros((P, P), dtype=np.complex128)
    np.add.at(T, (AP, A), C * dF[FI])
    return T


def self_volume_dk(h: float, k: float, nq: int = 28) -> complex:
    """d/dk of the cell integral of G: the integral of i e^{ikr}/(4 pi) over
    [-h/2, h/2]^3, by the same pyramid decomposition as fmm.self_volume."""
    u, wu = _gauss(nq, -h / 2, h / 2)
    s, ws = _gauss(nq, 0.0, 1.0)
    U, V = np.meshgrid(u, u, indexing="ij")
    W2 = np.outer(wu, wu)
    R = np.sqrt(h * h / 4 + U * U + V * V)
    total = 0.0 + 0.0j
    for si, wsi in zip(s, ws):
        total += wsi * np.sum(W2 * si * si * 1j * np.exp(1j * k * si * R) / (4 * pi))
    return 6 * (h / 2) * total


def self_panel_dk(h: float, k: float, nq: int = 28) -> complex:
    """d/dk of the panel integral of G (triangle decomposition as in
    fmm.self_panel)."""
    u, wu = _gauss(nq, -h / 2, h / 2)
    s, ws = _gauss(nq, 0.0, 1.0)
    R = np.sqrt(h * h / 4 + u * u)
    total = 0.0 + 0.0j
    for si, wsi in zip(s, ws):
        total += wsi * np.sum(wu * si * 1j * np.exp(1j * k * si * R) / (4 * pi))
    return 4 * (h / 2) * total


def apply_dk(fmm: FMM, q, src_mask, tgt_mask, dsigma):
    """d/dk of FMM.apply(q, src_mask, tgt_mask, sigma) for fixed q, with
    dsigma the self coefficients' k-derivatives (zero at non-targets)."""
    k, p, P, L = fmm.k, fmm.p, fmm.P, fmm.L
    tr = fmm.tree
    # P2M and its tangent
    M = {L: fmm.p2m(q, src_mask)}
    dM = {L: np.zeros((8 ** L, P), dtype=np.complex128)}
    j = np.flatnonzero(src_mask)
    if len(j):
        leaf = tr.leaf[j]
        c = centres(L)[leaf]
        dR = regular_dk_all(p, k, tr.points[j] - c)
        np.add.at(dM[L], leaf, (q[j][None, :] * np.conj(dR)).T)
    # M2M
    for l in range(L - 1, 1, -1):
        s = 2 ** l
        g = np.arange(s)
        iz, iy, ix = np.meshgrid(g, g, g, indexing="ij")
        I = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
        wc = fmm.w(l + 1)
        M[l] = np.zeros((8 ** l, P), dtype=np.complex128)
        dM[l] = np.zeros((8 ** l, P), dtype=np.complex128)
        for o in np.ndindex(2, 2, 2):
            o = np.array(o)
            t = (0.5 - o) * wc
            T = TT.m2m_op(p, k, t)
            dT = _op_dk("RR", p, k, t)
            child = flat(2 * I + o, l + 1)
            M[l] += M[l + 1][child] @ T.T
            dM[l] += M[l + 1][child] @ dT.T + dM[l + 1][child] @ T.T
    # M2L
    Lc, dLc = {}, {}
    for l in range(2, L + 1):
        Lc[l] = np.zeros((8 ** l, P), dtype=np.complex128)
        dLc[l] = np.zeros((8 ** l, P), dtype=np.complex128)
        for v, (t_idx, s_idx) in tr.m2l_pairs(l).items():
            t = -np.array(v, dtype=np.float64) * fmm.w(l)
            T = TT.m2l_op(p, k, t)
            dT = _op_dk("SR", p, k, t)
            Lc[l][t_idx] += M[l][s_idx] @ T.T
            dLc[l][t_idx] += M[l][s_idx] @ dT.T + dM[l][s_idx] @ T.T
    # L2L
    for l in range(2, L):
        s = 2 ** l
        g = np.arange(s)
        iz, iy, ix = np.meshgrid(g, g, g, indexing="ij")
        I = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
        wc = fmm.w(l + 1)
        for o in np.ndindex(2, 2, 2):
            o = np.array(o)
            t = (o - 0.5) * wc
            T = TT.l2l_op(p, k, t)
            dT = _op_dk("RR", p, k, t)
            child = flat(2 * I + o, l + 1)
            par = flat(I, l)
            Lc[l + 1][child] += Lc[l][par] @ T.T
            dLc[l + 1][child] += Lc[l][par] @ dT.T + dLc[l][par] @ T.T
    # L2P
    dphi = np.zeros(len(tr.points), dtype=np.complex128)
    i = np.flatnonzero(tgt_mask)
    if len(i):
        leaf = tr.leaf[i]
        c = centres(L)[leaf]
        R = S.regular_all(p, k, tr.points[i] - c)
        dR = regular_dk_all(p, k, tr.points[i] - c)
        Ll, dLl = Lc[L][leaf].T, dLc[L][leaf].T
        dphi[i] = (1j * np.sum(Ll * R, axis=0) + 1j * k * np.sum(dLl * R, axis=0)
                   + 1j * k * np.sum(Ll * dR, axis=0))
    # P2P with dG/dk = i e^{ikr} / (4 pi), j != i
    s = 2 ** L
    src = np.flatnonzero(src_mask)
    tgt = np.flatnonzero(tgt_mask)
    src_by_leaf, tgt_by_leaf = {}, {}
    for jj, lf in zip(src, tr.leaf[src]):
        src_by_leaf.setdefault(int(lf), []).append(jj)
    for ii, lf in zip(tgt, tr.leaf[tgt]):
        tgt_by_leaf.setdefault(int(lf), []).append(ii)
    near = np.array(tr.near)
    for lf, ti in tgt_by_leaf.items():
        ti = np.array(ti)
        cc = tr.leaf_c[ti[0]]
        nb = cc + near
        ok = np.all((nb >= 0) & (nb < s), axis=1)
        sj = [src_by_leaf.get(int(f), []) for f in flat(nb[ok], L)]
        sj = np.array([x for lst in sj for x in lst], dtype=np.int64)
        if len(sj) == 0:
            continue
        d = tr.points[ti][:, None, :] - tr.points[sj][None, :, :]
        r = np.sqrt(np.sum(d * d, axis=-1))
        same = ti[:, None] == sj[None, :]
        g = np.where(same, 0.0, 1j * np.exp(1j * k * r) / (4 * pi))
        dphi[ti] += g @ q[sj]
    # self terms
    dphi[tgt_mask] += np.where(src_mask[tgt_mask], dsigma[tgt_mask] * q[tgt_mask], 0.0)
    return dphi


def apply_adjoint(fmm: FMM, y, src_mask, tgt_mask, sigma):
    """Conjugate transpose of FMM.apply(., src_mask, tgt_mask, sigma): the
    weights y live on the targets, the result on the sources.  Every stage of
    Sec. 5.1.2 conjugate-transposed, in reverse order:

      L2P^H   Lh_a(leaf) = sum_i conj(i k R_a(x_i - c)) y_i
      L2L^H   Lh_par    += sum_children T^H Lh_child          (upward)
      M2L^H   Mh_S      += sum_{T: S in list(T)} T_v^H Lh_T
      M2M^H   Mh_child   = T^H Mh_par                          (downward)
      P2M^H   out_j      = sum_a R_a(y_j - c) Mh_a
      P2P^H   out_j     += sum_{i near, i != j} conj(G(x_i, x_j)) y_i
      self    out_j     += conj(sigma_j) y_j
    """
    k, p, P, L = fmm.k, fmm.p, fmm.P, fmm.L
    tr = fmm.tree
    out = np.zeros(len(tr.points), dtype=np.complex128)
    # L2P^H
    Lh = {l: np.zeros((8 ** l, P), dtype=np.complex128) for l in range(2, L + 1)}
    i = np.flatnonzero(tgt_mask)
    if len(i):
        leaf = tr.leaf[i]
        c = centres(L)[leaf]
        R = S.regular_all(p, k, tr.points[i] - c)
        np.add.at(Lh[L], leaf, (np.conj(1j * k * R) * y[i][None, :]).T)
    # L2L^H, levels L-1 .. 2 (children at l + 1 feed their parent at l)
    for l in range(L - 1, 1, -1):
        s = 2 ** l
        g = np.arange(s)
        iz, iy, ix = np.meshgrid(g, g, g, indexing="ij")
        I = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
        wc = fmm.w(l + 1)
        for o in np.ndindex(2, 2, 2):
            o = np.array(o)
            T = TT.l2l_op(p, k, (o - 0.5) * wc)
            child = flat(2 * I + o, l + 1)
            Lh[l][flat(I, l)] += Lh[l + 1][child] @ np.conj(T)
    # M2L^H
    Mh = {l: np.zeros((8 ** l, P), dtype=np.complex128) for l in range(2, L + 1)}
    for l in range(2, L + 1):
        for v, (t_idx, s_idx) in tr.m2l_pairs(l).items():
            T = TT.m2l_op(p, k, -np.array(v, dtype=np.float64) * fmm.w(l))
            np.add.at(Mh[l], s_idx, Lh[l][t_idx] @ np.conj(T))
    # M2M^H, levels 2 .. L-1 (parent at l feeds its children at l + 1)
    for l in range(2, L):
        s = 2 ** l
        g = np.arange(s)
        iz, iy, ix = np.meshgrid(g, g, g, indexing="ij")
        I = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
        wc = fmm.w(l + 1)
        for o in np.ndindex(2, 2, 2):
            o = np.array(o)
            T = TT.m2m_op(p, k, (0.5 - o) * wc)
            child = flat(2 * I + o, l + 1)
            Mh[l + 1][child] += Mh[l][flat(I, l)] @ np.conj(T)
    # P2M^H
    j = np.flatnonzero(src_mask)
    if len(j):
        leaf = tr.leaf[j]
        c = centres(L)[leaf]
        R = S.regular_all(p, k, tr.points[j] - c)
        out[j] += np.sum(R * Mh[L][leaf].T, axis=0)
    # P2P^H: for every source leaf, the targets of its near leaves
    s = 2 ** L
    src = np.flatnonzero(src_mask)
    tgt = np.flatnonzero(tgt_mask)
    tgt_by_leaf, src_by_leaf = {}, {}
    for ii, lf in zip(tgt, tr.leaf[tgt]):
        tgt_by_leaf.setdefault(int(lf), []).append(ii)
    for jj, lf in zip(src, tr.leaf[src]):
        src_by_leaf.setdefault(int(lf), []).append(jj)
    near = np.array(tr.near)
    for lf, sj in src_by_leaf.items():
        sj = np.array(sj)
        cc = tr.leaf_c[sj[0]]
        nb = cc + near
        ok = np.all((nb >= 0) & (nb < s), axis=1)
        ti = [tgt_by_leaf.get(int(f), []) for f in flat(nb[ok], L)]
        ti = np.array([x for lst in ti for x in lst], dtype=np.int64)
        if len(ti) == 0:
            continue
        d = tr.points[ti][:, None, :] - tr.points[sj][None, :, :]
        r = np.sqrt(np.sum(d * d, axis=-1))
        same = ti[:, None] == sj[None, :]
        r = np.where(same, 1.0, r)
        G = np.where(same, 0.0, np.exp(1j * k * r) / (4 * pi * r))
        out[sj] += np.conj(G).T @ y[ti]
    # self terms
    both = src_mask & tgt_mask
    out[both] += np.conj(sigma[both]) * y[both]
    return out
