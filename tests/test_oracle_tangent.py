"""Pins for the oracle's tangent (d/dk) and adjoint FMM.  Tangent: every
piece against finite differences in k of the oracle's own forward pieces
(five-point stencil, step 1e-3: truncation ~1e-13), and the self-term
derivatives at k = 0 against their closed forms.  Adjoint: the dot-product
identity <G x, y> = <x, G^H y> with the forward oracle FMM, and the conjugate
transpose of the assembled forward matrix on a tiny tree."""
from math import pi

import numpy as np
import pytest

from oracle import bem
from oracle import fmm as F
from oracle import special as S
from oracle import tangent as TG
from oracle import translations as TT

STEP = 1e-3


def five_point(f, k, e=STEP):
    return (-f(k + 2 * e) + 8 * f(k + e) - 8 * f(k - e) + f(k - 2 * e)) / (12 * e)


def test_regular_dk_matches_finite_differences():
    rng = np.random.default_rng(0)
    v = rng.uniform(-0.4, 0.4, (20, 3))
    p, k = 7, 6.0
    got = TG.regular_dk_all(p, k, v)
    fd = five_point(lambda kk: S.regular_all(p, kk, v), k)
    assert np.abs(got - fd).max() < 1e-10 * max(1.0, np.abs(got).max())


@pytest.mark.parametrize("kind,t", [("RR", [0.125, -0.0625, 0.0625]), ("SR", [0.5, 0.25, -0.75]),
                                    ("SR", [0.0, 0.0, 0.375])])
def test_translation_dk_matches_finite_differences(kind, t):
    p, k = 5, 7.0
    op = TT.m2m_op if kind == "RR" else TT.m2l_op
    got = TG._op_dk(kind, p, k, t)
    fd = five_point(lambda kk: op(p, kk, t), k)
    assert np.abs(got - fd).max() < 1e-9 * max(1.0, np.abs(got).max())


@pytest.mark.parametrize("k", [0.0, 3.0, 11.0])
def test_self_term_derivatives(k):
    h = 1.0 / 17
    dv, dp = TG.self_volume_dk(h, k), TG.self_panel_dk(h, k)
    fv = five_point(lambda kk: F.self_volume(h, kk), k)
    fp = five_point(lambda kk: F.self_panel(h, kk), k)
    assert abs(dv - fv) < 1e-9 * abs(dv) and abs(dp - fp) < 1e-9 * abs(dp)
    if k == 0.0:
        # d/dk of the integral of e^{ikr}/(4 pi r) at k = 0 is i |cell| / (4 pi)
        assert abs(dv - 1j * h ** 3 / (4 * pi)) < 1e-15
        assert abs(dp - 1j * h ** 2 / (4 * pi)) < 1e-15


def _dsigma(pr, k):
    h = pr.h
    return np.concatenate([np.full(pr.NO, TG.self_volume_dk(h, k) / h ** 3),
                           np.full(pr.NG, TG.self_panel_dk(h, k) / h ** 2)])


def test_tangent_fmm_matches_finite_differences():
    """dphi/dk of the whole truncated FMM (same tree, same p) against the
    five-point difference of the forward oracle apply."""
    n, k, p, leaf = 8, 4.0, 5, 8
    pr = bem.Problem(n, k, p, leaf, 0.4)
    rng = np.random.default_rng(1)
    N = pr.NO + pr.NG
    q = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    allm = np.ones(N, bool)
    d = TG.apply_dk(pr.fmm, q, allm, allm, _dsigma(pr, k))

    def fwd(kk):
        P = bem.Problem(n, kk, p, leaf, 0.4)
        return P.fmm.apply(q, allm, allm, P.sigma)

    fd = five_point(fwd, k)
    assert np.linalg.norm(d - fd) / np.linalg.norm(fd) < 1e-10


def test_tangent_fmm_set_masks_and_linearity():
    n, k, p, leaf = 6, 3.0, 4, 8
    pr = bem.Problem(n, k, p, leaf, 0.4)
    rng = np.random.default_rng(2)
    N = pr.NO + pr.NG
    q = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    ds = _dsigma(pr, k)
    d_all = TG.apply_dk(pr.fmm, q, pr.vol | pr.bnd, pr.vol, ds)
    assert np.all(d_all[pr.bnd] == 0)
    # splitting the sources splits the tangent (linearity in q)
    d_v = TG.apply_dk(pr.fmm, q, pr.vol, pr.vol, ds)
    d_b = TG.apply_dk(pr.fmm, q, pr.bnd, pr.vol, ds)
    assert np.allclose(d_v + d_b, d_all, rtol=1e-12, atol=1e-12 * np.abs(d_all).max())


@pytest.mark.parametrize("sets", ["all", "vol_to_bnd", "bnd_to_vol"])
def test_adjoint_dot_product_identity(sets):
    n, k, p, leaf = 8, 5.0, 5, 8
    pr = bem.Problem(n, k, p, leaf, 0.4)
    N = pr.NO + pr.NG
    rng = np.random.default_rng(3)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    y = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    sm, tm = {"all": (pr.vol | pr.bnd, pr.vol | pr.bnd), "vol_to_bnd": (pr.vol, pr.bnd),
              "bnd_to_vol": (pr.bnd, pr.vol)}[sets]
    Gx = pr.fmm.apply(np.where(sm, x, 0), sm, tm, pr.sigma)
    GHy = TG.apply_adjoint(pr.fmm, np.where(tm, y, 0), sm, tm, pr.sigma)
    assert np.all(GHy[~sm] == 0)
    lhs = np.vdot(y[tm], Gx[tm])
    rhs = np.vdot(GHy[sm], x[sm])
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_adjoint_is_the_conjugate_transpose():
    n, k, p, leaf = 4, 3.0, 4, 4
    pr = bem.Problem(n, k, p, leaf, 0.4)
    N = pr.NO + pr.NG
    allm = np.ones(N, bool)
    G = np.stack([pr.fmm.apply(e, allm, allm, pr.sigma) for e in np.eye(N, dtype=np.complex128)], axis=1)
    rng = np.random.default_rng(4)
    y = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    got = TG.apply_adjoint(pr.fmm, y, allm, allm, pr.sigma)
    ref = G.conj().T @ y
    assert np.linalg.norm(got - ref) < 1e-13 * np.linalg.norm(ref)
