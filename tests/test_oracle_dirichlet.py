"""Pins for the oracle's inhomogeneous-Dirichlet pieces: the gradient of the
regular basis, the double-layer kernel and sums (direct and FMM), the
finite-difference lift of boundary data and the BEM solve with boundary data
(paper Sec. 5.2-5.3, Eq. (ubound) and Eq. (uinter))."""
from math import pi, sqrt

import numpy as np
import pytest

from oracle import dirichlet as D
from oracle import fdm, geometry, gmres
from oracle import fmm as F
from oracle import special as S
from paper_1608_02461_gb300 import inputs


def test_regular_gradient_matches_finite_differences():
    """grad R_a against central differences of R_a itself (step 1e-5: the
    difference error is ~1e-10 of the values)."""
    rng = np.random.default_rng(0)
    v = rng.uniform(-0.3, 0.3, (25, 3))
    p, k = 7, 9.0
    g = S.regular_grad_all(p, k, v)
    d = 1e-5
    fd = np.stack([(S.regular_all(p, k, v + d * e) - S.regular_all(p, k, v - d * e)) / (2 * d)
                   for e in np.eye(3)])
    assert np.abs(g - fd).max() < 1e-8 * max(1.0, np.abs(g).max())


def test_regular_gradient_degree_zero_closed_form():
    """R_0 = j_0(k rho) / sqrt(4 pi), so grad R_0 = -k j_1(k rho) rho^ / sqrt(4 pi)."""
    rng = np.random.default_rng(1)
    v = rng.uniform(-1, 1, (10, 3))
    k = 4.0
    r = np.linalg.norm(v, axis=1)
    kr = k * r
    j1 = np.sin(kr) / kr ** 2 - np.cos(kr) / kr
    want = -k * j1[None, :] * (v / r[:, None]).T / sqrt(4 * pi)
    got = S.regular_grad_all(3, k, v)[:, 0, :]
    assert np.abs(got - want).max() < 1e-14


def test_regular_gradient_on_the_polar_axis_and_at_the_centre():
    """Points on the z axis (either side) and the centre itself, where
    spherical coordinates are singular: central differences of R_a still
    agree (lattice panels do lie on the axis of their leaf centre when n + 1
    is a power of two)."""
    v = np.array([[0.0, 0.0, 0.2], [0.0, 0.0, -0.35], [0.0, 0.0, 0.0], [1e-9, 0.0, 0.3]])
    p, k = 6, 5.0
    g = S.regular_grad_all(p, k, v)
    # five-point differences with a wide step: near the axis the Legendre
    # values of R carry the cancellation of 1 - cos^2(theta), so the step
    # stays far from the axis scale of rounding
    d = 1e-3

    def Rv(x):
        return S.regular_all(p, k, x)

    fd = np.stack([(-Rv(v + 2 * d * e) + 8 * Rv(v + d * e) - 8 * Rv(v - d * e) + Rv(v - 2 * d * e)) / (12 * d)
                   for e in np.eye(3)])
    assert np.all(np.isfinite(g))
    assert np.abs(g - fd).max() < 1e-8 * max(1.0, np.abs(g).max())


def test_dgreen_dn_is_the_source_normal_derivative_of_g():
    """dG/dn_y against central differences of G in y along n_y (fixes the
    sign and the dr/dn factor of reading S3)."""
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (6, 3))
    y = rng.uniform(0, 1, (5, 3))
    ny = rng.standard_normal((5, 3))
    ny /= np.linalg.norm(ny, axis=1)[:, None]
    k = 6.0
    d = 1e-6
    fd = (F.green(x, y + d * ny, k) - F.green(x, y - d * ny, k)) / (2 * d)
    got = D.dgreen_dn(x, y, ny, k)
    assert np.abs(got - fd).max() < 1e-7 * np.abs(got).max()


@pytest.mark.parametrize("x", [[0.5, 0.5, 0.5], [0.3, 0.62, 0.45]])
def test_double_layer_gauss_identity(x):
    """k = 0: the closed-surface integral of dG/dn_y is -1 at every interior
    point.  The panel sum (edges excluded, one-point rule) approaches it at
    first order in h."""
    errs = []
    for n in (7, 15, 31):
        X, N = geometry.boundary_panels(n)
        h = 1.0 / (n + 1)
        s = (h * h * D.dgreen_dn(np.array([x]), X, N, 0.0)).sum()
        assert abs(s.imag) == 0.0
        errs.append(abs(s + 1.0))
        assert errs[-1] < 1.2 * h
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_green_representation_of_a_plane_wave():
    """Eq. (uinter) with f = 0 and exact boundary data of u = exp(i k d.x):
    u(x) = sum_j h^2 (du/dn)_j G(x, y_j) - sum_j h^2 u_j dG/dn_y(x, y_j)
    at interior points away from the boundary, to first order in h.  A wrong
    sign on either layer leaves an O(1) error."""
    k = 5.0
    dvec = np.array([2.0, -1.0, 2.0]) / 3.0
    x = np.array([[0.5, 0.5, 0.5], [0.35, 0.6, 0.42], [0.62, 0.41, 0.55]])
    ue = np.exp(1j * k * x @ dvec)
    errs = []
    for n in (15, 31, 63):
        X, N = geometry.boundary_panels(n)
        h = 1.0 / (n + 1)
        ub = np.exp(1j * k * X @ dvec)
        dudn = 1j * k * (N @ dvec) * ub
        u = h * h * (F.green(x, X, k) @ dudn - D.dgreen_dn(x, X, N, k) @ ub)
        errs.append(np.abs(u - ue).max())
    assert errs[0] < 0.1
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1]


def test_double_layer_direct_masks_and_diagonal():
    """Targets outside the mask stay zero, a point never acts on itself, and
    the sum is linear in the strengths."""
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 1, (40, 3))
    nrm = rng.standard_normal((40, 3))
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    mu = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    src = rng.uniform(size=40) < 0.5
    tgt = rng.uniform(size=40) < 0.5
    phi = D.double_layer_direct(pts, mu, nrm, src, tgt, 3.0)
    assert np.all(phi[~tgt] == 0)
    for i in np.flatnonzero(tgt):
        js = [j for j in np.flatnonzero(src) if j != i]
        want = sum(mu[j] * D.dgreen_dn(pts[i:i + 1], pts[j:j + 1], nrm[j:j + 1], 3.0)[0, 0] for j in js)
        assert abs(phi[i] - want) < 1e-12 * max(1.0, abs(want))
    phi2 = D.double_layer_direct(pts, (2 - 1j) * mu, nrm, src, tgt, 3.0)
    assert np.allclose(phi2, (2 - 1j) * phi, rtol=1e-13, atol=1e-13)


def _dipole_problem(N, seed):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.01, 0.99, (N, 3))
    nrm = rng.standard_normal((N, 3))
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    mu = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return pts, nrm, mu


def test_dipole_fmm_converges_to_direct_sum():
    """The dipole FMM (P2M from the basis gradient, the rest of Sec. 5.1.2
    unchanged) approaches the direct double-layer sum geometrically in p."""
    pts, nrm, mu = _dipole_problem(400, 4)
    allm = np.ones(len(pts), bool)
    k = 6.0
    d = D.double_layer_direct(pts, mu, nrm, allm, allm, k)
    errs = []
    for p in (3, 5, 7, 9):
        f = D.double_layer_fmm(F.FMM(pts, len(pts), 4, 0.4, k, p), mu, nrm, allm, allm)
        errs.append(np.linalg.norm(f - d) / np.linalg.norm(d))
    assert all(errs[i + 1] < 0.3 * errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-4


def test_dipole_fmm_high_order_matches_direct():
    pts, nrm, mu = _dipole_problem(200, 5)
    rng = np.random.default_rng(6)
    src = rng.uniform(size=200) < 0.6
    tgt = rng.uniform(size=200) < 0.6
    k = 3.0
    d = D.double_layer_direct(pts, mu, nrm, src, tgt, k)
    f = D.double_layer_fmm(F.FMM(pts, len(pts), 4, 0.4, k, 13), mu, nrm, src, tgt)
    assert np.all(f[~tgt] == 0)
    assert np.linalg.norm(f - d) / np.linalg.norm(d) < 5e-8


def test_dirichlet_lift_is_exact_for_cubics():
    """The 7-point Laplacian is exact on polynomials of degree <= 3 in each
    variable, so for such u: A_h u_int - lift(u_Gamma) = -Lap u - k^2 u at the
    interior nodes to rounding.  Uses every face and orientation."""
    n, k = 9, 2.5

    def u(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return (1 + 2 * X - Y + 3j * Z + X * X * Y - 2 * Y * Z * Z + (1 + 1j) * X * Y * Z
                + 0.5 * X ** 3 - 1.5j * Z ** 3 + 0.25 * Y ** 3)

    def lap(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return 2 * Y - 4 * Y + 3 * X - 9j * Z + 1.5 * Y

    xv = geometry.interior_nodes(n)
    xb, _ = geometry.boundary_panels(n)
    f = -lap(xv) - k * k * u(xv)
    got = fdm.fdm_apply(u(xv), n, k) - D.dirichlet_lift(n, u(xb))
    assert np.abs(got - f).max() < 1e-9 * np.abs(f).max()


def test_panel_of_neighbour_counts():
    n = 6
    nb = D.panel_of_neighbour(n)
    # every panel is the neighbour of exactly one interior node
    used = nb[nb >= 0]
    assert len(used) == 6 * n * n and len(np.unique(used)) == 6 * n * n
    # interior nodes with 0, 1, 2, 3 boundary neighbours: inside, faces, edges, corners
    cnt = (nb >= 0).sum(axis=1)
    assert [int((cnt == c).sum()) for c in range(4)] == [(n - 2) ** 3, 6 * (n - 2) ** 2, 12 * (n - 2), 8]


def _plane_wave_data(pr, k, dvec):
    ub = np.exp(1j * k * pr.x_bnd @ dvec)
    ue = np.exp(1j * k * pr.x_vol @ dvec)
    return ub, ue


def test_bem_solve_plane_wave_converges():
    """Eq. (ubound) then Eq. (uinter) with Dirichlet data of a plane wave and
    f = 0 reproduce it in the interior to first order in h (exact inner
    solve, direct sums)."""
    k = 3.0
    dvec = np.array([1.0, 2.0, 2.0]) / 3.0
    errs = []
    for n in (7, 13):
        pr = D.DirichletProblem(n, k, 4, 8, 0.4)
        ub, ue = _plane_wave_data(pr, k, dvec)
        u, _, _ = pr.bem_solve(np.zeros(pr.NO), ub, method="direct", inner="dense")
        errs.append(np.linalg.norm(u - ue) / np.linalg.norm(ue))
    assert errs[0] < 0.03
    assert errs[0] / errs[1] > 1.5     # h ratio 1.75


def test_bem_solve_with_volume_and_boundary_data():
    """u = plane wave + sin(pi x) sin(pi y) sin(pi z): f = (3 pi^2 - k^2) times
    the sine part, Dirichlet data from the plane wave.  Both data terms act
    together; the interior error stays first order in h."""
    k = 3.0
    dvec = np.array([0.0, 0.6, 0.8])
    errs = []
    for n in (7, 11):
        pr = D.DirichletProblem(n, k, 4, 8, 0.4)
        ub, ue = _plane_wave_data(pr, k, dvec)
        x = pr.x_vol
        s = np.sin(pi * x[:, 0]) * np.sin(pi * x[:, 1]) * np.sin(pi * x[:, 2])
        u, _, _ = pr.bem_solve((3 * pi ** 2 - k * k) * s, ub, method="direct", inner="dense")
        errs.append(np.linalg.norm(u - ue - s) / np.linalg.norm(ue + s))
    assert errs[0] < 0.05 and errs[1] < errs[0]


def test_bem_solve_fmm_matches_direct():
    """All five sums by the FMM with an iterative inner solve reproduce the
    direct sums with a dense solve to FMM accuracy."""
    n, k = 8, 4.0
    pr = D.DirichletProblem(n, k, 10, 4, 0.4)
    rng = np.random.default_rng(8)
    f = rng.standard_normal(pr.NO) + 1j * rng.standard_normal(pr.NO)
    ub = rng.standard_normal(pr.NG) + 1j * rng.standard_normal(pr.NG)
    ud, _, _ = pr.bem_solve(f, ub, method="direct", inner="dense")
    uf, _, its = pr.bem_solve(f, ub, method="fmm", inner_rtol=1e-12)
    assert its > 0
    assert np.linalg.norm(uf - ud) / np.linalg.norm(ud) < 1e-5


def test_fdm_solve_with_dirichlet_data():
    """A_h u = f + lift(u_Gamma) for a plane wave (f = 0): the discrete
    solution is second-order accurate.  GMRES with the homogeneous
    preconditioner (it acts on residuals, which carry no boundary data)
    reaches the same solution from zero and from the BEM solution, the latter
    in no more iterations."""
    k = 3.0
    dvec = np.array([1.0, 2.0, 2.0]) / 3.0
    errs = []
    for n in (7, 11):
        pr = D.DirichletProblem(n, k, 4, 8, 0.4)
        ub, ue = _plane_wave_data(pr, k, dvec)
        b = D.dirichlet_lift(n, ub)
        A = np.stack([fdm.fdm_apply(e, n, k) for e in np.eye(n ** 3)], axis=1)
        errs.append(np.linalg.norm(np.linalg.solve(A, b) - ue) / np.linalg.norm(ue))
    assert errs[0] < 5e-3 and 1.8 < errs[0] / errs[1] < 2.8
    n = 7
    pr = D.DirichletProblem(n, k, 4, 8, 0.4)
    ub, _ = _plane_wave_data(pr, k, dvec)
    b = D.dirichlet_lift(n, ub)
    A = lambda v: fdm.fdm_apply(v, n, k)
    M = lambda r: pr.precond(r, method="direct", inner_rtol=1e-8)[0]
    x, info = gmres.fgmres(A, b, M, m=30, rtol=1e-10)
    x0, _, _ = pr.bem_solve(np.zeros(pr.NO), ub, method="direct", inner="dense")
    x1, info1 = gmres.fgmres(A, b, M, x0=x0, m=30, rtol=1e-10)
    assert info["converged"] and info1["converged"]
    assert np.linalg.norm(x1 - x) / np.linalg.norm(x) < 1e-8
    assert info1["iters"] <= info["iters"]


def test_input_boundary_data_follows_the_panel_order():
    """The seeded-input module's panel centres and plane-wave data are in the
    oracle's panel order (faces x=0, x=1, y=0, y=1, z=0, z=1, first free
    coordinate fastest)."""
    for n in (3, 6):
        X, _ = geometry.boundary_panels(n)
        assert np.array_equal(inputs.boundary_coords(n), X)
        d = np.array([1.0, 2.0, 2.0]) / 3.0
        assert np.allclose(inputs.plane_wave_boundary(n, 4.0), np.exp(4j * X @ d), rtol=0, atol=1e-15)
