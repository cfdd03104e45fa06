"""Pins for the oracle's FDM operator, GMRES and BEM preconditioner."""
import numpy as np
import pytest

from oracle import bem, fdm, gmres


def test_fdm_discrete_eigenvector():
    """sin(a pi x) sin(b pi y) sin(c pi z) is an eigenvector of the 7-point
    operator with eigenvalue (4/h^2) sum sin^2(. pi h / 2) - k^2."""
    n, k = 9, 3.3
    h = 1 / (n + 1)
    g = np.arange(1, n + 1) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    for (a, b, c) in [(1, 1, 1), (2, 5, 3), (9, 1, 4)]:
        u = (np.sin(a * np.pi * X) * np.sin(b * np.pi * Y) * np.sin(c * np.pi * Z)).ravel()
        lam = 4 / h ** 2 * sum(np.sin(t * np.pi * h / 2) ** 2 for t in (a, b, c)) - k * k
        np.testing.assert_allclose(fdm.fdm_apply(u, n, k), lam * u, atol=1e-9 * abs(lam))


def test_fdm_matches_assembled_matrix():
    n, k = 4, 2.0
    N = n ** 3
    A = np.column_stack([fdm.fdm_apply(e, n, k) for e in np.eye(N)])
    assert np.allclose(A, A.T)
    h = 1 / (n + 1)
    assert np.allclose(np.diag(A), 6 / h ** 2 - k * k)
    # each row has at most 6 off-diagonal entries equal to -1/h^2
    off = A - np.diag(np.diag(A))
    assert np.all(np.isin(np.round(off * h * h, 12), [0.0, -1.0]))
    assert np.all((off != 0).sum(1) <= 6)


def test_gmres_matches_direct_solve():
    rng = np.random.default_rng(0)
    N = 40
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)) + 20 * np.eye(N)
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    x, info = gmres.fgmres(lambda v: A @ v, b, m=10, rtol=1e-12)
    assert info["converged"]
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    assert abs(info["relres_true"] - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) < 1e-15


def test_gmres_full_space_terminates():
    """GMRES(m >= N) finds the solution in at most N iterations."""
    rng = np.random.default_rng(1)
    N = 12
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    b = rng.standard_normal(N) + 0j
    x, info = gmres.fgmres(lambda v: A @ v, b, m=N, rtol=1e-10)
    assert info["iters"] <= N
    assert info["relres_true"] < 1e-9


def test_gmres_exact_preconditioner_one_step():
    rng = np.random.default_rng(2)
    N = 30
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    Ainv = np.linalg.inv(A)
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    x, info = gmres.fgmres(lambda v: A @ v, b, lambda v: Ainv @ v, m=5, rtol=1e-10)
    assert info["iters"] == 1
    assert info["relres_true"] < 1e-12


def test_gmres_residual_history_monotone():
    rng = np.random.default_rng(3)
    N = 60
    A = rng.standard_normal((N, N)) + 3 * np.eye(N)
    b = rng.standard_normal(N) + 0j
    _, info = gmres.fgmres(lambda v: A @ v, b, m=60, rtol=1e-8)
    h = np.array(info["history"])
    assert np.all(np.diff(h) <= 1e-14)


def test_gmres_not_converged_reports():
    rng = np.random.default_rng(4)
    N = 50
    A = rng.standard_normal((N, N))
    b = rng.standard_normal(N) + 0j
    _, info = gmres.fgmres(lambda v: A @ v, b, m=5, rtol=1e-12, maxit=7)
    assert not info["converged"] and info["iters"] == 7


def test_givens_annihilates():
    for a, b in [(1 + 2j, 3 - 1j), (0j, 2 + 1j), (-2.0 + 0j, 1e-3j)]:
        c, s = gmres.givens(a, b)
        assert abs(-np.conj(s) * a + c * b) < 1e-15
        assert abs(abs(c * a + s * b) - np.sqrt(abs(a) ** 2 + abs(b) ** 2)) < 1e-14


def test_preconditioner_manufactured_solution():
    """With f = (3 pi^2 - k^2) sin(pi x) sin(pi y) sin(pi z) the continuous
    solution is u = sin sin sin; the BEM representation (Sec. 5.2) with an
    exact inner solve must reproduce it to O(h), shrinking as h does.  This
    fixes the sign of the volume term and the boundary scaling."""
    errs = []
    for n in (7, 11, 15):
        k = 3.0
        pr = bem.Problem(n, k, 4, 8, 0.4)
        x = pr.x_vol
        u = np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.sin(np.pi * x[:, 2])
        z, _ = pr.precond((3 * np.pi ** 2 - k * k) * u, method="direct", inner_rtol=1e-12)
        errs.append(np.linalg.norm(z - u) / np.linalg.norm(u))
    assert errs[0] < 0.05 and errs[2] < errs[1] < errs[0]
    # roughly first order in h
    assert errs[0] / errs[2] > 1.6


def test_preconditioner_fmm_vs_dense():
    """FMM-based Passes A/B/C with a tight inner GMRES reproduce the dense
    direct-sum preconditioner with an exact solve to FMM accuracy."""
    n, k = 8, 4.0
    pr = bem.Problem(n, k, 10, 4, 0.4)
    rng = np.random.default_rng(7)
    r = rng.standard_normal(n ** 3) + 1j * rng.standard_normal(n ** 3)
    zd, _ = pr.precond(r, method="direct", inner="dense")
    zf, its = pr.precond(r, method="fmm", inner_rtol=1e-12)
    assert its > 0
    assert np.linalg.norm(zf - zd) / np.linalg.norm(zd) < 1e-5


def test_preconditioned_gmres_beats_unpreconditioned():
    n, k = 10, 4.0
    pr = bem.Problem(n, k, 4, 8, 0.4)
    rng = np.random.default_rng(8)
    b = rng.uniform(-1, 1, n ** 3) + 0j
    A = lambda u: fdm.fdm_apply(u, n, k)
    _, i0 = gmres.fgmres(A, b, None, m=30, rtol=1e-6)
    _, i1 = gmres.fgmres(A, b, lambda r: pr.precond(r, inner_rtol=1e-4)[0], m=30, rtol=1e-6)
    assert i1["converged"] and i0["converged"]
    assert i1["iters"] * 4 < i0["iters"]


def test_single_layer_is_near_singular_at_the_first_cube_eigen_wavenumber():
    """The single-layer operator of the boundary equation (Eq. (ubound)) is
    not invertible when k^2 is an interior Dirichlet eigenvalue of the cube
    (k = pi sqrt(3) = 5.441 for the first mode); the collocated matrix V of
    the preconditioner's inner solve shows it as a dip of its smallest
    singular value near that k (shifted by the discretisation), an order of
    magnitude below its value away from it."""
    n = 7
    ks = np.linspace(4.8, 6.2, 29)
    smin = []
    for k in ks:
        pr = bem.Problem(n, k, 4, 64, 0.4)
        X = pr.x_bnd
        d = X[:, None, :] - X[None, :, :]
        r = np.sqrt(np.sum(d * d, axis=-1))
        np.fill_diagonal(r, 1.0)
        V = pr.h ** 2 * np.exp(1j * k * r) / (4 * np.pi * r)
        np.fill_diagonal(V, pr.s_bnd)
        smin.append(np.linalg.svd(V, compute_uv=False)[-1])
    smin = np.array(smin)
    i = int(np.argmin(smin))
    assert abs(ks[i] - np.pi * np.sqrt(3.0)) < 0.03 * np.pi * np.sqrt(3.0)
    assert smin[i] < 0.1 * min(smin[0], smin[-1])
