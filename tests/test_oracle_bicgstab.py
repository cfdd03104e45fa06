"""Pins for the oracle's right-preconditioned BiCGSTAB (readings K1-K4):
direct solve of a dense system, one iteration with the exact preconditioner,
the same iterates as scipy's independent implementation (unpreconditioned,
real and complex), and convergence on the FMM-preconditioned FDM system."""
import numpy as np
import pytest

from oracle import bem, bicgstab, fdm, gmres

scipy_linalg = pytest.importorskip("scipy.sparse.linalg")


def _system(seed, N, shift, cplx):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((N, N)) + shift * np.eye(N)
    b = rng.standard_normal(N)
    if cplx:
        A = A + 1j * rng.standard_normal((N, N))
        b = b + 1j * rng.standard_normal(N)
    return A, b


def test_bicgstab_matches_direct_solve():
    A, b = _system(0, 50, 25.0, True)
    x, info = bicgstab.bicgstab(lambda v: A @ v, b, rtol=1e-12)
    assert info["converged"] and not info["breakdown"]
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    assert info["relres_true"] < 1e-11


def test_bicgstab_exact_preconditioner_half_step():
    """With M = A^-1, v = A M^-1 p = p = r0, alpha = 1 and s = 0: converged
    at the half step of the first iteration with one preconditioner apply."""
    A, b = _system(1, 30, 0.0, True)
    Ainv = np.linalg.inv(A)
    x, info = bicgstab.bicgstab(lambda v: A @ v, b, lambda r: Ainv @ r, rtol=1e-10)
    assert info["iters"] == 1 and info["precond_applies"] == 1 and info["converged"]
    assert info["relres_true"] < 1e-10


@pytest.mark.parametrize("cplx", [False, True])
def test_bicgstab_iterates_match_scipy(cplx):
    """scipy's bicgstab runs the same recurrence: the iteration count and the
    solution agree (unpreconditioned)."""
    # well conditioned, so that rounding does not decide the iteration count
    A, b = _system(2, 60, 8.0 if not cplx else 20.0, cplx)
    rtol = 1e-8
    x, info = bicgstab.bicgstab(lambda v: A @ v, b, rtol=rtol, maxit=400)
    count = [0]

    def cb(_):
        count[0] += 1

    try:
        xs, flag = scipy_linalg.bicgstab(A, b, rtol=rtol, atol=0.0, maxiter=400, callback=cb)
    except TypeError:  # older scipy: tol instead of rtol
        xs, flag = scipy_linalg.bicgstab(A, b, tol=rtol, atol=0.0, maxiter=400, callback=cb)
    assert flag == 0 and info["converged"]
    assert abs(info["iters"] - count[0]) <= 1, (info["iters"], count[0])
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-6


def test_bicgstab_fmm_preconditioned_fdm():
    """On the FDM Helmholtz system the FMM preconditioner turns BiCGSTAB into
    a few iterations, like GMRES (two preconditioner applies per iteration)."""
    n, k = 8, 4.0
    pr = bem.Problem(n, k, 4, 8, 0.4)
    rng = np.random.default_rng(8)
    b = rng.uniform(-1, 1, n ** 3) + 0j
    A = lambda u: fdm.fdm_apply(u, n, k)
    M = lambda r: pr.precond(r, inner_rtol=1e-4)[0]
    _, ib = bicgstab.bicgstab(A, b, M, rtol=1e-6)
    _, ig = gmres.fgmres(A, b, M, m=30, rtol=1e-6)
    _, i0 = bicgstab.bicgstab(A, b, None, rtol=1e-6, maxit=2000)
    assert ib["converged"] and ib["relres_true"] < 1e-6
    assert ib["precond_applies"] <= 3 * ig["iters"]
    assert ib["iters"] * 4 < i0["iters"]
