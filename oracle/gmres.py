"""Restarted flexible right-preconditioned GMRES (oracle, FP64).

Paper Sec. 3 (GMRES(m), restarts limit storage) and Sec. 4 (right
preconditioning A M^-1 x^ = b, so the minimised residual is the true one);
Sec. 6 (zero initial iterate, stop when the relative residual is below the
tolerance).  Readings:

G1  stop when the residual estimate |g_{j+1}| < rtol ||b||; the true
    residual is reported at exit.
G2  at most maxit preconditioner applications in total (default 20 m).
G3  modified Gram-Schmidt Arnoldi.
G4  complex Givens rotation c = |a| / nu, s = (a/|a|) conj(b) / nu,
    nu = sqrt(|a|^2 + |b|^2); if a = 0 then c = 0, s = 1.
G5  iterations = preconditioner applications summed over restarts.
G6  h_{j+1,j} <= 1e-14 ||w|| is a lucky breakdown: solve and stop.
B5  the preconditioner may be a nonlinear (inexact) solve, so the
    flexible variant keeps Z = [M^-1 v_1, ...] and updates x with Z y.
"""
from __future__ import annotations

import numpy as np


def givens(a: complex, b: complex):
    """G4."""
    if a == 0:
        return 0.0, 1.0 + 0.0j
    nu = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    c = abs(a) / nu
    s = (a / abs(a)) * np.conj(b) / nu
    return c, s


def fgmres(A, b, M=None, x0=None, m=30, rtol=1e-6, maxit=None):
    """Solve A x = b.  A and M are callables on complex128 vectors.
    Returns (x, info) with info = dict(iters, restarts, converged,
    relres_est, relres_true, history)."""
    b = np.asarray(b, dtype=np.complex128)
    N = len(b)
    if maxit is None:
        maxit = 20 * m
    x = np.zeros(N, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return np.zeros(N, dtype=np.complex128), dict(iters=0, restarts=0, converged=True,
                                                      relres_est=0.0, relres_true=0.0, history=[])
    iters = 0
    restarts = 0
    history = []
    converged = False
    relres = None
    while True:
        r = b - A(x)
        beta = np.linalg.norm(r)
        relres = beta / bnorm
        if relres < rtol:
            converged = True
            break
        if iters >= maxit:
            break
        V = np.zeros((m + 1, N), dtype=np.complex128)
        Z = np.zeros((m, N), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        stop = False
        for j in range(m):
            Z[j] = M(V[j]) if M is not None else V[j]
            w = A(Z[j])
            iters += 1
            wnorm0 = np.linalg.norm(w)
            for i in range(j + 1):              # G3: modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            hnext = np.linalg.norm(w)
            H[j + 1, j] = hnext
            breakdown = hnext <= 1e-14 * wnorm0
            for i in range(j):                  # previous rotations
                a_, b_ = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a_ + sn[i] * b_
                H[i + 1, j] = -np.conj(sn[i]) * a_ + cs[i] * b_
            c, s = givens(H[j, j], H[j + 1, j])
            cs[j], sn[j] = c, s
            H[j, j] = c * H[j, j] + s * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            relres = abs(g[j + 1]) / bnorm
            history.append(relres)
            j_done = j + 1
            if relres < rtol or breakdown or iters >= maxit:
                stop = True
                break
            V[j + 1] = w / hnext
        # x += Z y with H y = g (upper triangular)
        y = np.zeros(j_done, dtype=np.complex128)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        x = x + y @ Z[:j_done]
        if stop:
            converged = relres < rtol or breakdown
            break
        restarts += 1
    relres_true = np.linalg.norm(b - A(x)) / bnorm
    return x, dict(iters=iters, restarts=restarts, converged=bool(converged),
                   relres_est=float(relres), relres_true=float(relres_true),
                   history=history)
