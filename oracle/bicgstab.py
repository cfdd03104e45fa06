"""Right-preconditioned BiCGSTAB (oracle, FP64).  Test infrastructure: only
tests/, the smoke check and the CPU-baseline legs of the benchmark use it.

The paper's Sec. 3 names BiCGSTAB (van der Vorst, 1992) as the
short-recurrence alternative to GMRES, and Sec. 3's figure compares the
iteration counts of the two methods under the FMM preconditioner.  The
method is van der Vorst's Bi-CGSTAB written for A M^-1 y = b, x = M^-1 y
(right preconditioning as in the paper's Sec. 4, so the monitored residual
is the true one).  Readings:

K1  right preconditioning; zero initial iterate unless x0 is given; the
    shadow residual is the initial residual.
K2  one iteration = one pass of the recurrence: two operator and two
    preconditioner applications (one of each when it stops at the half step).
K3  stop when ||r|| < rtol ||b|| (checked at the half step on s and at the
    full step on r); rho = 0 or omega = 0 is a breakdown and stops.
K4  complex inner products conjugate their first argument.
"""
from __future__ import annotations

import numpy as np


def bicgstab(A, b, M=None, x0=None, rtol=1e-6, maxit=500):
    """Solve A x = b.  A and M are callables on complex128 vectors.  Returns
    (x, info) with info = dict(iters, converged, breakdown, relres_true,
    history (relative residual after every iteration), precond_applies)."""
    b = np.asarray(b, dtype=np.complex128)
    N = len(b)
    Minv = M if M is not None else (lambda v: v)
    x = np.zeros(N, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    info = dict(iters=0, converged=False, breakdown=False, relres_true=0.0, history=[], precond_applies=0)
    if bnorm == 0:
        info["converged"] = True
        return np.zeros(N, dtype=np.complex128), info
    r = b - A(x)
    if np.linalg.norm(r) / bnorm < rtol:
        info["converged"] = True
        info["relres_true"] = np.linalg.norm(r) / bnorm
        return x, info
    rhat = r.copy()
    rho_old = alpha = omega = 1.0 + 0j
    v = np.zeros(N, dtype=np.complex128)
    p = np.zeros(N, dtype=np.complex128)
    for it in range(1, maxit + 1):
        info["iters"] = it
        rho = np.vdot(rhat, r)
        if rho == 0:
            info["breakdown"] = True
            break
        if it == 1:
            p = r.copy()
        else:
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
        phat = Minv(p)
        info["precond_applies"] += 1
        v = A(phat)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        rel_s = np.linalg.norm(s) / bnorm
        if rel_s < rtol:                         # half step
            x = x + alpha * phat
            info["history"].append(rel_s)
            info["converged"] = True
            break
        shat = Minv(s)
        info["precond_applies"] += 1
        t = A(shat)
        tt = np.vdot(t, t)
        omega = np.vdot(t, s) / tt if tt != 0 else 0.0
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rel = np.linalg.norm(r) / bnorm
        info["history"].append(rel)
        rho_old = rho
        if rel < rtol:
            info["converged"] = True
            break
        if omega == 0:
            info["breakdown"] = True
            break
    info["relres_true"] = np.linalg.norm(b - A(x)) / bnorm
    return x, info
