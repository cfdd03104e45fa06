"""7-point finite-difference Helmholtz operator (oracle, FP64).

Paper Sec. 2: the discretisation of the Helmholtz equation gives a sparse
complex symmetric indefinite system A x = b.  Reading S1: the equation is
-Lap u - k^2 u = f with u = 0 on the boundary; on the n^3 interior nodes with
h = 1/(n+1),
  (A u)_i = (6 u_i - sum of the 6 neighbours u_j) / h^2 - k^2 u_i,
neighbours outside the interior being zero.  Vectors are lexicographic with x
fastest.
"""
from __future__ import annotations

import numpy as np


def fdm_apply(u: np.ndarray, n: int, k: float) -> np.ndarray:
    h = 1.0 / (n + 1)
    U = np.asarray(u).reshape(n, n, n)          # [z, y, x]
    Up = np.zeros((n + 2, n + 2, n + 2), dtype=U.dtype)
    Up[1:-1, 1:-1, 1:-1] = U
    nb = (Up[:-2, 1:-1, 1:-1] + Up[2:, 1:-1, 1:-1] + Up[1:-1, :-2, 1:-1]
          + Up[1:-1, 2:, 1:-1] + Up[1:-1, 1:-1, :-2] + Up[1:-1, 1:-1, 2:])
    out = (6.0 * U - nb) / (h * h) - k * k * U
    return out.ravel()
