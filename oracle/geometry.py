"""Geometry of the discretised unit cube (oracle).

Interior nodes (paper Sec. 5.3, volume term of Eq. (uinter)): x = (i, j, l) h,
h = 1/(n+1), i, j, l = 1..n, lexicographic with x fastest; each carries the
midpoint quadrature weight h^3 (reading B2).

Boundary elements (paper Sec. 5.3: constant elements, no nodal points at the
corners; reading B1): one square panel of side h, area h^2, centred at every
boundary grid node that is not on an edge or corner.  Face order x=0, x=1,
y=0, y=1, z=0, z=1; within a face the first free coordinate runs fastest.
"""
from __future__ import annotations

import numpy as np


def interior_nodes(n: int) -> np.ndarray:
    h = 1.0 / (n + 1)
    g = np.arange(1, n + 1) * h
    z, y, x = np.meshgrid(g, g, g, indexing="ij")   # x varies fastest
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def boundary_panels(n: int):
    """Panel centres (6 n^2, 3) and outward unit normals (6 n^2, 3)."""
    h = 1.0 / (n + 1)
    centres, normals = [], []
    for axis in range(3):
        free = [a for a in range(3) if a != axis]
        for side, val in ((0, 0.0), (1, 1.0)):
            for b in range(1, n + 1):
                for a in range(1, n + 1):
                    x = [0.0, 0.0, 0.0]
                    x[axis] = val
                    x[free[0]] = a * h
                    x[free[1]] = b * h
                    nrm = [0.0, 0.0, 0.0]
                    nrm[axis] = -1.0 if side == 0 else 1.0
                    centres.append(x)
                    normals.append(nrm)
    return np.array(centres), np.array(normals)
