"""Seeded synthetic workloads for the FMM-preconditioned Helmholtz solver.

This module only draws random numbers and names problem sizes.  It holds none
of the method's arithmetic (no Green's function, no expansion, no stencil), so
both the CUDA path and the independent CPU oracle may take their inputs from it.

Problem (paper Sec. 2, Eq. (helm), Dirichlet variant of Sec. 6/7): the 3D
Helmholtz equation -Lap u - k^2 u = f on the unit cube, u = 0 on the boundary,
discretised on the n^3 interior nodes x = (i, j, l) h, h = 1/(n+1),
i, j, l = 1..n.  Vectors over the interior are in lexicographic order with the
x index fastest.

The paper measures on 2D MATLAB model problems and on 3D problems whose data
it does not print; these synthetic right-hand sides stand in for them.
"""
from __future__ import annotations

import numpy as np

# name -> workload description.  k is the wavenumber, p the expansion order
# (degrees 0..p-1), leaf the target number of volume nodes per leaf, theta the
# multipole acceptance parameter, restart the GMRES restart length m.
WORKLOADS = {
    # plain FP64 method, small enough for the oracle
    "helmholtz_n16_k4_p4": dict(n=16, k=4.0, p=4, leaf=32, theta=0.4, restart=30,
                                rhs="uniform_real", seed=1),
    # plain method vs FP32 form
    "helmholtz_n64_k16_p6": dict(n=64, k=16.0, p=6, leaf=64, theta=0.4, restart=50,
                                 rhs="gaussians", seed=2),
    # FP32 form at scale
    "helmholtz_n128_k32_p8": dict(n=128, k=32.0, p=8, leaf=64, theta=0.35, restart=50,
                                  rhs="complex_normal", seed=3),
    # smallest point of the fixed-kh sweep (kh = 0.3125), small enough for the oracle
    "helmholtz_n15_k5_p8": dict(n=15, k=5.0, p=8, leaf=32, theta=0.4, restart=30,
                                rhs="uniform_real", seed=6),
    # free-space volume FMM for the differentiable form
    "fmm_n64_k12_p6": dict(n=64, k=12.0, p=6, leaf=64, theta=0.4, restart=50,
                           rhs="complex_normal_unit", seed=5),
}


# Sweeps that mirror the paper's experiments in 3D (rhs uniform_real, seed 6):
# fixed kh = 0.3125 with h = 1/(n+1) halved and k doubled (the paper's
# (h, kappa) = (2^-4, 5) ... (2^-7, 40) table), and the expansion order p at
# fixed (n, k) (the paper's accuracy-vs-iterations figure).
SWEEP_KH = [dict(n=15, k=5.0), dict(n=31, k=10.0), dict(n=63, k=20.0), dict(n=127, k=40.0)]
SWEEP_KH_P = 8
SWEEP_P = dict(n=31, k=10.0, ps=[2, 3, 4, 5, 6, 7, 8, 10])


def node_coords(n: int) -> np.ndarray:
    """Interior node coordinates, shape (n^3, 3), lexicographic with x fastest."""
    h = 1.0 / (n + 1)
    i = np.arange(1, n + 1, dtype=np.float64) * h
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def rhs(kind: str, n: int, seed: int) -> np.ndarray:
    """Right-hand side f on the interior nodes as complex128, shape (n^3,)."""
    rng = np.random.default_rng(seed)
    N = n ** 3
    if kind == "uniform_real":
        return rng.uniform(-1.0, 1.0, N).astype(np.complex128)
    if kind == "gaussians":
        # 8 Gaussian sources, sigma 0.05, unit amplitude, centres uniform in
        # [0.2, 0.8]^3, over a uniform[-1, 1] background.
        centres = rng.uniform(0.2, 0.8, (8, 3))
        background = rng.uniform(-1.0, 1.0, N)
        x = node_coords(n)
        f = background.copy()
        for c in centres:
            d2 = np.sum((x - c) ** 2, axis=1)
            f += np.exp(-d2 / (2.0 * 0.05 ** 2))
        return f.astype(np.complex128)
    if kind == "complex_normal":
        # real and imaginary parts each N(0, 1)
        re = rng.standard_normal(N)
        im = rng.standard_normal(N)
        return re + 1j * im
    if kind == "complex_normal_unit":
        # circular complex normal with E|z|^2 = 1
        re = rng.standard_normal(N)
        im = rng.standard_normal(N)
        return (re + 1j * im) / np.sqrt(2.0)
    raise ValueError(f"unknown rhs kind {kind!r}")


def boundary_coords(n: int) -> np.ndarray:
    """Centres of the 6 n^2 boundary panels (boundary grid nodes off the
    cube's edges), faces x=0, x=1, y=0, y=1, z=0, z=1, first free coordinate
    fastest within a face: shape (6 n^2, 3)."""
    h = 1.0 / (n + 1)
    a = np.arange(1, n + 1) * h
    B, A = np.meshgrid(a, a, indexing="ij")          # A (first free) fastest
    out = []
    for axis in range(3):
        free = [c for c in range(3) if c != axis]
        for val in (0.0, 1.0):
            x = np.zeros((n * n, 3))
            x[:, axis] = val
            x[:, free[0]] = A.ravel()
            x[:, free[1]] = B.ravel()
            out.append(x)
    return np.concatenate(out)


def plane_wave_boundary(n: int, k: float, direction=(1.0, 2.0, 2.0)) -> np.ndarray:
    """Dirichlet data u_Gamma = exp(i k d.x) at the panel centres, d the unit
    vector along `direction` (synthetic boundary data), complex128 (6 n^2,)."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.exp(1j * k * boundary_coords(n) @ d)


def workload_rhs(name: str) -> np.ndarray:
    w = WORKLOADS[name]
    return rhs(w["rhs"], w["n"], w["seed"])


def complex_normal(shape, seed: int) -> np.ndarray:
    """Circular complex normal samples (E|z|^2 = 1), complex128."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) / np.sqrt(2.0)


def uniform_points(count: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Points uniform in [lo, hi)^3, shape (count, 3), float64."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (count, 3))


def batched_problems(count: int = 48, seed: int = 4):
    """Independent solves of uneven size: n from {24,32,48,64,96}, k uniform in
    [4, min(32, 2 pi (n+1) / 8)] (at least 8 points per wavelength), p in {4, 6}.
    Each solve s gets f ~ uniform[-1, 1] from seed 1000 + s."""
    rng = np.random.default_rng(seed)
    sizes = np.array([24, 32, 48, 64, 96])
    out = []
    for s in range(count):
        n = int(rng.choice(sizes))
        kmax = min(32.0, 2.0 * np.pi * (n + 1) / 8.0)
        k = float(rng.uniform(4.0, kmax))
        p = int(rng.choice([4, 6]))
        out.append(dict(n=n, k=k, p=p, leaf=64, theta=0.4, restart=50,
                        rhs="uniform_real", seed=1000 + s))
    return out
