"""Thin ctypes binding of the C ABI in include/hfmm.h.

Argument marshalling only: every step of the computation runs in the CUDA
library libhfmm.so.  PyTorch supplies device memory (complex128 tensors on a
CUDA device) and the current stream.  If the library is missing this module
raises on first use; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HFMM_OK = 0
HFMM_ERR_INVALID_ARG = -1
HFMM_ERR_CUDA = -2
HFMM_ERR_NOMEM = -3
HFMM_ERR_NONFINITE = -4
HFMM_ERR_NOT_CONVERGED = -5
HFMM_ERR_TIMEOUT = -6
HFMM_ERR_UNSUPPORTED = -7

HFMM_FP64 = 0
HFMM_FP32 = 1
SET_VOL = 1
SET_BND = 2
FWD = 0
ADJ = 1
DK = 2
DLP = 3

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhfmm.so")


class hfmm_params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("theta", ctypes.c_double), ("leaf_size", ctypes.c_int),
                ("k", ctypes.c_double), ("precision", ctypes.c_int)]


class hfmm_gmres_params(ctypes.Structure):
    _fields_ = [("restart_m", ctypes.c_int), ("rtol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("inner_rtol", ctypes.c_double), ("inner_maxit", ctypes.c_int),
                ("inner_m", ctypes.c_int)]


class hfmm_gmres_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int),
                ("inner_iters_total", ctypes.c_int), ("status", ctypes.c_int),
                ("relres_est", ctypes.c_double), ("relres_true", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)), ("history_len", ctypes.c_int)]


NSTAGES = 9
STAGES = ["gather", "p2m", "m2m", "m2l", "l2l", "l2p", "p2p", "fdm", "bnd"]


class hfmm_stats(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("p", ctypes.c_int), ("n_vol", ctypes.c_int64),
                ("n_bnd", ctypes.c_int64), ("leaves", ctypes.c_int64),
                ("m2l_pairs", ctypes.c_int64), ("p2p_pairs", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("ms_last_apply", ctypes.c_double),
                ("launches", ctypes.c_int64), ("stage_ms", ctypes.c_double * NSTAGES),
                ("stage_launches", ctypes.c_int64 * NSTAGES),
                ("stage_work", ctypes.c_double * NSTAGES)]


# name -> (restype, argtypes) for every entry point of include/hfmm.h
SIGNATURES = {
    "hfmm_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fmm_build_tree": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.POINTER(hfmm_params), ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "fmm_destroy_tree": (None, [ctypes.c_void_p]),
    "fmm_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                 ctypes.c_void_p]),
    "fmm_precond_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "hfmm_fdm_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "hfmm_order_for_k": (ctypes.c_int, [ctypes.c_double, ctypes.c_int]),
    "fmm_grad_k": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "hfmm_solve_grad_k": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "bem_solve_dirichlet": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "hfmm_dirichlet_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "gmres_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(hfmm_gmres_params),
                                   ctypes.POINTER(hfmm_gmres_info), ctypes.c_void_p]),
    "bicgstab_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.POINTER(hfmm_gmres_params),
                                      ctypes.POINTER(hfmm_gmres_info), ctypes.c_void_p]),
    "fmm_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(hfmm_stats)]),
    "fmm_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "gmres_solve_batched": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                           ctypes.POINTER(hfmm_gmres_params),
                                           ctypes.POINTER(hfmm_gmres_info), ctypes.c_void_p]),
    "fmm_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "fmm_set_inner_order": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "fmm_use_graphs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hfmm_direct_sum_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int64, ctypes.c_void_p, ctypes.c_double,
                                               ctypes.c_void_p, ctypes.c_void_p]),
    "hfmm_pipe_peaks": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "hfmm_partition_ranges": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "hfmm_partition_let": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_void_p]),
}

# order of hfmm_pipe_peaks' outputs
PEAKS = ("fp32_tflops", "fp64_tflops", "xu_gops", "smem_gbs", "tf32_tflops")

# scratch limit of hfmm_direct_sum_noalloc (targets)
NOALLOC_MAX_TARGETS = 1 << 18

_lib = None


def lib():
    """Load libhfmm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run python -m paper_1608_02461_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class HfmmError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {lib().hfmm_error_string(status).decode()} ({status})")


def _check(status: int, what: str):
    if status != HFMM_OK:
        raise HfmmError(status, what)


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _dev_c128(t, n, name):
    torch = _torch()
    if t.dtype != torch.complex128 or not t.is_cuda or t.numel() != n or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA complex128 tensor with {n} entries")
    return t


@dataclass
class GmresInfo:
    iters: int
    restarts: int
    inner_iters_total: int
    status: int
    relres_est: float
    relres_true: float
    history: list


class Tree:
    """Handle of fmm_build_tree: octree, lists, operators and self terms for
    one grid (n), wavenumber k and expansion order p."""

    def __init__(self, n: int, k: float, p: int, theta: float = 0.4, leaf: int = 64,
                 precision: str = "fp64", vol_xyz=None, bnd_xyz=None, stream=None):
        L = lib()
        self.n, self.k, self.p, self.theta, self.leaf = n, k, p, theta, leaf
        self.precision = precision
        prm = hfmm_params(p, theta, leaf, k, HFMM_FP32 if precision == "fp32" else HFMM_FP64)
        handle = ctypes.c_void_p()
        n_vol = vol_xyz.shape[0] if vol_xyz is not None else n ** 3
        n_bnd = bnd_xyz.shape[0] if bnd_xyz is not None else 6 * n * n
        self._keep = (vol_xyz, bnd_xyz)
        st = L.fmm_build_tree(n, _ptr(vol_xyz), n_vol, _ptr(bnd_xyz), n_bnd, ctypes.byref(prm),
                              _stream_ptr(stream), ctypes.byref(handle))
        _check(st, "fmm_build_tree")
        self._h = handle
        self.n_vol, self.n_bnd = n_vol, n_bnd

    def close(self):
        if getattr(self, "_h", None):
            lib().fmm_destroy_tree(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, q_vol=None, q_bnd=None, src=SET_VOL | SET_BND, tgt=SET_VOL | SET_BND,
              phi_vol=None, phi_bnd=None, mode=FWD, stream=None):
        """fmm_apply.  FWD/DK: q on `src`, phi on `tgt`; ADJ: q on `tgt`,
        phi on `src` (conjugate transpose); DLP: double layer, q on the
        boundary panels (src = SET_BND), phi on `tgt`."""
        torch = _torch()
        dev = (q_vol if q_vol is not None else q_bnd).device
        out_set = src if mode == ADJ else tgt
        if (out_set & SET_VOL) and phi_vol is None:
            phi_vol = torch.empty(self.n_vol, dtype=torch.complex128, device=dev)
        if (out_set & SET_BND) and phi_bnd is None:
            phi_bnd = torch.empty(self.n_bnd, dtype=torch.complex128, device=dev)
        if q_vol is not None:
            _dev_c128(q_vol, self.n_vol, "q_vol")
        if q_bnd is not None:
            _dev_c128(q_bnd, self.n_bnd, "q_bnd")
        st = lib().fmm_apply(self._h, src, tgt, _ptr(q_vol), _ptr(q_bnd), _ptr(phi_vol),
                             _ptr(phi_bnd), mode, _stream_ptr(stream))
        _check(st, "fmm_apply")
        return phi_vol, phi_bnd

    def precond(self, r, z=None, inner_rtol=1e-4, inner_maxit=200, inner_m=50, stream=None):
        torch = _torch()
        _dev_c128(r, self.n_vol, "r")
        if z is None:
            z = torch.empty_like(r)
        its = ctypes.c_int(0)
        st = lib().fmm_precond_apply(self._h, _ptr(r), _ptr(z), inner_rtol, inner_maxit, inner_m,
                                     ctypes.byref(its), _stream_ptr(stream))
        _check(st, "fmm_precond_apply")
        return z, its.value

    def dirichlet_rhs(self, f, u_bnd, b=None, stream=None):
        """hfmm_dirichlet_rhs: b = f + (1/h^2) (Dirichlet values at the
        boundary neighbours of each interior node)."""
        torch = _torch()
        _dev_c128(f, self.n_vol, "f")
        _dev_c128(u_bnd, self.n_bnd, "u_bnd")
        if b is None:
            b = torch.empty_like(f)
        _check(lib().hfmm_dirichlet_rhs(self._h, _ptr(f), _ptr(u_bnd), _ptr(b), _stream_ptr(stream)),
               "hfmm_dirichlet_rhs")
        return b

    def bem_solve_dirichlet(self, f, u_bnd, u=None, inner_rtol=1e-4, inner_maxit=200, inner_m=50,
                            stream=None):
        """bem_solve_dirichlet: the BEM solution with volume data f and
        Dirichlet data u_bnd.  Returns (u, inner iterations)."""
        torch = _torch()
        _dev_c128(f, self.n_vol, "f")
        _dev_c128(u_bnd, self.n_bnd, "u_bnd")
        if u is None:
            u = torch.empty_like(f)
        its = ctypes.c_int(0)
        st = lib().bem_solve_dirichlet(self._h, _ptr(f), _ptr(u_bnd), _ptr(u), inner_rtol, inner_maxit,
                                       inner_m, ctypes.byref(its), _stream_ptr(stream))
        _check(st, "bem_solve_dirichlet")
        return u, its.value

    def fdm(self, u, out=None, stream=None):
        torch = _torch()
        _dev_c128(u, self.n_vol, "u")
        if out is None:
            out = torch.empty_like(u)
        _check(lib().hfmm_fdm_apply(self._h, _ptr(u), _ptr(out), _stream_ptr(stream)),
               "hfmm_fdm_apply")
        return out

    def grad_k(self, q, g, stream=None):
        """fmm_grad_k: Re sum conj(g) (dG~/dk q) on the volume points, as a
        float64 CUDA scalar tensor."""
        torch = _torch()
        _dev_c128(q, self.n_vol, "q")
        _dev_c128(g, self.n_vol, "g")
        out = torch.empty((), dtype=torch.float64, device=q.device)
        _check(lib().fmm_grad_k(self._h, _ptr(q), _ptr(g), _ptr(out), _stream_ptr(stream)), "fmm_grad_k")
        return out

    def solve_grad_k(self, lam, x, stream=None):
        """hfmm_solve_grad_k: 2k Re sum conj(lam) x, as a float64 CUDA scalar
        tensor."""
        torch = _torch()
        _dev_c128(lam, self.n_vol, "lam")
        _dev_c128(x, self.n_vol, "x")
        out = torch.empty((), dtype=torch.float64, device=x.device)
        _check(lib().hfmm_solve_grad_k(self._h, _ptr(lam), _ptr(x), _ptr(out), _stream_ptr(stream)),
               "hfmm_solve_grad_k")
        return out

    def gmres(self, b, x=None, restart=30, rtol=1e-6, maxit=0, inner_rtol=1e-4, inner_maxit=200,
              inner_m=50, history_len=2000, raise_on_nonconvergence=False, stream=None):
        torch = _torch()
        _dev_c128(b, self.n_vol, "b")
        if x is None:
            x = torch.zeros_like(b)
        gp = hfmm_gmres_params(restart, rtol, maxit, inner_rtol, inner_maxit, inner_m)
        hist = (ctypes.c_double * history_len)()
        info = hfmm_gmres_info(0, 0, 0, 0, 0.0, 0.0, hist, history_len)
        st = lib().gmres_solve(self._h, _ptr(b), _ptr(x), ctypes.byref(gp), ctypes.byref(info),
                               _stream_ptr(stream))
        if st != HFMM_OK and (st != HFMM_ERR_NOT_CONVERGED or raise_on_nonconvergence):
            raise HfmmError(st, "gmres_solve")
        gi = GmresInfo(info.iters, info.restarts, info.inner_iters_total, info.status,
                       info.relres_est, info.relres_true, list(hist[:min(info.iters, history_len)]))
        return x, gi

    def bicgstab(self, b, x=None, rtol=1e-6, maxit=0, inner_rtol=1e-4, inner_maxit=200, inner_m=50,
                 history_len=2000, raise_on_nonconvergence=False, stream=None):
        """bicgstab_solve: right-preconditioned BiCGSTAB with the FMM
        preconditioner.  Returns (x, GmresInfo) with iters = BiCGSTAB
        iterations and restarts = preconditioner applications."""
        torch = _torch()
        _dev_c128(b, self.n_vol, "b")
        if x is None:
            x = torch.zeros_like(b)
        gp = hfmm_gmres_params(1, rtol, maxit, inner_rtol, inner_maxit, inner_m)
        hist = (ctypes.c_double * history_len)()
        info = hfmm_gmres_info(0, 0, 0, 0, 0.0, 0.0, hist, history_len)
        st = lib().bicgstab_solve(self._h, _ptr(b), _ptr(x), ctypes.byref(gp), ctypes.byref(info),
                                  _stream_ptr(stream))
        if st != HFMM_OK and (st != HFMM_ERR_NOT_CONVERGED or raise_on_nonconvergence):
            raise HfmmError(st, "bicgstab_solve")
        gi = GmresInfo(info.iters, info.restarts, info.inner_iters_total, info.status,
                       info.relres_est, info.relres_true, list(hist[:min(info.iters, history_len)]))
        return x, gi

    def set_timing(self, on=True, stages=None):
        """Per-stage CUDA-event timing; `stages` = names from STAGES (all when None)."""
        mask = 0
        if on:
            names = STAGES if stages is None else stages
            for nm in names:
                mask |= 1 << STAGES.index(nm)
        _check(lib().fmm_set_timing(self._h, mask), "fmm_set_timing")

    def stage_times(self):
        """{stage: (ms, launches, work)} accumulated since set_timing(True);
        work is point pairs for p2p and flops for m2l."""
        s = self.stats()
        return {name: (s.stage_ms[i], s.stage_launches[i], s.stage_work[i])
                for i, name in enumerate(STAGES)}

    def use_graphs(self, on: bool):
        _check(lib().fmm_use_graphs(self._h, 1 if on else 0), "fmm_use_graphs")

    def autotune(self, stream=None):
        _check(lib().fmm_autotune(self._h, _stream_ptr(stream)), "fmm_autotune")

    def set_inner_order(self, p_inner, stream=None):
        """fmm_set_inner_order: expansion order of the inner solve's
        boundary -> boundary applies (0: the tree's own p)."""
        _check(lib().fmm_set_inner_order(self._h, p_inner, _stream_ptr(stream)), "fmm_set_inner_order")

    def stats(self) -> hfmm_stats:
        s = hfmm_stats()
        _check(lib().fmm_get_stats(self._h, ctypes.byref(s)), "fmm_get_stats")
        return s


def gmres_solve_batched(trees, bs, xs=None, restart=50, rtol=1e-6, maxit=0, inner_rtol=1e-2,
                        inner_maxit=20, inner_m=20, history_len=0, stream=None):
    """Concurrent independent solves (one tree per right-hand side).  Returns
    (xs, [GmresInfo]); non-convergence is reported in the infos."""
    torch = _torch()
    n = len(trees)
    if len(bs) != n:
        raise ValueError("one right-hand side per tree")
    for t, b in zip(trees, bs):
        _dev_c128(b, t.n_vol, "b")
    if xs is None:
        xs = [torch.zeros_like(b) for b in bs]
    hs = (ctypes.c_void_p * n)(*[t._h.value for t in trees])
    bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    gp = hfmm_gmres_params(restart, rtol, maxit, inner_rtol, inner_maxit, inner_m)
    hist = [(ctypes.c_double * max(1, history_len))() for _ in range(n)]
    infos = (hfmm_gmres_info * n)(*[hfmm_gmres_info(0, 0, 0, 0, 0.0, 0.0, hist[i], history_len)
                                    for i in range(n)])
    st = lib().gmres_solve_batched(hs, bp, xp, n, ctypes.byref(gp), infos, _stream_ptr(stream))
    if st not in (HFMM_OK, HFMM_ERR_NOT_CONVERGED):
        raise HfmmError(st, "gmres_solve_batched")
    out = [GmresInfo(i.iters, i.restarts, i.inner_iters_total, i.status, i.relres_est, i.relres_true,
                     list(hist[j][:min(i.iters, history_len)])) for j, i in enumerate(infos)]
    return xs, out


def order_for_k(k: float, p_min: int) -> int:
    """hfmm_order_for_k: the expansion order to build a tree with for
    wavenumber k when at least p_min is asked for."""
    st = lib().hfmm_order_for_k(float(k), int(p_min))
    if st < 1:
        raise HfmmError(st, "hfmm_order_for_k")
    return st


def _host_array(a, dtype, n, name):
    """A contiguous host numpy array of `dtype` with n entries (or None)."""
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=dtype)
    if a.shape != (n,):
        raise ValueError(f"{name}: expected {n} entries, got shape {a.shape}")
    return a


def _aptr(a):
    return None if a is None else a.ctypes.data


def partition_ranges(L: int, nranks: int, leaf_cost=None):
    """hfmm_partition_ranges: contiguous Morton leaf ranges, one per rank,
    balanced by leaf_cost (8^L entries in Morton order, or None for equal
    costs).  Returns leaf_begin (nranks + 1 int64)."""
    nleaf = 1 << (3 * int(L))
    cost = _host_array(leaf_cost, np.float64, nleaf, "leaf_cost")
    out = np.zeros(int(nranks) + 1, dtype=np.int64)
    _check(lib().hfmm_partition_ranges(int(L), _aptr(cost), int(nranks), out.ctypes.data),
           "hfmm_partition_ranges")
    return out


def partition_let(L: int, theta: float, leaf_begin, rank: int, leaf_tgt=None, leaf_src=None):
    """hfmm_partition_let: the locally essential tree of `rank` under the
    partition leaf_begin.  Returns (near_leaves, cells) with near_leaves an
    int64 array of Morton leaf codes and cells a dict level -> int64 array of
    Morton cell codes (levels 2..L)."""
    L = int(L)
    nleaf = 1 << (3 * L)
    b = np.ascontiguousarray(leaf_begin, dtype=np.int64)
    tg = _host_array(leaf_tgt, np.uint8, nleaf, "leaf_tgt")
    sr = _host_array(leaf_src, np.uint8, nleaf, "leaf_src")
    n_near = ctypes.c_int64(0)
    cnt = np.zeros(L + 1, dtype=np.int64)
    f = lib().hfmm_partition_let
    args = (L, float(theta), len(b) - 1, b.ctypes.data, int(rank), _aptr(tg), _aptr(sr))
    _check(f(*args, None, 0, ctypes.byref(n_near), None, 0, cnt.ctypes.data), "hfmm_partition_let")
    near = np.zeros(max(n_near.value, 1), dtype=np.int64)
    cells = np.zeros(max(int(cnt.sum()), 1), dtype=np.int64)
    _check(f(*args, near.ctypes.data, len(near), ctypes.byref(n_near), cells.ctypes.data, len(cells),
             cnt.ctypes.data), "hfmm_partition_let")
    out, c0 = {}, 0
    for l in range(2, L + 1):
        out[l] = cells[c0:c0 + cnt[l]].copy()
        c0 += cnt[l]
    return near[:n_near.value].copy(), out


def check_noalloc_args(src_xyz, q, tgt_xyz, phi, require_cuda=True):
    """Argument checks of direct_sum_noalloc, made before anything is launched:
    both coordinate arrays contiguous float64 of shape (n, 3); q and phi
    contiguous complex128 with n_src and n_tgt entries; every tensor a CUDA
    tensor on one device (require_cuda=False skips the device checks, for
    host-side tests of the others).  Raises ValueError."""
    torch = _torch()
    for name, t in (("src_xyz", src_xyz), ("tgt_xyz", tgt_xyz)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.dim() != 2 \
                or t.shape[1] != 3 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 tensor of shape (n, 3)")
    n_src, n_tgt = src_xyz.shape[0], tgt_xyz.shape[0]
    for name, t, n in (("q", q, n_src), ("phi", phi, n_tgt)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or t.dim() != 1 \
                or t.numel() != n or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous complex128 tensor with {n} entries")
    if n_tgt > NOALLOC_MAX_TARGETS:
        raise ValueError(f"at most {NOALLOC_MAX_TARGETS} targets per call (got {n_tgt})")
    if require_cuda:
        devs = {t.device for t in (src_xyz, q, tgt_xyz, phi)}
        if len(devs) != 1 or not all(t.is_cuda for t in (src_xyz, q, tgt_xyz, phi)):
            raise ValueError("src_xyz, q, tgt_xyz and phi must be CUDA tensors on one device")
    return n_src, n_tgt


def direct_sum_noalloc(src_xyz, q, tgt_xyz, k, phi, stream=None):
    """Allocation-free direct sum (hfmm_direct_sum_noalloc) into the caller's
    complex128 tensor `phi`; all arguments are CUDA tensors on one device,
    checked before the call."""
    n_src, n_tgt = check_noalloc_args(src_xyz, q, tgt_xyz, phi)
    if not (float(k) >= 0.0):
        raise ValueError("k must be >= 0")
    torch = _torch()
    with torch.cuda.device(phi.device):
        st = lib().hfmm_direct_sum_noalloc(n_src, _ptr(src_xyz), _ptr(q), n_tgt, _ptr(tgt_xyz), float(k),
                                           _ptr(phi), _stream_ptr(stream))
    _check(st, "hfmm_direct_sum_noalloc")
    return phi


def pipe_peaks(stream=None):
    """hfmm_pipe_peaks: measured pipe rates of the current device, as a dict
    keyed by PEAKS (TFLOP/s, TFLOP/s, 1e9 XU ops/s, GB/s, TFLOP/s)."""
    out = (ctypes.c_double * len(PEAKS))()
    _check(lib().hfmm_pipe_peaks(out, _stream_ptr(stream)), "hfmm_pipe_peaks")
    return {name: out[i] for i, name in enumerate(PEAKS)}
