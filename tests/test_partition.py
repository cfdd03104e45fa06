"""Partition of one FMM apply across ranks (hfmm_partition_ranges,
hfmm_partition_let), on the CPU: the Morton ranges and their balance, the
locally essential tree against its definition written out on the oracle's own
near and M2L lists, the size query and argument errors, and a distributed
apply over gloo ranks (world sizes 2 and 3) that exchanges only what the plan
lists and reproduces the single-rank oracle apply, and the whole preconditioner
(passes A and C, the inner GMRES over pass B with all-reduced dots) split over
two ranks against the oracle's.  The per-rank arithmetic is
the oracle's FMM stages (Sec. 5.1.2); the library supplies the plan alone.
No GPU is involved."""
import ctypes
import os
import socket
import sys

import numpy as np
import pytest

from oracle import bem
from oracle.tree import flat, near_offsets
from paper_1608_02461_gb300 import hfmm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
THETA = 0.4


def morton(c):
    """Morton code of integer cell coordinates c (..., 3): bit 3i + a is bit i
    of coordinate a (x, y, z)."""
    c = np.asarray(c, dtype=np.int64)
    m = np.zeros(c.shape[:-1], dtype=np.int64)
    for i in range(10):
        for a in range(3):
            m |= ((c[..., a] >> i) & 1) << (3 * i + a)
    return m


def demorton(m):
    m = np.asarray(m, dtype=np.int64)
    c = np.zeros(m.shape + (3,), dtype=np.int64)
    for i in range(10):
        for a in range(3):
            c[..., a] |= ((m >> (3 * i + a)) & 1) << i
    return c


def test_morton_helpers_invert():
    c = np.stack(np.meshgrid(*[np.arange(8)] * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    m = morton(c)
    assert sorted(m.tolist()) == list(range(512))
    assert np.array_equal(demorton(m), c)
    assert morton([1, 0, 0]) == 1 and morton([0, 1, 0]) == 2 and morton([0, 0, 1]) == 4


def _problem(n=20, k=4.0, p=4, leaf=8):
    return bem.Problem(n, k, p, leaf, THETA)


def _leaf_of_points(pr):
    return morton(pr.fmm.tree.leaf_c)


# ---------------------------------------------------------------- ranges

def test_ranges_uniform_and_weighted():
    b = hfmm.partition_ranges(3, 3)
    assert b.tolist() == [0, 171, 341, 512]
    assert hfmm.partition_ranges(2, 64).tolist() == list(range(65))
    assert hfmm.partition_ranges(3, 1).tolist() == [0, 512]
    # all-zero costs count as equal costs
    assert hfmm.partition_ranges(3, 3, np.zeros(512)).tolist() == [0, 171, 341, 512]
    # points per leaf: the boundary leaves hold more
    pr = _problem()
    L = pr.fmm.L
    cost = np.bincount(_leaf_of_points(pr), minlength=8 ** L).astype(np.float64)
    for R in (2, 3, 5, 8):
        b = hfmm.partition_ranges(L, R, cost)
        assert b[0] == 0 and b[-1] == 8 ** L and np.all(np.diff(b) >= 1)
        pre = np.concatenate([[0.0], np.cumsum(cost)])
        for r in range(1, R):
            # the cut lies at the leaf boundary closest to r / R of the total
            assert abs(pre[b[r]] - cost.sum() * r / R) <= cost.max() / 2 + 1e-9
        assert len(set(b.tolist())) == R + 1


def test_ranges_argument_errors():
    f = hfmm.lib().hfmm_partition_ranges
    out = np.full(4, -9, dtype=np.int64)
    for L, nr in ((1, 2), (9, 2), (2, 0), (2, 65)):
        assert f(L, None, nr, out.ctypes.data) == hfmm.HFMM_ERR_INVALID_ARG
    bad = np.ones(64)
    bad[5] = -1.0
    assert f(2, bad.ctypes.data, 3, out.ctypes.data) == hfmm.HFMM_ERR_INVALID_ARG
    bad[5] = np.nan
    assert f(2, bad.ctypes.data, 3, out.ctypes.data) == hfmm.HFMM_ERR_INVALID_ARG
    assert f(2, None, 3, None) == hfmm.HFMM_ERR_INVALID_ARG
    assert np.all(out == -9)


# ---------------------------------------------------------------- the LET

def _let_by_definition(pr, b, rank, leaf_tgt, leaf_src):
    """The locally essential tree written out on the oracle's lists: foreign
    source leaves in the near lists of the rank's target leaves; per level,
    cells paired by the oracle's M2L lists with a cell holding one of the
    rank's target leaves that hold a foreign source leaf."""
    tr = pr.fmm.tree
    L = tr.L
    s = 2 ** L
    leaves = np.arange(8 ** L)
    owner = np.searchsorted(b, leaves, side="right") - 1
    mine = owner == rank
    near = set()
    c = demorton(leaves[mine & leaf_tgt])
    for v in near_offsets(THETA):
        j = c + np.array(v)
        mj = morton(j[np.all((j >= 0) & (j < s), axis=1)])
        near.update(mj[~mine[mj] & leaf_src[mj]].tolist())
    cells = {}
    for l in range(2, L + 1):
        sh = 3 * (L - l)
        tcell = np.zeros(8 ** l, bool)
        tcell[leaves[mine & leaf_tgt] >> sh] = True
        foreign = np.zeros(8 ** l, bool)
        foreign[leaves[~mine & leaf_src] >> sh] = True
        g = np.arange(2 ** l)
        iz, iy, ix = np.meshgrid(g, g, g, indexing="ij")
        coords = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)   # by flat index
        mort_of_flat = morton(coords)
        want = set()
        for v, (ti, si) in tr.m2l_pairs(l).items():
            mt, ms = mort_of_flat[ti], mort_of_flat[si]
            sel = tcell[mt] & foreign[ms]
            want.update(ms[sel].tolist())
        cells[l] = sorted(want)
    return sorted(near), cells


@pytest.mark.parametrize("case", ["all_all", "vol_bnd", "bnd_bnd"])
def test_let_equals_its_definition(case):
    pr = _problem()
    L = pr.fmm.L
    leaf = _leaf_of_points(pr)
    src_pts = {"all_all": pr.vol | pr.bnd, "vol_bnd": pr.vol, "bnd_bnd": pr.bnd}[case]
    tgt_pts = {"all_all": pr.vol | pr.bnd, "vol_bnd": pr.bnd, "bnd_bnd": pr.bnd}[case]
    leaf_src = np.zeros(8 ** L, bool)
    leaf_src[leaf[src_pts]] = True
    leaf_tgt = np.zeros(8 ** L, bool)
    leaf_tgt[leaf[tgt_pts]] = True
    cost = np.bincount(leaf, minlength=8 ** L).astype(np.float64)
    for R in (2, 3):
        b = hfmm.partition_ranges(L, R, cost)
        for rank in range(R):
            near, cells = hfmm.partition_let(L, THETA, b, rank, leaf_tgt, leaf_src)
            dnear, dcells = _let_by_definition(pr, b, rank, leaf_tgt, leaf_src)
            assert near.tolist() == dnear
            assert set(cells) == set(dcells)
            for l in cells:
                assert cells[l].tolist() == dcells[l], (R, rank, l)
            # the exchange is smaller than an all-gather of the leaf level
            assert len(cells[L]) < 8 ** L - (b[rank + 1] - b[rank])


def test_let_size_query_and_errors():
    f = hfmm.lib().hfmm_partition_let
    L = 3
    b = hfmm.partition_ranges(L, 2)
    nn = ctypes.c_int64(-1)
    cnt = np.full(L + 1, -1, dtype=np.int64)
    assert f(L, THETA, 2, b.ctypes.data, 0, None, None, None, 0, ctypes.byref(nn), None, 0,
             cnt.ctypes.data) == 0
    near, cells = hfmm.partition_let(L, THETA, b, 0)
    assert nn.value == len(near) and cnt[0] == 0 and cnt[1] == 0
    assert [cnt[l] for l in range(2, L + 1)] == [len(cells[l]) for l in range(2, L + 1)]
    # too small, or one array without the other: an error, nothing written
    a = np.full(max(nn.value, 1), -7, dtype=np.int64)
    c = np.full(int(cnt.sum()), -7, dtype=np.int64)
    st = f(L, THETA, 2, b.ctypes.data, 0, None, None, a.ctypes.data, nn.value - 1, ctypes.byref(nn),
           c.ctypes.data, len(c), cnt.ctypes.data)
    assert st == hfmm.HFMM_ERR_INVALID_ARG and np.all(a == -7) and np.all(c == -7)
    st = f(L, THETA, 2, b.ctypes.data, 0, None, None, a.ctypes.data, len(a), ctypes.byref(nn), None, 0,
           cnt.ctypes.data)
    assert st == hfmm.HFMM_ERR_INVALID_ARG and np.all(a == -7)
    bad_ranges = ([0, 300, 200, 512], [1, 256, 512], [0, 256, 511])
    for bb in bad_ranges:
        bb = np.array(bb, dtype=np.int64)
        assert f(L, THETA, len(bb) - 1, bb.ctypes.data, 0, None, None, None, 0, ctypes.byref(nn), None, 0,
                 cnt.ctypes.data) == hfmm.HFMM_ERR_INVALID_ARG
    for th, rank in ((0.0, 0), (0.6, 0), (THETA, 2), (THETA, -1)):
        assert f(L, th, 2, b.ctypes.data, rank, None, None, None, 0, ctypes.byref(nn), None, 0,
                 cnt.ctypes.data) == hfmm.HFMM_ERR_INVALID_ARG
    # an empty range is a valid partition: that rank needs nothing
    b3 = np.array([0, 256, 256, 512], dtype=np.int64)
    near, cells = hfmm.partition_let(L, THETA, b3, 1)
    assert len(near) == 0 and all(len(v) == 0 for v in cells.values())


# ---------------------------------------------------------------- distributed apply

CASES = {"all_all": ("all", "all"), "vol_bnd": ("vol", "bnd"), "bnd_bnd": ("bnd", "bnd")}


def _distributed_apply(pr, q, src_mask, tgt_mask, b, rank, world, dist, torch):
    """One FMM apply with the sources and targets of rank `rank`'s leaves,
    receiving from the other ranks exactly what its LET lists (partial
    multipoles, halo source weights).  Returns phi on the rank's own targets
    (zero elsewhere) and the float64 words it received."""
    fmm = pr.fmm
    L = fmm.L
    leaf = _leaf_of_points(pr)
    owner = np.searchsorted(b, leaf, side="right") - 1
    leaf_src = np.zeros(8 ** L, bool)
    leaf_src[leaf[src_mask]] = True
    leaf_tgt = np.zeros(8 ** L, bool)
    leaf_tgt[leaf[tgt_mask]] = True
    lets = [hfmm.partition_let(L, THETA, b, r, leaf_tgt, leaf_src) for r in range(world)]
    leaves = np.arange(8 ** L)
    leaf_owner = np.searchsorted(b, leaves, side="right") - 1

    def holds_src(rk, l):
        """cells of level l (Morton) holding a source leaf of rank rk"""
        h = np.zeros(8 ** l, bool)
        h[leaves[(leaf_owner == rk) & leaf_src] >> (3 * (L - l))] = True
        return h

    g = {l: None for l in range(2, L + 1)}
    for l in g:
        gg = np.arange(2 ** l)
        iz, iy, ix = np.meshgrid(gg, gg, gg, indexing="ij")
        g[l] = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)

    def to_flat(cells_m, l):
        return flat(demorton(cells_m), l)

    def plan(sender, receiver):
        """what `sender` sends `receiver`: per level the cells, and the halo points"""
        near, cells = lets[receiver]
        cl = {l: cells[l][holds_src(sender, l)[cells[l]]] for l in cells}
        in_halo = np.isin(leaf, near[leaf_owner[near] == sender]) & src_mask & (owner == sender)
        return cl, np.flatnonzero(in_halo)

    own_src = src_mask & (owner == rank)
    M = {L: fmm.p2m(q, own_src)}
    for l in range(L - 1, 1, -1):
        M[l] = fmm.m2m(M[l + 1], l)
    reqs = []
    for r in range(world):
        if r == rank:
            continue
        cl, pts = plan(rank, r)
        parts = [M[l][to_flat(cl[l], l)].ravel() for l in range(2, L + 1)] + [q[pts]]
        msg = np.ascontiguousarray(np.concatenate(parts)).view(np.float64)
        reqs.append((dist.isend(torch.from_numpy(msg.copy()), dst=r), None))
    Mu = {l: M[l].copy() for l in M}
    q_used = np.where(own_src, q, 0.0)
    src_used = own_src.copy()
    words = 0
    for s in range(world):
        if s == rank:
            continue
        cl, pts = plan(s, rank)
        n_c = sum(len(cl[l]) for l in cl) * fmm.P + len(pts)
        buf = torch.zeros(2 * n_c, dtype=torch.float64)
        dist.recv(buf, src=s)
        words += buf.numel()
        z = buf.numpy().view(np.complex128)
        o = 0
        for l in range(2, L + 1):
            k = len(cl[l]) * fmm.P
            Mu[l][to_flat(cl[l], l)] += z[o:o + k].reshape(-1, fmm.P)
            o += k
        q_used[pts] = z[o:]
        src_used[pts] = True
    for rq, _ in reqs:
        rq.wait()
    own_tgt = tgt_mask & (owner == rank)
    Lc = {l: fmm.m2l(Mu[l], l) for l in range(2, L + 1)}
    for l in range(2, L):
        Lc[l + 1] = fmm.l2l(Lc[l], Lc[l + 1], l)
    phi = fmm.l2p(Lc[L], own_tgt)
    phi += fmm.p2p(q_used, src_used, own_tgt)
    phi[own_tgt] += np.where(src_used[own_tgt], pr.sigma[own_tgt] * q_used[own_tgt], 0.0)
    return phi, words


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pr = _problem()
        L = pr.fmm.L
        cost = np.bincount(_leaf_of_points(pr), minlength=8 ** L).astype(np.float64)
        b = hfmm.partition_ranges(L, world, cost)
        rng = np.random.default_rng(40 + world)
        sets = {"all": pr.vol | pr.bnd, "vol": pr.vol, "bnd": pr.bnd}
        for name, (s, t) in CASES.items():
            q = rng.standard_normal(len(pr.points)) + 1j * rng.standard_normal(len(pr.points))
            src, tgt = sets[s], sets[t]
            phi, words = _distributed_apply(pr, q, src, tgt, b, rank, world, dist, torch)
            tot = torch.from_numpy(phi.view(np.float64).copy())
            dist.all_reduce(tot)
            got = tot.numpy().view(np.complex128)
            ref = pr.fmm.apply(q, src, tgt, pr.sigma)
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            out[(rank, name)] = (float(err), int(words))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _spawn(worker, world):
    """Run worker(rank, world, port, out) on `world` gloo ranks; returns out."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    # one BLAS thread per rank: the ranks share the host's cores
    keep = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    try:
        mp.spawn(worker, args=(world, _free_port(), out), nprocs=world, join=True)
    finally:
        for v, x in keep.items():
            if x is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = x
    return dict(out)


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_apply_matches_single_rank_oracle(world):
    out = _spawn(_worker, world)
    pr = _problem()
    full_M = sum(8 ** l for l in range(2, pr.fmm.L + 1)) * pr.fmm.P
    for rank in range(world):
        for name in CASES:
            err, words = out[(rank, name)]
            assert err < 1e-12, (world, rank, name, err)
            # less than the multipoles of every cell plus every source weight
            assert 0 < words < 2 * (full_M + len(pr.points)), (rank, name, words)


# ---------------------------------------------------------------- distributed preconditioner

INNER_STEPS = 8


def _dist_dot(u, v, dist, torch):
    """sum over all ranks of vdot(u, v); each rank's vectors are zero off its own points"""
    z = np.vdot(u, v)
    t = torch.tensor([z.real, z.imag], dtype=torch.float64)
    dist.all_reduce(t)
    return complex(t[0].item(), t[1].item())


def _dist_gmres(A, b, steps, dist, torch):
    """The oracle's GMRES (readings G1-G6: zero start, modified Gram-Schmidt,
    complex Givens rotations) for one cycle of `steps` steps, on vectors held
    in pieces: every inner product and norm is a sum over the ranks
    (all-reduce), the scalars of the least-squares problem are then the same
    on every rank.  Returns x and the number of all-reduces."""
    from oracle.gmres import givens
    nred = 0

    def dot(u, v):
        nonlocal nred
        nred += 1
        return _dist_dot(u, v, dist, torch)

    beta = np.sqrt(dot(b, b).real)
    m = steps
    V = [b / beta]
    H = np.zeros((m + 1, m), dtype=np.complex128)
    cs = np.zeros(m)
    sn = np.zeros(m, dtype=np.complex128)
    g = np.zeros(m + 1, dtype=np.complex128)
    g[0] = beta
    for j in range(m):
        w = A(V[j])
        for i in range(j + 1):
            H[i, j] = dot(V[i], w)
            w = w - H[i, j] * V[i]
        hnext = np.sqrt(dot(w, w).real)
        H[j + 1, j] = hnext
        for i in range(j):
            a_, b_ = H[i, j], H[i + 1, j]
            H[i, j] = cs[i] * a_ + sn[i] * b_
            H[i + 1, j] = -np.conj(sn[i]) * a_ + cs[i] * b_
        c, s = givens(H[j, j], H[j + 1, j])
        cs[j], sn[j] = c, s
        H[j, j] = c * H[j, j] + s * H[j + 1, j]
        H[j + 1, j] = 0.0
        g[j + 1] = -np.conj(s) * g[j]
        g[j] = c * g[j]
        V.append(w / hnext)
    y = np.zeros(m, dtype=np.complex128)
    for i in range(m - 1, -1, -1):
        y[i] = (g[i] - H[i, i + 1:m] @ y[i + 1:]) / H[i, i]
    return sum(y[i] * V[i] for i in range(m)), nred


def _precond_worker(rank, world, port, out):
    """z = M^-1 r (Sec. 5.2-5.3: Pass A, the inner boundary solve, Pass C) with
    every point owned by the rank of its leaf: the three FMM passes exchange
    what the plan lists, the inner GMRES all-reduces its dots and norms."""
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pr = _problem()
        L = pr.fmm.L
        leaf = _leaf_of_points(pr)
        cost = np.bincount(leaf, minlength=8 ** L).astype(np.float64)
        b = hfmm.partition_ranges(L, world, cost)
        mine = (np.searchsorted(b, leaf, side="right") - 1) == rank
        NO, h = pr.NO, pr.h
        rng = np.random.default_rng(77)
        r = rng.standard_normal(NO) + 1j * rng.standard_normal(NO)     # every rank draws the same r
        r_loc = np.where(mine[:NO], r, 0.0)                              # and keeps its own part
        words = 0

        def apply(q, src, tgt):
            nonlocal words
            phi, wd = _distributed_apply(pr, np.where(mine, q, 0.0), src, tgt, b, rank, world, dist, torch)
            words += wd
            return phi

        qa = np.zeros(NO + pr.NG, dtype=np.complex128)
        qa[:NO] = h ** 3 * r_loc
        g = apply(qa, pr.vol, pr.bnd)[NO:]                                # Pass A

        def V(qb):                                                        # Pass B
            qq = np.zeros(NO + pr.NG, dtype=np.complex128)
            qq[NO:] = h ** 2 * qb
            return apply(qq, pr.bnd, pr.bnd)[NO:]

        q, nred = _dist_gmres(V, -g, INNER_STEPS, dist, torch)
        qa[NO:] = h ** 2 * q
        z = apply(qa, pr.vol | pr.bnd, pr.vol)[:NO]                      # Pass C
        tot = torch.from_numpy(z.view(np.float64).copy())
        dist.all_reduce(tot)
        zg = tot.numpy().view(np.complex128)
        ref, its = pr.precond(r, inner_rtol=1e-15, inner_maxit=INNER_STEPS, inner_m=INNER_STEPS)
        err = np.linalg.norm(zg - ref) / np.linalg.norm(ref)
        out[rank] = (float(err), int(its), int(nred), int(words))
    finally:
        dist.destroy_process_group()


def test_distributed_preconditioner_matches_oracle():
    out = _spawn(_precond_worker, 2)
    for rank in range(2):
        err, its, nred, words = out[rank]
        assert its == INNER_STEPS
        assert err < 1e-12, (rank, err)
        # one dot per Gram-Schmidt coefficient and one norm per step, plus the first norm
        assert nred == 1 + sum(j + 2 for j in range(INNER_STEPS))
        assert words > 0
