"""The allocation-free direct sum (hfmm_direct_sum_noalloc), for callers that
cannot allocate device memory, called through the C ABI twice in a row and
checked against the FMM apply of the existing entry points on the same
points (tolerance 1e-7 relative L2, as for explicit points elsewhere) and
against the oracle's exact O(N^2) sum (1e-12: both compute the same sum in
FP64).  The file name sorts last so that a run stopping at the first failure
has run every other test first."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fmm as ofmm  # noqa: E402
from paper_1608_02461_gb300 import hfmm, inputs  # noqa: E402

DEV = "cuda:0"


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def oracle_sum(src, q, tgt, k):
    """The oracle's direct sum with sources and targets as one point set (the
    two sets are disjoint index ranges, so no pair is excluded)."""
    pts = np.concatenate([src, tgt])
    qq = np.concatenate([q, np.zeros(len(tgt), dtype=np.complex128)])
    sm = np.zeros(len(pts), bool)
    sm[:len(src)] = True
    tm = ~sm
    return ofmm.direct_sum(pts, qq, sm, tm, k, np.zeros(len(pts)))[len(src):]


def noalloc_twice(src, q, tgt, k):
    outs = []
    for _ in range(2):
        phi = torch.full((tgt.shape[0],), complex(np.nan, np.nan), dtype=torch.complex128, device=DEV)
        hfmm.direct_sum_noalloc(src, q, tgt, k, phi)
        torch.cuda.synchronize()
        outs.append(phi.cpu().numpy())
    for got in outs:
        assert np.all(np.isfinite(got))
    assert np.array_equal(outs[0], outs[1])
    return outs[0]


def test_noalloc_direct_sum_matches_fmm_apply_twice():
    N = 1500
    pts_np = inputs.uniform_points(N, 61)
    q_np = inputs.complex_normal(N, 62)
    pts = torch.from_numpy(pts_np).to(DEV)
    q = torch.from_numpy(q_np).to(DEV)
    k = 7.0
    tree = hfmm.Tree(0, k, 12, 0.4, 8, "fp64", vol_xyz=pts)
    ref, _ = tree.apply(q, None, src=hfmm.SET_VOL, tgt=hfmm.SET_VOL)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    got = noalloc_twice(pts, q, pts, k)
    assert rel(got, ref) < 1e-7
    # the oracle's exact sum over the same set (pairs j = i excluded, no self term)
    allm = np.ones(N, bool)
    exact = ofmm.direct_sum(pts_np, q_np, allm, allm, k, np.zeros(N))
    assert rel(got, exact) < 1e-12
    tree.close()


@pytest.mark.parametrize("n_src,n_tgt", [(700, 2300), (40000, 700)])
def test_noalloc_direct_sum_separate_sets_matches_oracle(n_src, n_tgt):
    """Separate source and target sets; 40000 sources make 32 chunks of more
    than the minimum chunk length, reduced in chunk order."""
    src_np = inputs.uniform_points(n_src, 63)
    tgt_np = inputs.uniform_points(n_tgt, 64, -0.5, 1.5)
    q_np = inputs.complex_normal(n_src, 65)
    k = 11.0
    got = noalloc_twice(torch.from_numpy(src_np).to(DEV), torch.from_numpy(q_np).to(DEV),
                        torch.from_numpy(tgt_np).to(DEV), k)
    assert rel(got, oracle_sum(src_np, q_np, tgt_np, k)) < 1e-12


def test_noalloc_rejects_sizes_beyond_scratch():
    L = hfmm.lib()
    n = hfmm.NOALLOC_MAX_TARGETS + 1
    st = L.hfmm_direct_sum_noalloc(1, ctypes.c_void_p(16), ctypes.c_void_p(16), n,
                                   ctypes.c_void_p(16), 1.0, ctypes.c_void_p(16), None)
    assert st == hfmm.HFMM_ERR_INVALID_ARG
