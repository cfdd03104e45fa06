"""The allocation-free direct sum (hfmm_direct_sum_noalloc), for callers that
cannot allocate device memory, called through the C ABI twice in a row and
checked against the FMM apply of the existing entry points on the same
points (tolerance 1e-7 relative L2, as for explicit points elsewhere).  The
file name sorts last so that a run stopping at the first failure has run
every other test first."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1608_02461_gb300 import hfmm, inputs  # noqa: E402

DEV = "cuda:0"


def test_noalloc_direct_sum_matches_fmm_apply_twice():
    N = 1500
    pts = torch.from_numpy(inputs.uniform_points(N, 61)).to(DEV)
    q = torch.from_numpy(inputs.complex_normal(N, 62)).to(DEV)
    k = 7.0
    tree = hfmm.Tree(0, k, 12, 0.4, 8, "fp64", vol_xyz=pts)
    ref, _ = tree.apply(q, None, src=hfmm.SET_VOL, tgt=hfmm.SET_VOL)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    outs = []
    for _ in range(2):
        phi = torch.full((N,), complex(np.nan, np.nan), dtype=torch.complex128, device=DEV)
        hfmm.direct_sum_noalloc(pts, q, pts, k, phi)
        torch.cuda.synchronize()
        outs.append(phi.cpu().numpy())
    for got in outs:
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-7
    assert np.array_equal(outs[0], outs[1])
    tree.close()


def test_noalloc_rejects_sizes_beyond_scratch():
    L = hfmm.lib()
    n = hfmm.NOALLOC_MAX_TARGETS + 1
    st = L.hfmm_direct_sum_noalloc(1, ctypes.c_void_p(16), ctypes.c_void_p(16), n,
                                   ctypes.c_void_p(16), 1.0, ctypes.c_void_p(16), None)
    assert st == hfmm.HFMM_ERR_INVALID_ARG
