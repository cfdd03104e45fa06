"""The tiled form of the FP32 lattice near field (4 x 4 target-source tiles
over x-runs of lattice nodes, switch HFMM_P2P_TILE=1) against the untiled
form, for every pass, in forward and adjoint mode, on trees whose leaves are
4 x 4 x 4 blocks of nodes (all tiles take the seven-read path) and on ragged
ones (rows of 3 or 5 nodes: the per-pair path), and one preconditioned solve.
Both forms sum the same FP32 products in a different order."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1608_02461_gb300 import hfmm, inputs  # noqa: E402

DEV = "cuda:0"


def _tree_with_env(env, *args):
    import os
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return hfmm.Tree(*args)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _apply(tree, qv, qb, src, tgt, mode=hfmm.FWD):
    tv = torch.from_numpy(qv).to(DEV) if src & 1 or mode == hfmm.ADJ else None
    tb = torch.from_numpy(qb).to(DEV) if src & 2 or mode == hfmm.ADJ else None
    pv, pb = tree.apply(tv, tb, src=src, tgt=tgt, mode=mode)
    torch.cuda.synchronize()
    out_set = src if mode == hfmm.ADJ else tgt
    out = []
    if out_set & 1:
        out.append(pv.cpu().numpy())
    if out_set & 2:
        out.append(pb.cpu().numpy())
    return np.concatenate(out)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("case", [(32, 8.0, 6, 64, 0.4),    # leaves 4 x 4 x 4 (L = 3)
                                  (64, 16.0, 6, 64, 0.4),   # the benchmark's tree (L = 4)
                                  (24, 6.0, 4, 64, 0.4),    # rows of 3 (L = 3)
                                  (20, 5.0, 5, 8, 0.35)])   # rows of 2 and 3 (L = 4)
def test_tiled_near_field_matches_untiled(case):
    n, k, p, leaf, th = case
    base = hfmm.Tree(n, k, p, th, leaf, "fp32")
    tile = _tree_with_env({"HFMM_P2P_TILE": "1"}, n, k, p, th, leaf, "fp32")
    qv = inputs.complex_normal(n ** 3, 61)
    qb = inputs.complex_normal(6 * n * n, 62)
    for src, tgt in [(3, 3), (1, 2), (2, 2), (3, 1)]:
        a = _apply(tile, qv, qb, src, tgt)
        b = _apply(base, qv, qb, src, tgt)
        assert rel(a, b) < 2e-6, (case, src, tgt, rel(a, b))
    a = _apply(tile, qv, qb, 3, 3, mode=hfmm.ADJ)
    b = _apply(base, qv, qb, 3, 3, mode=hfmm.ADJ)
    assert rel(a, b) < 2e-6
    base.close()
    tile.close()


def test_tiled_near_field_solve():
    name = "helmholtz_n64_k16_p6"
    w = inputs.WORKLOADS[name]
    b = torch.from_numpy(inputs.workload_rhs(name)).to(DEV)
    base = hfmm.Tree(w["n"], w["k"], w["p"], w["theta"], w["leaf"], "fp32")
    tile = _tree_with_env({"HFMM_P2P_TILE": "1"}, w["n"], w["k"], w["p"], w["theta"], w["leaf"], "fp32")
    kw = dict(restart=w["restart"], rtol=1e-6, inner_rtol=1e-2, inner_maxit=20, inner_m=20)
    _, i0 = base.gmres(b, **kw)
    _, i1 = tile.gmres(b, **kw)
    assert i0.status == 0 and i1.status == 0 and abs(i0.iters - i1.iters) <= 1
    base.close()
    tile.close()
