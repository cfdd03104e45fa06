"""GPU parity of the tangent and adjoint modes (fmm_apply HFMM_DK, HFMM_ADJ)
against the oracle's exact tangent and stage-by-stage adjoint FMM
(oracle.tangent.apply_dk, apply_adjoint), FP64, 1e-11 relative L2."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from oracle import bem, tangent  # noqa: E402
from paper_1608_02461_gb300 import hfmm, inputs  # noqa: E402

DEV = "cuda:0"


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("case", [(8, 4.0, 5, 8, 0.4), (10, 9.0, 6, 16, 0.35), (9, 25.0, 4, 8, 0.4)])
def test_dk_fp64_matches_oracle_tangent(case):
    n, k, p, leaf, theta = case
    tree = hfmm.Tree(n, k, p, theta, leaf, "fp64")
    pr = bem.Problem(n, k, p, leaf, theta)
    h = pr.h
    ds = np.concatenate([np.full(pr.NO, tangent.self_volume_dk(h, k) / h ** 3),
                         np.full(pr.NG, tangent.self_panel_dk(h, k) / h ** 2)])
    qv = inputs.complex_normal(pr.NO, 400 + n)
    qb = inputs.complex_normal(pr.NG, 500 + n)
    for src, tgt in [(3, 3), (1, 2), (2, 2), (3, 1), (1, 1)]:
        q = np.concatenate([qv if src & 1 else np.zeros(pr.NO, complex), qb if src & 2 else np.zeros(pr.NG, complex)])
        sm = np.zeros(pr.NO + pr.NG, bool)
        tm = np.zeros(pr.NO + pr.NG, bool)
        sm[:pr.NO] = bool(src & 1)
        sm[pr.NO:] = bool(src & 2)
        tm[:pr.NO] = bool(tgt & 1)
        tm[pr.NO:] = bool(tgt & 2)
        ref = tangent.apply_dk(pr.fmm, q, sm, tm, ds)[tm]
        tv = torch.from_numpy(qv).to(DEV) if src & 1 else None
        tb = torch.from_numpy(qb).to(DEV) if src & 2 else None
        pv, pb = tree.apply(tv, tb, src=src, tgt=tgt, mode=hfmm.DK)
        torch.cuda.synchronize()
        got = np.concatenate(([pv.cpu().numpy()] if tgt & 1 else []) + ([pb.cpu().numpy()] if tgt & 2 else []))
        assert rel(got, ref) < 1e-11, (case, src, tgt, rel(got, ref))
    tree.close()


@pytest.mark.parametrize("case", [(10, 4.0, 5, 8, 0.4), (12, 9.0, 6, 16, 0.35)])
def test_adjoint_fp64_matches_oracle_adjoint(case):
    """fmm_apply HFMM_ADJ against the oracle's stage-by-stage adjoint FMM
    (oracle.tangent.apply_adjoint), FP64, 1e-11 relative L2."""
    n, k, p, leaf, theta = case
    tree = hfmm.Tree(n, k, p, theta, leaf, "fp64")
    pr = bem.Problem(n, k, p, leaf, theta)
    yv = inputs.complex_normal(pr.NO, 600 + n)
    yb = inputs.complex_normal(pr.NG, 700 + n)
    for src, tgt in [(3, 3), (1, 2), (2, 2), (3, 1), (2, 1)]:
        sm = np.zeros(pr.NO + pr.NG, bool)
        tm = np.zeros(pr.NO + pr.NG, bool)
        sm[:pr.NO] = bool(src & 1)
        sm[pr.NO:] = bool(src & 2)
        tm[:pr.NO] = bool(tgt & 1)
        tm[pr.NO:] = bool(tgt & 2)
        y = np.concatenate([yv if tgt & 1 else np.zeros(pr.NO, complex), yb if tgt & 2 else np.zeros(pr.NG, complex)])
        ref = tangent.apply_adjoint(pr.fmm, y, sm, tm, pr.sigma)[sm]
        tv = torch.from_numpy(yv).to(DEV) if tgt & 1 else None
        tb = torch.from_numpy(yb).to(DEV) if tgt & 2 else None
        pv, pb = tree.apply(tv, tb, src=src, tgt=tgt, mode=hfmm.ADJ)
        torch.cuda.synchronize()
        got = np.concatenate(([pv.cpu().numpy()] if src & 1 else []) + ([pb.cpu().numpy()] if src & 2 else []))
        assert rel(got, ref) < 1e-11, (case, src, tgt, rel(got, ref))
    tree.close()
