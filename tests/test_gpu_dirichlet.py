"""GPU parity for the double layer of Eq. (bem) (paper Sec. 5.2; Dirichlet
data, Eq. (ubound) and Eq. (uinter)) against the FP64 oracle, through the C
ABI: fmm_apply in mode HFMM_DLP (dipole P2M and P2P, the rest of the FMM of
Sec. 5.1.2 unchanged) on boundary, volume and all targets.

Tolerance as for the single layer: FP64 FMM 1e-11 relative L2 (the same
truncated expansions on both sides)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dirichlet  # noqa: E402
from paper_1608_02461_gb300 import hfmm, inputs  # noqa: E402

DEV = "cuda:0"


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def gpu_dlp(tree, mu, tgt):
    pv, pb = tree.apply(None, dev(mu), src=hfmm.SET_BND, tgt=tgt, mode=hfmm.DLP)
    torch.cuda.synchronize()
    out = []
    if tgt & hfmm.SET_VOL:
        out.append(pv.cpu().numpy())
    if tgt & hfmm.SET_BND:
        out.append(pb.cpu().numpy())
    return np.concatenate(out)


DLP_CASES = [
    # n, k, p, leaf, theta
    (8, 4.0, 5, 8, 0.4),
    (10, 9.0, 6, 16, 0.35),
    (9, 25.0, 4, 8, 0.4),   # high k w at the coarse levels
]


@pytest.mark.parametrize("case", DLP_CASES)
def test_double_layer_fp64_matches_oracle_fmm(case):
    n, k, p, leaf, theta = case
    tree = hfmm.Tree(n, k, p, theta, leaf, "fp64")
    pr = dirichlet.DirichletProblem(n, k, p, leaf, theta)
    assert tree.stats().L == pr.fmm.L
    mu = inputs.complex_normal(pr.NG, 300 + n)
    mall = np.zeros(pr.NO + pr.NG, dtype=np.complex128)
    mall[pr.NO:] = mu
    for tgt in (hfmm.SET_BND, hfmm.SET_VOL, hfmm.SET_VOL | hfmm.SET_BND):
        tm = np.zeros(pr.NO + pr.NG, dtype=bool)
        if tgt & hfmm.SET_VOL:
            tm[:pr.NO] = True
        if tgt & hfmm.SET_BND:
            tm[pr.NO:] = True
        ref = dirichlet.double_layer_fmm(pr.fmm, mall, pr.normals, pr.bnd, tm)[tm]
        got = gpu_dlp(tree, mu, tgt)
        assert rel(got, ref) < 1e-11, (case, tgt, rel(got, ref))
    tree.close()
