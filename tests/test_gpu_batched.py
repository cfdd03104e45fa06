"""Batched form: concurrent independent solves (uneven sizes and wavenumbers)
give exactly the results of the same solves run one at a time; the M2L
autotuner changes only the summation order of the far field (rounding).
Concurrent solves run their inner solves on the stage chain (the one-kernel
boundary operator wants the whole GPU), so the one-at-a-time solves they are
compared with bit for bit use the stage chain too."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fdm  # noqa: E402
from paper_1608_02461_gb300 import hfmm, inputs  # noqa: E402

DEV = "cuda:0"
PROBLEMS = [(10, 4.0, 4), (16, 9.5, 6), (12, 6.0, 4), (14, 11.0, 6), (10, 7.5, 6), (16, 5.0, 4),
            (13, 8.0, 4)]


def _trees(prec, bnd_op=True):
    old = os.environ.get("HFMM_BND_OP")
    os.environ["HFMM_BND_OP"] = "1" if bnd_op else "0"
    try:
        return [hfmm.Tree(n, k, p, 0.4, 32, prec) for n, k, p in PROBLEMS]
    finally:
        if old is None:
            os.environ.pop("HFMM_BND_OP", None)
        else:
            os.environ["HFMM_BND_OP"] = old


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batched_equals_sequential(prec):
    bs = [torch.from_numpy(inputs.rhs("uniform_real", n, 1000 + i)).to(DEV)
          for i, (n, _, _) in enumerate(PROBLEMS)]
    tb = _trees(prec)
    xs, infos = hfmm.gmres_solve_batched(tb, bs, restart=30, inner_rtol=1e-2, inner_maxit=20, inner_m=20)
    torch.cuda.synchronize()
    ts = _trees(prec, bnd_op=False)
    for i, (t, b) in enumerate(zip(ts, bs)):
        x, info = t.gmres(b, restart=30, inner_rtol=1e-2, inner_maxit=20, inner_m=20)
        assert info.iters == infos[i].iters and info.inner_iters_total == infos[i].inner_iters_total
        assert torch.equal(x, xs[i])
        n, k, _ = PROBLEMS[i]
        bh = b.cpu().numpy()
        res = np.linalg.norm(bh - fdm.fdm_apply(xs[i].cpu().numpy(), n, k)) / np.linalg.norm(bh)
        assert infos[i].status == 0 and res < 1e-6


def test_batched_rejects_repeated_handles():
    t = hfmm.Tree(8, 4.0, 4, 0.4, 8, "fp64")
    b = torch.from_numpy(inputs.rhs("uniform_real", 8, 1)).to(DEV)
    with pytest.raises(hfmm.HfmmError):
        hfmm.gmres_solve_batched([t, t], [b, b.clone()])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotune_keeps_results(prec):
    n = 16
    t = hfmm.Tree(n, 9.0, 6, 0.4, 32, prec)
    qv = torch.from_numpy(inputs.complex_normal(n ** 3, 3)).to(DEV)
    qb = torch.from_numpy(inputs.complex_normal(6 * n * n, 4)).to(DEV)
    before = [x.clone() for x in t.apply(qv, qb)]
    t.autotune()
    after = t.apply(qv, qb)
    torch.cuda.synchronize()
    tol = 1e-13 if prec == "fp64" else 1e-6
    for a, b in zip(before, after):
        assert (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(a)).item() < tol
    again = t.apply(qv, qb)  # a tuned handle is deterministic
    for a, b in zip(after, again):
        assert torch.equal(a, b)
