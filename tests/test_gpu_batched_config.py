"""The batched workload: 48 independent solves of uneven size (n from
{24, 32, 48, 64, 96}), wavenumber (k up to 32 at >= 8 points per wavelength)
and requested order (p from {4, 6}), each tree built with the order
hfmm_order_for_k gives for its k and requested p.  Every FP32 solve of the
batch (concurrent, gmres_solve_batched) reaches 1e-6 within 200 iterations,
and takes at most 1.1x the iterations of the same solve in the FP64 form
(solved one at a time)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fdm  # noqa: E402
from paper_1608_02461_gb300 import hfmm, inputs  # noqa: E402

DEV = "cuda:0"
KW = dict(restart=50, rtol=1e-6, maxit=200, inner_rtol=1e-2, inner_maxit=20, inner_m=20)


def test_batched_workload_converges_like_fp64():
    probs = inputs.batched_problems()
    assert len(probs) == 48
    orders = [hfmm.order_for_k(q["k"], q["p"]) for q in probs]
    bs = [torch.from_numpy(inputs.rhs(q["rhs"], q["n"], q["seed"])).to(DEV) for q in probs]
    t32 = [hfmm.Tree(q["n"], q["k"], p, q["theta"], q["leaf"], "fp32") for q, p in zip(probs, orders)]
    xs, infos = hfmm.gmres_solve_batched(t32, bs, **KW)
    torch.cuda.synchronize()
    for t in t32:
        t.close()
    bad = [(i, q["n"], round(q["k"], 2), orders[i], infos[i].iters) for i, q in enumerate(probs)
           if infos[i].status != 0]
    assert not bad, bad
    # the true residual of a few solves, independently of the library
    for i in (0, 9, 23, 42):
        q = probs[i]
        bh = bs[i].cpu().numpy()
        r = np.linalg.norm(bh - fdm.fdm_apply(xs[i].cpu().numpy(), q["n"], q["k"])) / np.linalg.norm(bh)
        assert r < 1e-6, (i, r)
    worse = []
    for i, (q, p) in enumerate(zip(probs, orders)):
        t = hfmm.Tree(q["n"], q["k"], p, q["theta"], q["leaf"], "fp64")
        _, i64 = t.gmres(bs[i], **KW)
        t.close()
        assert i64.status == 0, (i, i64.iters)
        if infos[i].iters > math.ceil(1.1 * i64.iters):
            worse.append((i, infos[i].iters, i64.iters))
    assert not worse, worse
