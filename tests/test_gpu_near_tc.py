"""The volume -> volume near field on the tensor cores (FP32 form, regular
lattice trees: every leaf the same block of nodes, so the kernel block between
two leaves depends only on their offset and the near field is a sum of dense
block products): pass C (sources volume + boundary, targets volume) and the
volume -> volume apply against the lattice near-field kernel of the same tree
(HFMM_NEAR_TC=0) and against the oracle's FMM on sampled volume targets; the
tensor-core form is the one that ran (its launches in the near-field stage),
repeated applies are bit-identical, and the 64^3 solve takes the same
iterations."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bem  # noqa: E402
from paper_1608_02461_gb300 import hfmm, inputs  # noqa: E402

DEV = "cuda:0"


def tree(w, near_tc=True):
    old = os.environ.get("HFMM_NEAR_TC")
    os.environ["HFMM_NEAR_TC"] = "1" if near_tc else "0"
    try:
        return hfmm.Tree(w["n"], w["k"], w["p"], w["theta"], w["leaf"], "fp32")
    finally:
        if old is None:
            os.environ.pop("HFMM_NEAR_TC", None)
        else:
            os.environ["HFMM_NEAR_TC"] = old


def apply(t, qv, qb, src):
    t.set_timing(True, stages=["p2p"])
    pv, _ = t.apply(qv, qb if src & 2 else None, src=src, tgt=1)
    torch.cuda.synchronize()
    launches = t.stage_times()["p2p"][1]
    t.set_timing(False)
    return pv.cpu().numpy(), launches


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", ["helmholtz_n64_k16_p6", "helmholtz_n128_k32_p8"])
def test_near_tc_matches_lattice_kernel(name):
    w = inputs.WORKLOADS[name]
    n = w["n"]
    qv = torch.from_numpy(inputs.complex_normal(n ** 3, 61)).to(DEV)
    qb = torch.from_numpy(inputs.complex_normal(6 * n * n, 62)).to(DEV)
    a, b = tree(w, True), tree(w, False)
    for src in (3, 1):
        pa, la = apply(a, qv, qb, src)
        pb, lb = apply(b, qv, qb, src)
        assert la > lb  # split, products, sum and add kernels instead of one near-field launch
        assert rel(pa, pb) < 1e-5, (src, rel(pa, pb))
        pa2, _ = apply(a, qv, qb, src)
        assert np.array_equal(pa, pa2)
    a.close()
    b.close()


def test_near_tc_pass_c_vs_oracle_sampled():
    name = "helmholtz_n64_k16_p6"
    w = inputs.WORKLOADS[name]
    n = w["n"]
    pr = bem.Problem(n, w["k"], w["p"], w["leaf"], w["theta"])
    rng = np.random.default_rng(63)
    idx = np.sort(rng.choice(pr.NO, size=1500, replace=False))  # volume targets
    sample = np.zeros(pr.NO + pr.NG, bool)
    sample[idx] = True
    qv = inputs.complex_normal(n ** 3, 64)
    qb = inputs.complex_normal(6 * n * n, 65)
    ref = pr.fmm.apply(np.concatenate([qv, qb]), np.ones(pr.NO + pr.NG, bool), sample, pr.sigma)[idx]
    t = tree(w, True)
    got, launches = apply(t, torch.from_numpy(qv).to(DEV), torch.from_numpy(qb).to(DEV), 3)
    assert launches > 1
    assert rel(got[idx], ref) < 1e-4, rel(got[idx], ref)
    t.close()


def test_near_tc_solve_iterations():
    name = "helmholtz_n64_k16_p6"
    w = inputs.WORKLOADS[name]
    b = torch.from_numpy(inputs.workload_rhs(name)).to(DEV)
    kw = dict(restart=w["restart"], rtol=1e-6, inner_rtol=1e-2, inner_maxit=20, inner_m=20)
    _, ia = tree(w, True).gmres(b, **kw)
    _, ib = tree(w, False).gmres(b, **kw)
    assert ia.status == 0 and ia.relres_true < 1e-6
    assert abs(ia.iters - ib.iters) <= 1, (ia.iters, ib.iters)
