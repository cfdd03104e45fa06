"""The smallest point of the fixed-kh sweep (n = 15, k = 5, p = 8, inner
boundary solve to 1e-4): the GPU FP64 solve against the oracle's recorded
solve (tests/golden/), iterations within one; the FP32 form alike."""
import json
import os

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1608_02461_gb300 import hfmm, inputs  # noqa: E402

DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_sweep_point_matches_recorded_oracle_solve():
    path = os.path.join(GOLDEN, "oracle_helmholtz_n15_k5_p8.json")
    if not os.path.exists(path):
        pytest.skip("recorded oracle solve not present")
    g = json.load(open(path))
    w = inputs.WORKLOADS[g["workload"]]
    b = torch.from_numpy(inputs.workload_rhs(g["workload"])).to(DEV)
    kw = dict(restart=g["restart"], rtol=g["rtol"], inner_rtol=g["inner_rtol"], inner_maxit=g["inner_maxit"],
              inner_m=g["inner_m"])
    for prec in ("fp64", "fp32"):
        t = hfmm.Tree(w["n"], w["k"], w["p"], w["theta"], w["leaf"], prec)
        _, info = t.gmres(b, **kw)
        assert info.status == 0 and info.relres_true < g["rtol"]
        assert abs(info.iters - g["iters"]) <= 1, (prec, info.iters, g["iters"])
