"""Writes tests/golden/oracle_<workload>.json (GMRES) or
tests/golden/oracle_bicgstab_<workload>.json (--method bicgstab): the FP64 CPU
oracle's own preconditioned solve of a workload (iteration counts, residual
history, true residual).  Calls only oracle/ and the seeded input module;
nothing here comes from the CUDA path.

Usage: python tests/golden/make_golden.py helmholtz_n64_k16_p6 [--inner-rtol 1e-2 --inner-maxit 20]
       [--method gmres|bicgstab]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import bem, bicgstab, fdm, gmres  # noqa: E402
from paper_1608_02461_gb300 import inputs  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--inner-rtol", type=float, default=1e-2)
    ap.add_argument("--inner-maxit", type=int, default=20)
    ap.add_argument("--method", choices=("gmres", "bicgstab"), default="gmres")
    a = ap.parse_args()
    w = inputs.WORKLOADS[a.workload]
    n, k = w["n"], w["k"]
    t0 = time.time()
    pr = bem.Problem(n, k, w["p"], w["leaf"], w["theta"])
    b = inputs.workload_rhs(a.workload)
    inner = []
    log = open(os.path.join(HERE, f".progress_{a.workload}.log"), "w")

    def M(r):
        z, its = pr.precond(r, inner_rtol=a.inner_rtol, inner_maxit=a.inner_maxit, inner_m=a.inner_maxit)
        inner.append(its)
        log.write(f"{time.time() - t0:.0f}s apply {len(inner)} inner {its}\n")
        log.flush()
        return z

    A = lambda u: fdm.fdm_apply(u, n, k)
    if a.method == "gmres":
        x, info = gmres.fgmres(A, b, M, m=w["restart"], rtol=1e-6)
    else:
        x, info = bicgstab.bicgstab(A, b, M, rtol=1e-6, maxit=500)
        info["restarts"] = info["precond_applies"]
        info["relres_est"] = info["history"][-1] if info["history"] else 0.0
    out = {
        "method": a.method,
        "source": "oracle/ (FP64 CPU), written by tests/golden/make_golden.py",
        "workload": a.workload, **{key: w[key] for key in ("n", "k", "p", "leaf", "theta", "restart")},
        "rtol": 1e-6, "inner_rtol": a.inner_rtol, "inner_maxit": a.inner_maxit, "inner_m": a.inner_maxit,
        "iters": info["iters"], "restarts": info["restarts"], "converged": info["converged"],
        "inner_iters_total": int(sum(inner)), "inner_iters": inner,
        "relres_est": info["relres_est"], "relres_true": info["relres_true"], "history": info["history"],
        "wall_s": time.time() - t0,
    }
    name = f"oracle_{a.workload}.json" if a.method == "gmres" else f"oracle_bicgstab_{a.workload}.json"
    json.dump(out, open(os.path.join(HERE, name), "w"), indent=1)
    print(json.dumps({k2: v for k2, v in out.items() if k2 not in ("history", "inner_iters")}))


if __name__ == "__main__":
    main()
