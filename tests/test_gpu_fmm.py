"""GPU parity: the CUDA FMM stages, preconditioner, FDM operator and GMRES
against the independent FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 FMM 1e-11 relative L2 (both sides compute the same truncated
expansion; only rounding differs).  FP32 form: errors are reported and bounded
by the FP32 arithmetic of the P2P/M2L sums (5e-5 relative L2).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bem, fdm, fmm as ofmm, gmres as ogmres  # noqa: E402
from paper_1608_02461_gb300 import hfmm, inputs  # noqa: E402

DEV = "cuda:0"


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def run_apply(tree, qv, qb, src, tgt):
    tv = torch.from_numpy(qv).to(DEV) if qv is not None else None
    tb = torch.from_numpy(qb).to(DEV) if qb is not None else None
    pv, pb = tree.apply(tv, tb, src=src, tgt=tgt)
    torch.cuda.synchronize()
    out = []
    if tgt & hfmm.SET_VOL:
        out.append(pv.cpu().numpy())
    if tgt & hfmm.SET_BND:
        out.append(pb.cpu().numpy())
    return np.concatenate(out)


def oracle_apply(pr, qv, qb, src, tgt):
    q = np.concatenate([qv if qv is not None else np.zeros(pr.NO, complex),
                        qb if qb is not None else np.zeros(pr.NG, complex)])
    sm = np.zeros(pr.NO + pr.NG, bool)
    tm = np.zeros(pr.NO + pr.NG, bool)
    if src & 1:
        sm[:pr.NO] = True
    if src & 2:
        sm[pr.NO:] = True
    if tgt & 1:
        tm[:pr.NO] = True
    if tgt & 2:
        tm[pr.NO:] = True
    phi = pr.fmm.apply(q, sm, tm, pr.sigma)
    return phi[tm]


CASES = [
    # n, k, p, leaf, theta  -- L = 3 with a ragged lattice-to-leaf map
    (16, 4.0, 4, 32, 0.4),
    (13, 9.0, 6, 16, 0.35),
    (10, 2.5, 5, 8, 0.4),
    # high k w at the coarse levels (k |t| up to ~50: upward Bessel recurrences)
    (12, 25.0, 4, 16, 0.4),
    (12, 25.0, 8, 16, 0.35),
]


@pytest.mark.parametrize("case", CASES)
def test_fmm_apply_fp64_matches_oracle(case):
    n, k, p, leaf, theta = case
    tree = hfmm.Tree(n, k, p, theta, leaf, "fp64")
    pr = bem.Problem(n, k, p, leaf, theta)
    assert tree.stats().L == pr.fmm.L
    qv = inputs.complex_normal(n ** 3, 100 + n)
    qb = inputs.complex_normal(6 * n * n, 200 + n)
    for src, tgt in [(3, 3), (1, 2), (2, 2), (3, 1), (1, 1)]:
        got = run_apply(tree, qv if src & 1 else None, qb if src & 2 else None, src, tgt)
        ref = oracle_apply(pr, qv if src & 1 else None, qb if src & 2 else None, src, tgt)
        assert rel(got, ref) < 1e-11, (case, src, tgt, rel(got, ref))
    tree.close()


def test_fmm_apply_fp32_error_bounded():
    n, k, p, leaf, theta = 16, 4.0, 4, 32, 0.4
    tree = hfmm.Tree(n, k, p, theta, leaf, "fp32")
    pr = bem.Problem(n, k, p, leaf, theta)
    qv = inputs.complex_normal(n ** 3, 7)
    qb = inputs.complex_normal(6 * n * n, 8)
    got = run_apply(tree, qv, qb, 3, 3)
    ref = oracle_apply(pr, qv, qb, 3, 3)
    err = rel(got, ref)
    print(f"fp32 rel err vs fp64 oracle: {err:.3e}")
    assert err < 5e-5


def test_fmm_high_order_matches_direct_sum():
    n, k = 9, 5.0
    tree = hfmm.Tree(n, k, 14, 0.4, 8, "fp64")
    pr = bem.Problem(n, k, 4, 8, 0.4)
    qv = inputs.complex_normal(n ** 3, 31)
    qb = inputs.complex_normal(6 * n * n, 32)
    got = run_apply(tree, qv, qb, 3, 3)
    q = np.concatenate([qv, qb])
    allm = np.ones(len(q), bool)
    ref = ofmm.direct_sum(pr.points, q, allm, allm, k, pr.sigma)
    assert rel(got, ref) < 3e-9   # truncation error of p = 14 at theta = 0.4


def test_fdm_matches_oracle():
    n, k = 12, 6.0
    tree = hfmm.Tree(n, k, 4, 0.4, 32, "fp64")
    u = inputs.complex_normal(n ** 3, 5)
    out = tree.fdm(torch.from_numpy(u).to(DEV)).cpu().numpy()
    ref = fdm.fdm_apply(u, n, k)
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_precond_matches_oracle():
    n, k, p, leaf, theta = 10, 4.0, 5, 8, 0.4
    tree = hfmm.Tree(n, k, p, theta, leaf, "fp64")
    pr = bem.Problem(n, k, p, leaf, theta)
    r = inputs.complex_normal(n ** 3, 41)
    z, its = tree.precond(torch.from_numpy(r).to(DEV), inner_rtol=1e-13, inner_maxit=300, inner_m=300)
    zr, its_ref = pr.precond(r, inner_rtol=1e-13, inner_maxit=300, inner_m=300)
    # both inner solves stop at 1e-13 relative residual; the boundary operator's
    # conditioning amplifies that difference (bounded here by 1e-10)
    assert rel(z.cpu().numpy(), zr) < 1e-10
    assert abs(its - its_ref) <= 1


def test_gmres_iterations_match_oracle():
    w = inputs.WORKLOADS["helmholtz_n16_k4_p4"]
    n, k = w["n"], w["k"]
    tree = hfmm.Tree(n, k, w["p"], w["theta"], w["leaf"], "fp64")
    b = inputs.workload_rhs("helmholtz_n16_k4_p4")
    x, info = tree.gmres(torch.from_numpy(b).to(DEV), restart=w["restart"], rtol=1e-6,
                         inner_rtol=1e-4)
    xs = x.cpu().numpy()
    res = np.linalg.norm(b - fdm.fdm_apply(xs, n, k)) / np.linalg.norm(b)
    assert info.status == 0 and res < 1e-6
    assert abs(info.relres_true - res) < 1e-9
    pr = bem.Problem(n, k, w["p"], w["leaf"], w["theta"])
    _, oi = ogmres.fgmres(lambda u: fdm.fdm_apply(u, n, k), b,
                          lambda r: pr.precond(r, inner_rtol=1e-4)[0], m=w["restart"], rtol=1e-6)
    assert abs(info.iters - oi["iters"]) <= 1, (info.iters, oi["iters"])


def test_gmres_fp32_form_converges():
    w = inputs.WORKLOADS["helmholtz_n16_k4_p4"]
    n, k = w["n"], w["k"]
    t64 = hfmm.Tree(n, k, w["p"], w["theta"], w["leaf"], "fp64")
    t32 = hfmm.Tree(n, k, w["p"], w["theta"], w["leaf"], "fp32")
    b = torch.from_numpy(inputs.workload_rhs("helmholtz_n16_k4_p4")).to(DEV)
    _, i64 = t64.gmres(b, restart=30, rtol=1e-6, inner_rtol=1e-4)
    x, i32 = t32.gmres(b, restart=30, rtol=1e-6, inner_rtol=1e-4)
    assert i32.status == 0 and i32.relres_true < 1e-6
    assert i32.iters <= int(np.ceil(1.1 * i64.iters)) + 1


def test_gmres_not_converged_status():
    n, k = 8, 4.0
    tree = hfmm.Tree(n, k, 4, 0.4, 8, "fp64")
    b = torch.from_numpy(inputs.rhs("uniform_real", n, 3)).to(DEV)
    x, info = tree.gmres(b, restart=2, rtol=1e-14, maxit=3, inner_rtol=1e-3)
    assert info.status == hfmm.HFMM_ERR_NOT_CONVERGED and info.iters == 3
    with pytest.raises(hfmm.HfmmError):
        tree.gmres(b, restart=2, rtol=1e-14, maxit=3, raise_on_nonconvergence=True)


def test_build_is_deterministic():
    n, k = 12, 7.0
    q = torch.from_numpy(inputs.complex_normal(n ** 3, 9)).to(DEV)
    outs = []
    for _ in range(2):
        t = hfmm.Tree(n, k, 5, 0.4, 16, "fp64")
        pv, _ = t.apply(q, None, src=1, tgt=1)
        outs.append(pv.cpu().numpy())
        t.close()
    assert np.array_equal(outs[0], outs[1])


def test_explicit_points_direct_sum():
    """Caller-supplied points (no lattice, no self terms): the FMM converges to
    the plain N-body sum of Sec. 5.1."""
    N = 700
    pts = inputs.uniform_points(N, 3)
    q = inputs.complex_normal(N, 4)
    k = 6.0
    t = hfmm.Tree(0, k, 12, 0.4, 8, "fp64", vol_xyz=torch.from_numpy(pts).to(DEV))
    pv, _ = t.apply(torch.from_numpy(q).to(DEV), None, src=1, tgt=1)
    got = pv.cpu().numpy()
    allm = np.ones(N, bool)
    ref = ofmm.direct_sum(pts, q, allm, allm, k, np.zeros(N))
    assert rel(got, ref) < 1e-7
    # the oracle's FMM on the same points agrees to rounding
    o = ofmm.FMM(pts, N, 8, 0.4, k, 12).apply(q, allm, allm, np.zeros(N))
    assert rel(got, o) < 1e-11


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_preconditioner_equals_host_driven(prec):
    """The CUDA-graph form of the preconditioner (device-driven inner cycle)
    reproduces the host-driven form exactly, including early convergence of
    the inner cycle (inner_rtol reached before inner_maxit)."""
    n, k = 12, 5.0
    b = torch.from_numpy(inputs.rhs("uniform_real", n, 9)).to(DEV)
    for inner_rtol, inner_maxit in [(1e-2, 20), (0.3, 30)]:
        tg = hfmm.Tree(n, k, 6, 0.4, 16, prec)
        th = hfmm.Tree(n, k, 6, 0.4, 16, prec)
        th.use_graphs(False)
        kw = dict(restart=30, rtol=1e-6, inner_rtol=inner_rtol, inner_maxit=inner_maxit, inner_m=inner_maxit)
        xg, ig = tg.gmres(b, **kw)
        xh, ih = th.gmres(b, **kw)
        assert ig.iters == ih.iters and ig.inner_iters_total == ih.inner_iters_total
        assert torch.equal(xg, xh)
        # a second solve replays the captured graph
        xg2, ig2 = tg.gmres(b, **kw)
        assert torch.equal(xg2, xh) and ig2.iters == ih.iters


def _tree_with_env(env, *args):
    """A tree built while the given environment switches are set (they are
    read when the handle is built)."""
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", [(16, 9.0, 6, 32, 0.4), (13, 25.0, 4, 16, 0.35)])
def test_lattice_tables_match_generic_paths(prec, case):
    """Lattice trees evaluate the near field through the kernel table over
    integer offsets and P2M/L2P through the per-point regular-basis table;
    both give the results of the per-pair / per-point evaluation (rounding
    only), for every pass, in both precisions, and in adjoint mode."""
    n, k, p, leaf, th = case
    fast = hfmm.Tree(n, k, p, th, leaf, prec)
    slow = _tree_with_env({"HFMM_LATTICE_P2P": "0", "HFMM_BASIS_TABLE": "0"}, n, k, p, th, leaf, prec)
    qv = inputs.complex_normal(n ** 3, 5)
    qb = inputs.complex_normal(6 * n * n, 6)
    tol = 1e-13 if prec == "fp64" else 2e-6
    for src, tgt in [(3, 3), (1, 2), (2, 2), (3, 1)]:
        a = run_apply(fast, qv if src & 1 else None, qb if src & 2 else None, src, tgt)
        b = run_apply(slow, qv if src & 1 else None, qb if src & 2 else None, src, tgt)
        assert rel(a, b) < tol, (src, tgt, rel(a, b))
    tv, tb = torch.from_numpy(qv).to(DEV), torch.from_numpy(qb).to(DEV)
    fa = fast.apply(tv, tb, src=3, tgt=3, mode=hfmm.ADJ)
    sa = slow.apply(tv, tb, src=3, tgt=3, mode=hfmm.ADJ)
    torch.cuda.synchronize()
    for x, y in zip(fa, sa):
        assert (torch.linalg.vector_norm(x - y) / torch.linalg.vector_norm(y)).item() < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_concurrent_near_field_is_bitwise_equal(prec):
    """P2P on its own stream (concurrent with the far field, summed into its
    own buffer and added by L2P; used for boundary targets) gives
    bit-identical results to P2P after L2P on one stream; eagerly and through
    the CUDA-graph solve."""
    n, k, p = 12, 7.0, 6
    a = hfmm.Tree(n, k, p, 0.4, 16, prec)
    b = _tree_with_env({"HFMM_OVERLAP_NEAR": "0"}, n, k, p, 0.4, 16, prec)
    qv = inputs.complex_normal(n ** 3, 11)
    qb = inputs.complex_normal(6 * n * n, 12)
    for src, tgt in [(3, 3), (2, 2), (1, 2), (3, 2)]:
        x = run_apply(a, qv if src & 1 else None, qb if src & 2 else None, src, tgt)
        y = run_apply(b, qv if src & 1 else None, qb if src & 2 else None, src, tgt)
        assert np.array_equal(x, y), (src, tgt)
    rhs = torch.from_numpy(inputs.rhs("uniform_real", n, 3)).to(DEV)
    kw = dict(restart=30, rtol=1e-6, inner_rtol=1e-2, inner_maxit=20, inner_m=20)
    xa, ia = a.gmres(rhs, **kw)
    xb, ib = b.gmres(rhs, **kw)
    assert ia.iters == ib.iters and torch.equal(xa, xb)


@pytest.mark.parametrize("p", [6, 8])
def test_tensor_core_m2l_matches_cuda_core(p):
    """The FP32 form's far field at levels >= 4 on the tensor cores (tcgen05,
    TF32 inputs split hi + lo, three products) against the CUDA-core M2L of
    the same form, against the FP64 form and against the oracle's FMM: all
    within the FP32 bound."""
    n, k, leaf = 32, 9.0, 8  # L = 4
    tc = hfmm.Tree(n, k, p, 0.4, leaf, "fp32")
    cc = _tree_with_env({"HFMM_M2L_TC": "0"}, n, k, p, 0.4, leaf, "fp32")
    f64 = hfmm.Tree(n, k, p, 0.4, leaf, "fp64")
    assert tc.stats().L == 4
    qv = inputs.complex_normal(n ** 3, 21)
    qb = inputs.complex_normal(6 * n * n, 22)
    for src, tgt in [(3, 1), (3, 3), (1, 1)]:
        a = run_apply(tc, qv if src & 1 else None, qb if src & 2 else None, src, tgt)
        b = run_apply(cc, qv if src & 1 else None, qb if src & 2 else None, src, tgt)
        c = run_apply(f64, qv if src & 1 else None, qb if src & 2 else None, src, tgt)
        assert rel(a, c) < 3e-5, (src, tgt, rel(a, c))
        assert rel(b, c) < 3e-5
    pr = bem.Problem(n, k, p, leaf, 0.4)
    assert pr.fmm.L == 4
    ref = oracle_apply(pr, qv, qb, 3, 3)
    got = run_apply(tc, qv, qb, 3, 3)
    assert rel(got, ref) < 3e-5, rel(got, ref)
    # repeated applies are bitwise identical (fixed summation order)
    a2 = run_apply(tc, qv, qb, 3, 3)
    assert np.array_equal(a2, run_apply(tc, qv, qb, 3, 3))
    # and the preconditioned solve converges like the CUDA-core form
    rhs = torch.from_numpy(inputs.rhs("uniform_real", n, 4)).to(DEV)
    kw = dict(restart=30, rtol=1e-6, inner_rtol=1e-2, inner_maxit=20, inner_m=20)
    _, it = tc.gmres(rhs, **kw)
    _, ic = cc.gmres(rhs, **kw)
    assert it.status == 0 and it.relres_true < 1e-6 and abs(it.iters - ic.iters) <= 1
