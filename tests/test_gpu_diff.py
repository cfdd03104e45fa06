"""GPU checks of the differentiable FMM: the adjoint apply (HFMM_ADJ), the
k-derivative apply (HFMM_DK) and the torch.autograd.Function built on them.

- dot-product test <G~x, y> = <x, G~^H y> (FP64, 1e-13) on both M2L paths
  (odd p: shared-memory tiled kernel; even p: bulk-copy pipeline)
- adjoint against the oracle's dense FMM matrix (conjugate transpose), 1e-11
- d/dk against central differences of the GPU apply and of the oracle apply
- autograd gradients of L = ||phi - phi_t||^2 against central differences
  (h = 1e-6, FP64) on the 64^3 k = 12 p = 6 workload, 1e-6 relative; the
  complex64 form against the FP64 gradient
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bem  # noqa: E402
from paper_1608_02461_gb300 import differentiable, hfmm, inputs  # noqa: E402

DEV = "cuda:0"


def cvec(n, seed):
    return torch.from_numpy(inputs.complex_normal(n, seed)).to(DEV)


def apply(tree, qv, qb, src, tgt, mode=hfmm.FWD):
    pv, pb = tree.apply(qv, qb, src=src, tgt=tgt, mode=mode)
    torch.cuda.synchronize()
    out_set = src if mode == hfmm.ADJ else tgt
    parts = []
    if out_set & 1:
        parts.append(pv.cpu().numpy())
    if out_set & 2:
        parts.append(pb.cpu().numpy())
    return np.concatenate(parts)


def side(tree, mask, seed):
    qv = cvec(tree.n_vol, seed) if mask & 1 else None
    qb = cvec(tree.n_bnd, seed + 1) if mask & 2 else None
    flat = np.concatenate(([qv.cpu().numpy()] if qv is not None else [])
                          + ([qb.cpu().numpy()] if qb is not None else []))
    return qv, qb, flat


@pytest.mark.parametrize("p", [5, 6])
def test_adjoint_dot_product(p):
    n, k = 10, 5.0
    tree = hfmm.Tree(n, k, p, 0.4, 8, "fp64")
    for src, tgt in [(1, 1), (3, 3), (1, 2), (2, 1), (3, 1), (2, 2)]:
        xv, xb, x = side(tree, src, 10 * src + tgt)
        yv, yb, y = side(tree, tgt, 100 + 10 * src + tgt)
        Gx = apply(tree, xv, xb, src, tgt)
        GHy = apply(tree, yv, yb, src, tgt, mode=hfmm.ADJ)
        lhs = np.vdot(y, Gx)
        rhs = np.vdot(GHy, x)
        assert abs(lhs - rhs) <= 1e-13 * abs(lhs), (p, src, tgt, lhs, rhs)


def test_adjoint_matches_oracle_dense():
    n, k, p = 5, 3.0, 4
    tree = hfmm.Tree(n, k, p, 0.4, 4, "fp64")
    pr = bem.Problem(n, k, p, 4, 0.4)
    N = pr.NO + pr.NG
    allm = np.ones(N, bool)
    G = np.stack([pr.fmm.apply(e, allm, allm, pr.sigma) for e in np.eye(N, dtype=np.complex128)], axis=1)
    yv, yb, y = side(tree, 3, 7)
    got = apply(tree, yv, yb, 3, 3, mode=hfmm.ADJ)
    ref = G.conj().T @ y
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-11


@pytest.mark.parametrize("p", [5, 6])
def test_dk_matches_central_differences(p):
    n, k, leaf = 8, 4.0, 8
    h = 1e-5
    tree = hfmm.Tree(n, k, p, 0.4, leaf, "fp64")
    qv, qb, q = side(tree, 3, 3)
    d = apply(tree, qv, qb, 3, 3, mode=hfmm.DK)
    tp = hfmm.Tree(n, k + h, p, 0.4, leaf, "fp64")
    tm = hfmm.Tree(n, k - h, p, 0.4, leaf, "fp64")
    fd = (apply(tp, qv, qb, 3, 3) - apply(tm, qv, qb, 3, 3)) / (2 * h)
    assert np.linalg.norm(d - fd) / np.linalg.norm(fd) < 1e-7
    # the oracle's FMM, differenced the same way
    allm = np.ones(len(q), bool)
    op = bem.Problem(n, k + h, p, leaf, 0.4)
    om = bem.Problem(n, k - h, p, leaf, 0.4)
    ofd = (op.fmm.apply(q, allm, allm, op.sigma) - om.fmm.apply(q, allm, allm, om.sigma)) / (2 * h)
    assert np.linalg.norm(d - ofd) / np.linalg.norm(ofd) < 1e-7


def _loss_and_grads(tree, q, phit, k):
    qq = q.clone().requires_grad_(True)
    kk = torch.tensor(k, dtype=torch.float64, device=DEV, requires_grad=True)
    phi = differentiable.fmm_potential(qq, kk, tree)
    L = ((phi - phit).abs() ** 2).sum()
    L.backward()
    return L.item(), qq.grad.detach(), kk.grad.item()


def test_autograd_against_finite_differences():
    w = inputs.WORKLOADS["fmm_n64_k12_p6"]
    n, k, p, leaf, th = w["n"], w["k"], w["p"], w["leaf"], w["theta"]
    tree = hfmm.Tree(n, k, p, th, leaf, "fp64")
    q = cvec(n ** 3, w["seed"])
    phit = cvec(n ** 3, w["seed"] + 100)
    L0, gq, gk = _loss_and_grads(tree, q, phit, k)
    h = 1e-6

    def loss(tr, qq):
        phi, _ = tr.apply(qq, None, src=1, tgt=1)
        return ((phi - phit).abs() ** 2).sum().item()

    for s in range(4):
        dirn = cvec(n ** 3, 500 + s)
        fd = (loss(tree, q + h * dirn) - loss(tree, q - h * dirn)) / (2 * h)
        an = torch.real(torch.vdot(gq, dirn)).item()
        assert abs(fd - an) <= 1e-6 * abs(an), (s, fd, an)
    tp = hfmm.Tree(n, k + h, p, th, leaf, "fp64")
    tm = hfmm.Tree(n, k - h, p, th, leaf, "fp64")
    fdk = (loss(tp, q) - loss(tm, q)) / (2 * h)
    assert abs(fdk - gk) <= 1e-6 * abs(gk), (fdk, gk)
    # complex64 form: same gradients to FP32 accuracy of the FMM stages
    t32 = hfmm.Tree(n, k, p, th, leaf, "fp32")
    _, gq32, gk32 = _loss_and_grads(t32, q, phit, k)
    assert (torch.linalg.vector_norm(gq32 - gq) / torch.linalg.vector_norm(gq)).item() < 1e-4
    assert abs(gk32 - gk) <= 1e-4 * abs(gk)


def test_gradient_through_the_solve():
    """x = A(k)^-1 b through the FMM-preconditioned GMRES: dL/db against a
    dense solve of the assembled 7-point matrix (independent of the FMM), and
    dL/db, dL/dk against central differences of the GPU solve."""
    from oracle import fdm
    n, k, p = 6, 3.0, 4
    kw = dict(restart=30, rtol=1e-12, inner_rtol=1e-10, inner_maxit=100, inner_m=100)
    tree = hfmm.Tree(n, k, p, 0.4, 8, "fp64")
    rng = np.random.default_rng(12)
    b = torch.from_numpy(rng.standard_normal(n ** 3) + 1j * rng.standard_normal(n ** 3)).to(DEV)
    xt = torch.from_numpy(rng.standard_normal(n ** 3) + 0j).to(DEV)
    bb = b.clone().requires_grad_(True)
    kk = torch.tensor(k, dtype=torch.float64, device=DEV, requires_grad=True)
    x = differentiable.helmholtz_solve(bb, kk, tree, **kw)
    L = ((x - xt).abs() ** 2).sum()
    L.backward()
    gb, gk = bb.grad.detach().cpu().numpy(), kk.grad.item()
    # dense check: dL/db = A^-1 (2 (x - xt)) with A real symmetric
    A = np.column_stack([fdm.fdm_apply(e, n, k) for e in np.eye(n ** 3, dtype=np.complex128)])
    xd = np.linalg.solve(A, b.cpu().numpy())
    gd = np.linalg.solve(A, 2 * (xd - xt.cpu().numpy()))
    assert np.linalg.norm(gb - gd) / np.linalg.norm(gd) < 1e-8
    # central differences along random directions, and in k
    h = 1e-6

    def loss(tr, bv):
        xv, _ = tr.gmres(bv, **kw)
        return ((xv - xt).abs() ** 2).sum().item()

    for s in range(3):
        d = torch.from_numpy(rng.standard_normal(n ** 3) + 1j * rng.standard_normal(n ** 3)).to(DEV)
        fd = (loss(tree, b + h * d) - loss(tree, b - h * d)) / (2 * h)
        an = torch.real(torch.vdot(bb.grad, d)).item()
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-9, (s, fd, an)
    # in k a larger step: the loss (about n^3) carries a rounding of about
    # 2e-16 n^3, which a difference over 2h = 2e-6 would turn into 1e-8, a
    # few 1e-6 of dL/dk here; with h = 1e-4 rounding gives 1e-10 and the
    # O(h^2) truncation about 1e-8 relative
    hk = 1e-4
    tp = hfmm.Tree(n, k + hk, p, 0.4, 8, "fp64")
    tm = hfmm.Tree(n, k - hk, p, 0.4, 8, "fp64")
    fdk = (loss(tp, b) - loss(tm, b)) / (2 * hk)
    assert abs(fdk - gk) <= 1e-6 * abs(gk), (fdk, gk)


def test_grad_k_entry_points():
    """fmm_grad_k against the GPU tangent apply summed on the host (1e-13)
    and against the oracle's FMM differenced in k (1e-7); hfmm_solve_grad_k
    against 2k Re <lam, x> on the host; both bit-identical on a second call."""
    n, k, p, leaf, h = 8, 4.0, 5, 8, 1e-5
    tree = hfmm.Tree(n, k, p, 0.4, leaf, "fp64")
    q, g = cvec(n ** 3, 21), cvec(n ** 3, 22)
    gk = tree.grad_k(q, g)
    assert gk.is_cuda and gk.dtype == torch.float64 and gk.dim() == 0
    gh = g.cpu().numpy()
    ref = np.real(np.vdot(gh, apply(tree, q, None, 1, 1, mode=hfmm.DK)))
    assert abs(gk.item() - ref) <= 1e-13 * abs(ref), (gk.item(), ref)
    assert torch.equal(gk, tree.grad_k(q, g))
    op = bem.Problem(n, k + h, p, leaf, 0.4)
    om = bem.Problem(n, k - h, p, leaf, 0.4)
    qf = np.concatenate([q.cpu().numpy(), np.zeros(op.NG, dtype=np.complex128)])
    dphi = (op.fmm.apply(qf, op.vol, op.vol, op.sigma) - om.fmm.apply(qf, om.vol, om.vol, om.sigma)) / (2 * h)
    oref = np.real(np.vdot(gh, dphi[op.vol]))
    assert abs(gk.item() - oref) <= 1e-7 * abs(oref), (gk.item(), oref)
    lam, x = cvec(n ** 3, 23), cvec(n ** 3, 24)
    sk = tree.solve_grad_k(lam, x)
    sref = 2 * k * np.real(np.vdot(lam.cpu().numpy(), x.cpu().numpy()))
    assert abs(sk.item() - sref) <= 1e-13 * abs(sref), (sk.item(), sref)
    assert torch.equal(sk, tree.solve_grad_k(lam, x))
    tree.close()
