"""GPU parity tests for Dirichlet data (paper Sec. 5.2-5.3, Eq. (ubound) and
Eq. (uinter) with boundary data).  Against the FP64 oracle, through the C ABI: the
double layer at high order, in FP32 and on an L = 2 tree whose panels lie on
the polar axis of their leaf centre; the FDM right-hand side with Dirichlet
data (hfmm_dirichlet_rhs); the BEM solution with data (bem_solve_dirichlet);
the FDM solve with data from zero and from the BEM solution."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from oracle import dirichlet, fdm  # noqa: E402
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


def test_double_layer_on_the_polar_axis_l2():
    """n + 1 = 8: panels lie on the polar axis of their leaf centre; L = 2."""
    n, k, p, leaf, theta = 7, 3.0, 4, 32, 0.4
    tree = hfmm.Tree(n, k, p, theta, leaf, "fp64")
    pr = dirichlet.DirichletProblem(n, k, p, leaf, theta)
    assert tree.stats().L == pr.fmm.L
    mu = inputs.complex_normal(pr.NG, 307)
    mall = np.zeros(pr.NO + pr.NG, dtype=np.complex128)
    mall[pr.NO:] = mu
    ref = dirichlet.double_layer_fmm(pr.fmm, mall, pr.normals, pr.bnd, pr.vol | pr.bnd)
    got = gpu_dlp(tree, mu, hfmm.SET_VOL | hfmm.SET_BND)
    assert rel(got, ref) < 1e-11
    tree.close()


def test_double_layer_high_order_matches_direct_sum():
    """p = 14: the truncated double layer reaches the O(N^2) definition."""
    n, k = 10, 5.0
    tree = hfmm.Tree(n, k, 14, 0.4, 8, "fp64")
    pr = dirichlet.DirichletProblem(n, k, 4, 8, 0.4)
    mu = inputs.complex_normal(pr.NG, 320)
    mall = np.zeros(pr.NO + pr.NG, dtype=np.complex128)
    mall[pr.NO:] = mu
    ref = dirichlet.double_layer_direct(pr.points, mall, pr.normals, pr.bnd, pr.vol | pr.bnd, k)
    got = gpu_dlp(tree, mu, hfmm.SET_VOL | hfmm.SET_BND)
    assert rel(got, ref) < 1e-7
    tree.close()


def test_double_layer_fp32_error_bounded():
    n, k, p, leaf, theta = 12, 8.0, 6, 16, 0.4
    t64 = hfmm.Tree(n, k, p, theta, leaf, "fp64")
    t32 = hfmm.Tree(n, k, p, theta, leaf, "fp32")
    mu = inputs.complex_normal(6 * n * n, 321)
    tgt = hfmm.SET_VOL | hfmm.SET_BND
    assert rel(gpu_dlp(t32, mu, tgt), gpu_dlp(t64, mu, tgt)) < 5e-5
    t64.close()
    t32.close()


def test_dirichlet_rhs_matches_oracle():
    n, k = 9, 3.0
    tree = hfmm.Tree(n, k, 4, 0.4, 8, "fp64")
    f = inputs.complex_normal(n ** 3, 330)
    ub = inputs.complex_normal(6 * n * n, 331)
    b = tree.dirichlet_rhs(dev(f), dev(ub)).cpu().numpy()
    ref = f + dirichlet.dirichlet_lift(n, ub)
    assert np.max(np.abs(b - ref)) <= 1e-12 * np.max(np.abs(ref))
    tree.close()


def test_bem_solve_dirichlet_matches_oracle():
    n, k, p, leaf, theta = 8, 4.0, 5, 8, 0.4
    pr = dirichlet.DirichletProblem(n, k, p, leaf, theta)
    f = inputs.complex_normal(pr.NO, 340)
    ub = inputs.complex_normal(pr.NG, 341)
    ref, _, its_ref = pr.bem_solve(f, ub, method="fmm", inner_rtol=1e-13, inner_maxit=300, inner_m=300)
    t64 = hfmm.Tree(n, k, p, theta, leaf, "fp64")
    u, its = t64.bem_solve_dirichlet(dev(f), dev(ub), inner_rtol=1e-13, inner_maxit=300, inner_m=300)
    # both inner solves stop at 1e-13; the boundary operator's conditioning
    # amplifies the difference (as for the preconditioner)
    assert rel(u.cpu().numpy(), ref) < 1e-10
    assert abs(its - its_ref) <= 1
    t32 = hfmm.Tree(n, k, p, theta, leaf, "fp32")
    u32, _ = t32.bem_solve_dirichlet(dev(f), dev(ub), inner_rtol=1e-6, inner_maxit=300, inner_m=300)
    # FP32 sums (5e-5 per apply) through the first-kind boundary solve
    assert rel(u32.cpu().numpy(), ref) < 1e-3
    t64.close()
    t32.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bem_solve_without_data_is_the_preconditioner(prec):
    """u_Gamma = 0 reduces the solve with data to M^-1 f, bit for bit."""
    n, k = 10, 5.0
    tree = hfmm.Tree(n, k, 5, 0.4, 8, prec)
    f = dev(inputs.complex_normal(n ** 3, 350))
    zero = torch.zeros(6 * n * n, dtype=torch.complex128, device=DEV)
    u, its_u = tree.bem_solve_dirichlet(f, zero, inner_rtol=1e-6, inner_maxit=100, inner_m=100)
    z, its_z = tree.precond(f, inner_rtol=1e-6, inner_maxit=100, inner_m=100)
    assert its_u == its_z and torch.equal(u, z)
    tree.close()


def test_fdm_solve_with_dirichlet_data():
    """A_h u = f + lift(u_Gamma) for a plane wave (f = 0): GMRES with the FMM
    preconditioner reaches the dense solution, from zero and from the BEM
    solution with the data (in no more iterations)."""
    n, k = 12, 4.0
    dvec = np.array([1.0, 2.0, 2.0]) / 3.0
    pr = dirichlet.DirichletProblem(n, k, 4, 8, 0.4)
    ub = np.exp(1j * k * pr.x_bnd @ dvec)
    f = np.zeros(pr.NO, dtype=np.complex128)
    A = np.stack([fdm.fdm_apply(e, n, k) for e in np.eye(n ** 3)], axis=1)
    ref = np.linalg.solve(A, f + dirichlet.dirichlet_lift(n, ub))
    tree = hfmm.Tree(n, k, 6, 0.4, 8, "fp64")
    b = tree.dirichlet_rhs(dev(f), dev(ub))
    x, i0 = tree.gmres(b, restart=30, rtol=1e-10, inner_rtol=1e-4, inner_maxit=100, inner_m=100)
    x0, _ = tree.bem_solve_dirichlet(dev(f), dev(ub), inner_rtol=1e-4, inner_maxit=100, inner_m=100)
    x1, i1 = tree.gmres(b, x=x0.clone(), restart=30, rtol=1e-10, inner_rtol=1e-4, inner_maxit=100, inner_m=100)
    assert i0.status == 0 and i1.status == 0
    # relative residual 1e-10 times the condition number of A (about 150 here)
    assert rel(x.cpu().numpy(), ref) < 1e-7 and rel(x1.cpu().numpy(), ref) < 1e-7
    assert i1.iters <= i0.iters
    # the BEM solution alone is a first-order approximation of the plane wave
    ue = np.exp(1j * k * pr.x_vol @ dvec)
    assert rel(x0.cpu().numpy(), ue) < 0.05
    tree.close()


def test_double_layer_fp32_full_size_tensor_core_levels():
    """64^3 (L = 4): the volume-target double layer takes the tensor-core M2L
    at level 4 with dipole multipoles; FP32 against FP64 on all targets."""
    name = "helmholtz_n64_k16_p6"
    w = inputs.WORKLOADS[name]
    n = w["n"]
    t64 = hfmm.Tree(n, w["k"], w["p"], w["theta"], w["leaf"], "fp64")
    t32 = hfmm.Tree(n, w["k"], w["p"], w["theta"], w["leaf"], "fp32")
    mu = inputs.complex_normal(6 * n * n, 322)
    for tgt in (hfmm.SET_VOL, hfmm.SET_BND):
        assert rel(gpu_dlp(t32, mu, tgt), gpu_dlp(t64, mu, tgt)) < 5e-5, tgt
    t64.close()
    t32.close()
