"""GPU parity of the multi-level test matrix X = X2 X1 (Sec. 2
eq:multilevelose): Omega against the oracle's draw (same Philox streams; the
float64 sums differ only in their order), float64 factors and solves against
the oracle build, the bf16 tensor-core kernel sketch, and the basis-less CSR
form that applies Omega as its two factors."""
import numpy as np
import pytest

from oracle import philox
from oracle import randrand as O
from workloads import generators as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("n,k,l1,g1", [(700, 60, 0, 0), (3001, 100, 250, 3), (257, 256, 300, 16)])
def test_multilevel_omega_fp64(cuda_lib, n, k, l1, g1):
    """Default and explicit sizes, ragged n, k close to n, gamma1 at its
    maximum: each entry of Omega equals the oracle's to float64 rounding
    (a sum of gamma1 products of Box-Muller numbers)."""
    rr = cuda_lib
    P = W.dense_power_spectrum(n, seed=101, power=2.0)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), 1e-3, k, "multilevel", seed=101, ml_l1=l1,
                  ml_gamma=g1)
    ref = philox.multilevel_omega(n, k, 101, l1, g1)
    got = h.export("omega").cpu().numpy()
    assert got.shape == ref.shape
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-15)


def test_multilevel_omega_bf16(cuda_lib):
    """Mixed precision: Omega is the float64 sum rounded once to bf16; equal to
    the oracle's rounding except where the two float64 sums straddle a
    rounding boundary (then one bf16 ulp)."""
    rr = cuda_lib
    n, k = 3001, 80
    X = W.mixture_points(n, seed=102)
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), 1e-3, k, "multilevel", seed=102,
                  precision="mixed")
    ref = philox.round_bf16(philox.multilevel_omega(n, k, 102))
    got = h.export("omega").cpu().numpy()
    diff = got != ref
    assert diff.mean() <= 1e-4
    assert np.all(np.abs(got - ref) <= 2.0 ** -7 * np.abs(ref) + 1e-30)


def test_multilevel_factors_and_solve_fp64(cuda_lib):
    rr = cuda_lib
    n, k, mu = 700, 60, 1e-4
    P = W.dense_power_spectrum(n, seed=W.SEED_DENSE, power=2.0)
    op = O.DenseOp(P.A)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mu, k, "multilevel", seed=103, max_rhs=2)
    bd = O.build(op, mu, k, "multilevel", seed=103)
    cond = np.linalg.cond(bd.R)
    assert rel(h.export("R").cpu().numpy(), bd.R) <= max(1e-12, 1e-15 * cond) * 100
    assert rel(h.export("G").cpu().numpy(), bd.G) <= max(1e-12, 1e-15 * cond ** 2) * 100
    tau, nE, lmax = h.scalars()
    assert tau == pytest.approx(bd.tau, rel=1e-8)
    assert nE == pytest.approx(bd.normE, rel=1e-8)
    B = W.gaussian_rhs(n, 2, 103)
    for budget in (3, 9):
        x, status, infos = h.solve(dev(B), rtol=1e-14, maxit=budget)
        xo, oinfo = O.solve(bd, B, rtol=1e-14, maxit=budget)
        assert [i["inner_iters"] for i in infos] == [i.inner_iters for i in oinfo]
        assert rel(x.cpu().numpy(), xo) <= 1e-9
    x, status, infos = h.solve(dev(B), rtol=1e-12)
    assert status == rr.RR_OK
    assert rel(x.cpu().numpy(), O.exact_solve(op, mu, B)) <= 1e-8


def test_multilevel_kernel_mixed_solve(cuda_lib):
    """bf16 multi-level Omega on the tensor-core kernel sketch, float32 PCG and
    float64 refinement: the float64 residual meets rtol, in about the
    iterations of the Gaussian test matrix of the same size."""
    rr = cuda_lib
    n, k, mu = 3001, 80, 1e-3
    X = W.mixture_points(n, seed=104)
    op = O.GaussKernelOp(X)
    B = W.gaussian_rhs(n, 4, 104)
    its = {}
    for sk in ("multilevel", "gaussian"):
        h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, sk, seed=104, precision="mixed",
                      max_rhs=4)
        x, status, infos = h.solve(dev(B), rtol=1e-6)
        assert status == rr.RR_OK
        assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)
        its[sk] = max(i["inner_iters"] for i in infos)
    assert its["multilevel"] <= 1.5 * its["gaussian"] + 5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multilevel_basis_less_solve(cuda_lib, precision):
    """CSR operator, Alg. 3 and no basis: Omega^T v = X2 (X1 v) and Omega s =
    X1^T (X2^T s) in every iteration; the float64 residual meets rtol and the
    float64 path reaches the dense Cholesky solution."""
    rr = cuda_lib
    C = W.diffusion_csr(side=40, seed=105, corr_len=4.0)
    op = O.CsrOp(C.rowptr, C.colidx, C.vals, C.n)
    vals = dev(C.vals.astype(np.float64)) if precision == "fp64" else dev(C.vals)
    mu, k = 1e-6, 32
    b = W.gaussian_rhs(C.n, 2, 105)
    h = rr.Handle(rr.Operator.csr(dev(C.rowptr), dev(C.colidx), vals), mu, k, "multilevel",
                  seed=105, orth="rand_cholqr", precision=precision, max_rhs=2)
    x, status, infos = h.solve(dev(b), rtol=1e-6, maxit=20000)
    assert status == rr.RR_OK
    assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), b) <= 1e-6)
    if precision == "fp64":
        x, status, infos = h.solve(dev(b), rtol=1e-12, maxit=20000)
        assert status == rr.RR_OK
        assert rel(x.cpu().numpy(), O.exact_solve(op, mu, b)) <= 1e-7


def test_multilevel_options(cuda_lib):
    rr = cuda_lib
    P = W.dense_power_spectrum(200, seed=106, power=2.0)
    A = rr.Operator.dense(dev(P.A))
    with pytest.raises(rr.RandRandError):          # l1 < k
        rr.Handle(A, 1e-3, 40, "multilevel", seed=106, ml_l1=30, ml_gamma=4)
    with pytest.raises(rr.RandRandError):          # gamma1 > 16
        rr.Handle(A, 1e-3, 40, "multilevel", seed=106, ml_l1=400, ml_gamma=17)
    h = rr.Handle(A, 1e-3, 40, "multilevel", seed=106, keep_sketch=True)
    h.set_mu(1e-2)                                 # several shifts from a multi-level sketch
    assert h.scalars()[0] > 0.0
