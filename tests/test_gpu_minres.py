"""GPU parity of G-RandRAND MINRES (Sec. 3.3 eq:g_randrand, Sec. 6.3) on
indefinite shifted systems: factors and estimates against the float64 oracle
build (same Omega), iterates at fixed budgets against the oracle's restarted
MINRES, and solves against the exact solution (float64) or checked by the
float64 residual (mixed precision, Gaussian kernel)."""
import numpy as np
import pytest

from oracle import randrand as O
from workloads import generators as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def indefinite_dense(n, seed, after=20):
    P = W.dense_power_spectrum(n, seed=seed, power=2.0)
    ev = np.sort(np.linalg.eigvalsh(P.A))[::-1]
    return P.A, -0.5 * (ev[after] + ev[after + 1])   # shift between two eigenvalues


def test_g_factors_fp64(cuda_lib):
    """R, G = (R^-T Omega^T Omega R^-1)^(1/2) (Newton-Schulz on the GPU,
    eigendecomposition in the oracle), the two norm estimates and tau."""
    rr = cuda_lib
    n, k, seed = 500, 60, 101
    A, mu = indefinite_dense(n, seed)
    op = O.DenseOp(A)
    h = rr.Handle(rr.Operator.dense(dev(A)), mu, k, "gaussian", seed=seed, variant="G", q=1,
                  max_rhs=2)
    bd = O.build(op, mu, k, "gaussian", seed=seed, variant="G", q=1)
    cond = np.linalg.cond(bd.R)
    assert rel(h.export("R").cpu().numpy(), bd.R) <= max(1e-12, 1e-15 * cond) * 100
    assert rel(h.export("G").cpu().numpy(), bd.G) <= 1e-9
    tau, nE, lmax = h.scalars()
    assert nE == pytest.approx(bd.normE, rel=1e-7)
    assert lmax == pytest.approx(bd.lam_max, rel=1e-7)
    assert tau == pytest.approx(bd.tau, rel=1e-7)


@pytest.mark.parametrize("m", [1, 3])
def test_g_minres_iteration_level_fp64(cuda_lib, m):
    """After small inner budgets the GPU iterate equals the oracle's restarted
    MINRES iterate."""
    rr = cuda_lib
    n, k, seed = 400, 50, 102
    A, mu = indefinite_dense(n, seed)
    op = O.DenseOp(A)
    B = W.gaussian_rhs(n, m, seed)
    h = rr.Handle(rr.Operator.dense(dev(A)), mu, k, "gaussian", seed=seed, variant="G", q=1,
                  max_rhs=m)
    bd = O.build(op, mu, k, "gaussian", seed=seed, variant="G", q=1)
    for budget in (3, 8):
        x, status, infos = h.solve(dev(B), rtol=1e-14, maxit=budget)
        xo, oinfo = O.solve(bd, B, rtol=1e-14, maxit=budget)
        assert [i["inner_iters"] for i in infos] == [i.inner_iters for i in oinfo]
        assert rel(x.cpu().numpy(), xo) <= 1e-9


def test_g_minres_solve_fp64(cuda_lib):
    rr = cuda_lib
    n, k, seed = 500, 60, 103
    A, mu = indefinite_dense(n, seed)
    B = W.gaussian_rhs(n, 2, seed)
    h = rr.Handle(rr.Operator.dense(dev(A)), mu, k, "gaussian", seed=seed, variant="G", q=1,
                  max_rhs=2)
    x, status, infos = h.solve(dev(B), rtol=1e-10, maxit=20000)
    assert status == rr.RR_OK
    xs = np.linalg.solve(A + mu * np.eye(n), B)
    assert rel(x.cpu().numpy(), xs) <= 1e-6
    assert all(i["rel_residual"] <= 1e-10 for i in infos)


def test_g_minres_kernel_mixed_indefinite(cuda_lib):
    """Gaussian kernel with a negative shift inside its spectrum, bf16 sketch,
    float32 MINRES iterations and float64 refinement: the float64 residual of
    the oracle's product meets rtol."""
    rr = cuda_lib
    n, k, seed = 2000, 100, 104
    X = W.mixture_points(n, seed=seed)
    op = O.GaussKernelOp(X)
    ev = np.sort(np.linalg.eigvalsh(op.dense()))[::-1]
    mu = -0.5 * (ev[30] + ev[31])
    B = W.gaussian_rhs(n, 4, seed)
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=seed, variant="G",
                  q=1, precision="mixed", max_rhs=4)
    x, status, infos = h.solve(dev(B), rtol=1e-6, maxit=20000)
    assert status == rr.RR_OK
    assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)


def test_g_options(cuda_lib):
    rr = cuda_lib
    n = 300
    A, mu = indefinite_dense(n, 105)
    Ad = rr.Operator.dense(dev(A))
    with pytest.raises(rr.RandRandError):          # C needs mu >= 0
        rr.Handle(Ad, mu, 20, "gaussian", seed=105)
    with pytest.raises(rr.RandRandError):          # G keeps an explicit basis
        rr.Handle(Ad, mu, 20, "gaussian", seed=105, variant="G", orth="rand_cholqr")
    h = rr.Handle(Ad, mu, 20, "gaussian", seed=105, variant="G")
    assert h.scalars()[0] > 0.0
