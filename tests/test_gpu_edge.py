"""Degenerate sizes through every path: one-point and few-point systems,
k = n, one right-hand side and the maximum of eight, each operator kind,
variant and test matrix.  The float64 residual of the oracle's product is the
criterion (these systems are too small for iteration counts to mean much)."""
import numpy as np
import pytest

from oracle import randrand as O
from workloads import generators as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,k", [(1, 1), (2, 1), (5, 5), (37, 36)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("sketch", ["gaussian", "srht", "multilevel"])
def test_tiny_kernel_systems(cuda_lib, n, k, precision, sketch):
    rr = cuda_lib
    if sketch == "srht" and n == 37 and k > n // 2:
        # zero-padded SRHT just above a power of two (s = 64): rows r and
        # r ^ 32 agree on all but 5 of the 37 coordinates, and 36 of the 64
        # rows leave Omega numerically rank-deficient (the build reports a
        # non-SPD Gram); half the rows are drawn instead
        k = n // 2
    X = W.mixture_points(n, seed=131 + n)
    op = O.GaussKernelOp(X)
    mu = 1e-2
    B = W.gaussian_rhs(n, 2, 131 + n)
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, sketch, seed=131 + n,
                  precision=precision, max_rhs=2)
    x, status, infos = h.solve(dev(B), rtol=1e-8 if precision == "fp64" else 1e-6)
    assert status == rr.RR_OK
    tol = 1e-8 if precision == "fp64" else 1e-6
    assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= tol)
    h.close()


@pytest.mark.parametrize("side", [2, 3, 4])
@pytest.mark.parametrize("variant", ["C", "R"])
@pytest.mark.parametrize("sketch", ["sparse_sign", "srht", "multilevel"])
def test_tiny_basis_less_csr(cuda_lib, side, variant, sketch):
    rr = cuda_lib
    C = W.diffusion_csr(side=side, seed=140 + side, corr_len=1.0)
    op = O.CsrOp(C.rowptr, C.colidx, C.vals, C.n)
    # k = n / 2: with k close to n the test matrices are nearly singular on
    # these few points (a dense sign Omega when gamma = k; the zero-padded
    # SRHT at n = 9, whose rows r and r ^ 8 differ in one coordinate), and the
    # build's float64 Cholesky then fails or not at rounding level
    k = max(1, C.n // 2)
    b = W.gaussian_rhs(C.n, 1, 140)
    h = rr.Handle(rr.Operator.csr(dev(C.rowptr), dev(C.colidx), dev(C.vals.astype(np.float64))),
                  1e-3, k, sketch, seed=140 + side, orth="rand_cholqr", variant=variant,
                  gamma=min(8, k), gamma_sk=min(8, 4 * k))
    x, status, infos = h.solve(dev(b), rtol=1e-10)
    assert status == rr.RR_OK
    assert O.true_rel_residual(op, 1e-3, x.cpu().numpy(), b)[0] <= 1e-10
    h.close()


def test_eight_rhs_kernel_mixed(cuda_lib):
    """The largest right-hand-side count: eight columns through the tensor-core
    product, the persistent step and the power projections (mp = 8)."""
    rr = cuda_lib
    n, k, mu = 2003, 60, 1e-3
    X = W.mixture_points(n, seed=150)
    op = O.GaussKernelOp(X)
    B = W.gaussian_rhs(n, 8, 150)
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=150,
                  precision="mixed", max_rhs=8)
    x, status, infos = h.solve(dev(B), rtol=1e-6)
    assert status == rr.RR_OK and len(infos) == 8
    assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)
    # five columns in a handle sized for eight
    x5, status, infos = h.solve(dev(B[:, :5]), rtol=1e-6)
    assert status == rr.RR_OK and len(infos) == 5
    assert np.all(O.true_rel_residual(op, mu, x5.cpu().numpy(), B[:, :5]) <= 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_non_finite_right_hand_side_column_breaks_down_alone(cuda_lib, precision):
    """A NaN or an Inf in one column of b ends that column at once with
    RR_ERR_BREAKDOWN (its |b| is not finite: it must not read as converged),
    and the other column still solves to the tolerance."""
    rr = cuda_lib
    n, k, mu = 1501, 40, 1e-3
    X = W.mixture_points(n, seed=160)
    op = O.GaussKernelOp(X)
    B = W.gaussian_rhs(n, 2, 160)
    tol = 1e-8 if precision == "fp64" else 1e-6
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=160,
                  precision=precision, max_rhs=2)
    for bad in (np.nan, np.inf):
        Bb = B.copy()
        Bb[7, 0] = bad
        x, status, infos = h.solve(dev(Bb), rtol=tol)
        assert status == rr.RR_ERR_BREAKDOWN
        assert infos[0]["status"] == rr.RR_ERR_BREAKDOWN and infos[0]["inner_iters"] == 0
        assert infos[1]["status"] == rr.RR_OK
        assert O.true_rel_residual(op, mu, x[:, 1:].cpu().numpy(), B[:, 1:])[0] <= tol
    h.close()
