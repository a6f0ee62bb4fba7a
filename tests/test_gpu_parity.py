"""GPU parity: the CUDA library through its C ABI against the float64 oracle.

Tolerances: float64 path 1e-10 relative (iterates, factors, solutions);
float32 / bf16-mixed paths: float32 unit roundoff times the condition
numbers involved, stated per test.  Sparse-sign patterns and seeds are
integer work and compared bit for bit.
"""
import math

import numpy as np
import pytest

from oracle import philox
from oracle import randrand as O
from workloads import generators as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def dense_problem(n, seed=W.SEED_DENSE, power=2.0):
    P = W.dense_power_spectrum(n, seed=seed, power=power)
    return P, O.DenseOp(P.A)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# ---------------------------------------------------------------- Omega
@pytest.mark.parametrize("n,k", [(1, 1), (37, 5), (1000, 100), (333, 64)])
def test_gaussian_omega_fp64_matches_oracle(cuda_lib, n, k):
    rr = cuda_lib
    A = dev(np.eye(n))
    h = rr.Handle(rr.Operator.dense(A), 0.1, k, "gaussian", seed=0xABCDEF12345)
    Om = h.export("omega").cpu().numpy()
    ref = philox.gaussian_omega(n, k, 0xABCDEF12345)
    assert np.max(np.abs(Om - ref)) <= 1e-14 * max(1.0, np.abs(ref).max())


def test_gaussian_omega_bf16_matches_oracle(cuda_lib):
    rr = cuda_lib
    n, k = 3000, 96
    X = W.mixture_points(n, seed=5)
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), 1e-3, k, "gaussian", seed=99,
                  precision="mixed")
    Om = h.export("omega").cpu().numpy()
    ref = philox.round_bf16(philox.gaussian_omega(n, k, 99))
    diff = Om != ref
    # float32 Box-Muller then bf16 rounding: rare flips of one bf16 ulp, or of
    # the float32 absolute error sqrt(-2 ln u) * 2^-23 near zeros of cos / sin
    assert diff.mean() < 1e-3
    tol = np.abs(ref) * 2.0 ** -7 + 6.0 * 2.0 ** -23 / np.sqrt(k)
    assert np.all(np.abs(Om - ref) <= tol)


def test_sparse_sign_omega_bitwise(cuda_lib):
    rr = cuda_lib
    n, k = 2000, 40
    A = dev(np.eye(n))
    h = rr.Handle(rr.Operator.dense(A), 0.5, k, "sparse_sign", seed=0x52523, gamma=8)
    Om = h.export("omega").cpu().numpy()
    ref = philox.sparse_sign_omega_dense(n, k, 8, 0x52523)
    assert np.array_equal(Om, ref)


# ------------------------------------------------------- build products
@pytest.mark.parametrize("precision", ["mixed", "fp32"])
@pytest.mark.parametrize("n,k", [(3001, 120), (2500, 260), (2000, 122)])
def test_float32_basis_orthonormal_and_factorizes(cuda_lib, precision, n, k):
    """Float32 paths (the last Cholesky QR pass taken to first order in
    |I - Q1^T Q1|): the stored basis is orthonormal to float32 rounding and
    Q R reproduces Y_mu = A_mu Omega of the oracle (same Omega).  The right
    multiplications run on the tensor cores for k a multiple of 4 (k = 260:
    two 256-column output tiles and a partial last K step) and on the float32
    cores otherwise (k = 122)."""
    rr = cuda_lib
    mu = 1e-3
    X = W.mixture_points(n, seed=121)
    op = O.GaussKernelOp(X)
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=121,
                  precision=precision)
    Q = h.export("Q").cpu().numpy().astype(np.float64)
    R = h.export("R").cpu().numpy()
    assert np.linalg.norm(Q.T @ Q - np.eye(k), 2) <= 2e-5
    Om = h.export("omega").cpu().numpy().astype(np.float64)
    Ymu = op.matmat(Om) + mu * Om
    # the mixed path forms Y_mu on the tensor cores with bf16 operands
    assert rel(Q @ R, Ymu) <= (1e-2 if precision == "mixed" else 1e-5)


@pytest.mark.parametrize("n,k,variant", [(300, 30, "C"), (517, 37, "C"), (517, 37, "R"),
                                         (129, 1, "C"), (64, 64, "C")])
def test_build_factors_fp64(cuda_lib, n, k, variant):
    rr = cuda_lib
    P, op = dense_problem(n)
    mu = 1e-4
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mu, k, "gaussian", seed=11, variant=variant)
    bd = O.build(op, mu, k, "gaussian", seed=11, variant=variant)
    Q = h.export("Q").cpu().numpy()
    R = h.export("R").cpu().numpy()
    cond = np.linalg.cond(bd.R)
    # R with positive diagonal is unique: CholeskyQR2 vs Householder
    assert rel(R, bd.R) <= 1e-15 * cond * 100
    assert rel(Q, bd.Q) <= 1e-15 * cond * 100
    assert np.linalg.norm(Q.T @ Q - np.eye(k), 2) <= 1e-13
    tau, nE, lmax = h.scalars()
    if k < n:                          # k = n: E = 0, both estimates are rounding noise
        assert nE == pytest.approx(bd.normE, rel=1e-9)
    assert tau == pytest.approx(bd.tau, rel=1e-9)
    if variant == "C":
        G = h.export("G").cpu().numpy()
        assert rel(G, bd.G) <= 1e-15 * cond ** 2 * 100
        assert lmax == pytest.approx(bd.lam_max, rel=1e-9)


@pytest.mark.parametrize("variant", ["C", "R"])
def test_preconditioner_apply_fp64(cuda_lib, variant):
    rr = cuda_lib
    n, k, mu = 401, 41, 1e-3
    P, op = dense_problem(n)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mu, k, "gaussian", seed=3, variant=variant, max_rhs=3)
    bd = O.build(op, mu, k, "gaussian", seed=3, variant=variant)
    r = np.random.default_rng(0).standard_normal((n, 3))
    z = h.apply(dev(r)).cpu().numpy()
    ref = bd.apply_P(r) if variant == "C" else bd.apply_B(r)
    assert rel(z, ref) <= 1e-11
    w = h.matvec(dev(r)).cpu().numpy()
    assert rel(w, P.A @ r + mu * r) <= 1e-14


# ---------------------------------------------------------------- solves
@pytest.mark.parametrize("variant", ["C", "R"])
@pytest.mark.parametrize("n,k,m", [(300, 30, 1), (777, 61, 3), (1025, 100, 2)])
def test_solve_fp64_iteration_level(cuda_lib, variant, n, k, m):
    """Same seeds, same restarts: after a fixed budget of inner iterations the
    GPU iterate equals the oracle iterate to 1e-10 (iteration-level parity)."""
    rr = cuda_lib
    P, op = dense_problem(n)
    mu = 1e-4
    B = W.gaussian_rhs(n, m, 5)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mu, k, "gaussian", seed=5, variant=variant, max_rhs=m)
    bd = O.build(op, mu, k, "gaussian", seed=5, variant=variant)
    for budget in (3, 12):
        x, status, infos = h.solve(dev(B), rtol=1e-14, maxit=budget)
        xo, oinfo = O.solve(bd, B, rtol=1e-14, maxit=budget)
        assert status == rr.RR_ERR_MAXIT
        assert [i["inner_iters"] for i in infos] == [i.inner_iters for i in oinfo]
        assert rel(x.cpu().numpy(), xo) <= 1e-10


@pytest.mark.parametrize("variant", ["C", "R"])
def test_solve_fp64_config_dense_full_size(cuda_lib, variant):
    """n=2000, lambda_i = i^-2, mu=1e-4, k=100, CG to rtol 1e-8: the oracle-measured
    float64 residual meets rtol; a tighter parity solve matches x* = A_mu^-1 b."""
    rr = cuda_lib
    n, k, mu = 2000, 100, 1e-4
    P, op = dense_problem(n)
    b = W.gaussian_rhs(n, 1, W.SEED_DENSE)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mu, k, "gaussian", seed=W.SEED_DENSE, variant=variant)
    x, status, infos = h.solve(dev(b), rtol=1e-8)
    assert status == rr.RR_OK
    xn = x.cpu().numpy()
    assert O.true_rel_residual(op, mu, xn, b)[0] <= 1e-8
    bd = O.build(op, mu, k, "gaussian", seed=W.SEED_DENSE, variant=variant)
    xo, oinfo = O.solve(bd, b, rtol=1e-8)
    assert abs(infos[0]["inner_iters"] - oinfo[0].inner_iters) <= 3
    xs = O.exact_solve(op, mu, b)
    x2, status, _ = h.solve(dev(b), rtol=1e-13, maxit=5000)
    assert rel(x2.cpu().numpy(), xs) <= 1e-10


def test_solve_initial_guess_and_zero_rhs(cuda_lib):
    rr = cuda_lib
    n, k, mu = 300, 20, 1e-3
    P, op = dense_problem(n)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mu, k, "gaussian", seed=1, max_rhs=2)
    b = W.gaussian_rhs(n, 2, 1)
    b[:, 1] = 0.0                                   # a zero column converges at once
    xs = O.exact_solve(op, mu, b)
    x0 = xs + 1e-3 * np.random.default_rng(1).standard_normal(xs.shape)
    x, status, infos = h.solve(dev(b), rtol=1e-10, x0=dev(x0))
    assert status == rr.RR_OK
    xn = x.cpu().numpy()
    assert np.all(xn[:, 1] == 0.0)
    assert O.true_rel_residual(op, mu, xn[:, :1], b[:, :1])[0] <= 1e-10


def test_maxit_returns_last_iterate(cuda_lib):
    rr = cuda_lib
    n, k, mu = 500, 5, 1e-6
    P, op = dense_problem(n)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mu, k, "gaussian", seed=2)
    b = W.gaussian_rhs(n, 1, 2)[:, 0]
    x, status, infos = h.solve(dev(b), rtol=1e-14, maxit=4)
    assert status == rr.RR_ERR_MAXIT and infos[0]["status"] == rr.RR_ERR_MAXIT
    assert infos[0]["inner_iters"] == 4
    r = O.true_rel_residual(op, mu, x.cpu().numpy(), b)[0]
    assert r == pytest.approx(infos[0]["rel_residual"], rel=1e-8)
    # CG residuals are not monotone: compare the iterate with the oracle's
    bd = O.build(op, mu, k, "gaussian", seed=2)
    xo, _ = O.solve(bd, b, rtol=1e-14, maxit=4)
    assert rel(x.cpu().numpy(), xo) <= 1e-10


def test_invalid_solve_arguments(cuda_lib):
    rr = cuda_lib
    P, op = dense_problem(50)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), 0.1, 5, "gaussian", seed=1)
    b = torch.zeros(50, dtype=torch.float64, device="cuda")
    with pytest.raises(rr.RandRandError):
        rr.randrand_solve(h.h, b.data_ptr(), 2, 50, b.data_ptr(), 50, 0, 1e-6, 10)  # nrhs > max_rhs
    with pytest.raises(rr.RandRandError):
        rr.randrand_solve(h.h, b.data_ptr(), 1, 49, b.data_ptr(), 50, 0, 1e-6, 10)  # ld < n
    with pytest.raises(rr.RandRandError):
        rr.randrand_solve(h.h, b.data_ptr(), 1, 50, b.data_ptr(), 50, 0, -1.0, 10)


# --------------------------------------------------------- kernel operator
def test_kernel_operator_fp64_solve(cuda_lib):
    rr = cuda_lib
    n, k, mu = 700, 40, 1e-3
    X = W.mixture_points(n, seed=21)
    op = O.GaussKernelOp(X)
    B = W.gaussian_rhs(n, 2, 21)
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=21, max_rhs=2)
    w = h.matvec(dev(B)).cpu().numpy()
    assert rel(w, op.matmat(B) + mu * B) <= 1e-13
    bd = O.build(op, mu, k, "gaussian", seed=21)
    assert h.scalars()[0] == pytest.approx(bd.tau, rel=1e-8)
    x, status, infos = h.solve(dev(B), rtol=1e-12)
    assert status == rr.RR_OK
    assert rel(x.cpu().numpy(), O.exact_solve(op, mu, B)) <= 1e-9


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_kernel_operator_low_precision(cuda_lib, precision):
    """bf16 sketch + float32 iterations + float64 refinement reaches the
    float64 oracle solution; the plain float32 path reaches float32-level
    residuals."""
    rr = cuda_lib
    n, k, mu = 2500, 100, 1e-3
    X = W.mixture_points(n, seed=22)
    op = O.GaussKernelOp(X)
    B = W.gaussian_rhs(n, 4, 22)
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=22,
                  precision=precision, max_rhs=4)
    xs = O.exact_solve(op, mu, B)
    if precision == "mixed":
        x, status, infos = h.solve(dev(B), rtol=1e-6)
        assert status == rr.RR_OK
        assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)
        x, status, infos = h.solve(dev(B), rtol=1e-10)
        assert status == rr.RR_OK
        assert rel(x.cpu().numpy(), xs) <= 1e-5
    else:
        x, status, infos = h.solve(dev(B), rtol=1e-4)
        assert status == rr.RR_OK
        assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 2e-4)


def test_kernel_sketch_matches_oracle_fp32(cuda_lib):
    """Y_mu = K_mu Omega with float32 kernel tiles: basis and tau close to the oracle."""
    rr = cuda_lib
    n, k, mu = 1500, 64, 1e-3
    X = W.mixture_points(n, seed=23)
    op = O.GaussKernelOp(X)
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=23, precision="fp32")
    bd = O.build(op, mu, k, "gaussian", seed=23, omega_precision="fp32")
    R = h.export("R").cpu().numpy()
    cond = np.linalg.cond(bd.R)
    assert rel(R, bd.R) <= 1e-6 * cond * 10
    tau, nE, lmax = h.scalars()
    assert tau == pytest.approx(bd.tau, rel=1e-3)


# ------------------------------------------------------------------- CSR
@pytest.mark.parametrize("sketch", ["sparse_sign", "gaussian"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_csr_solve(cuda_lib, sketch, precision):
    rr = cuda_lib
    C = W.diffusion_csr(side=40, seed=31, corr_len=4.0)
    op = O.CsrOp(C.rowptr, C.colidx, C.vals, C.n)
    mu, k = 1e-6, 32
    b = W.gaussian_rhs(C.n, 1, 31)
    vals = dev(C.vals.astype(np.float64)) if precision == "fp64" else dev(C.vals)
    h = rr.Handle(rr.Operator.csr(dev(C.rowptr), dev(C.colidx), vals), mu, k, sketch, seed=31,
                  precision=precision)
    x, status, infos = h.solve(dev(b), rtol=1e-6, maxit=20000)
    assert status == rr.RR_OK
    assert O.true_rel_residual(op, mu, x.cpu().numpy(), b)[0] <= 1e-6
    if precision == "fp64":
        bd = O.build(op, mu, k, sketch, seed=31)
        assert h.scalars()[0] == pytest.approx(bd.tau, rel=1e-8)


@pytest.mark.parametrize("n,m", [(3001, 4), (1000, 1), (777, 3)])
def test_kernel_product_double_float_accuracy(cuda_lib, n, m):
    """The refinement residual of the mixed path evaluates (K + mu I) v in
    double-float on the float32 pipes: it must match the float64 oracle product
    to ~1e-12 relative to the row magnitudes (float32 would give ~1e-7)."""
    rr = cuda_lib
    X = W.mixture_points(n, seed=24)
    op = O.GaussKernelOp(X)
    mu = 1e-3
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, 16, "gaussian", seed=24,
                  precision="mixed", max_rhs=m)
    V = np.random.default_rng(2).standard_normal((n, m))
    w = h.matvec(dev(V)).cpu().numpy().reshape(n, m)
    ref = op.matmat(V) + mu * V
    scale = op.matmat(np.abs(V)) + mu * np.abs(V)          # sum_j |K_ij v_j|
    assert np.max(np.abs(w - ref) / scale) <= 1e-11


@pytest.mark.parametrize("n,k", [(3001, 300), (1000, 256), (777, 40), (20000, 500), (25000, 200)])
def test_tensor_core_sketch_matches_float_cores(cuda_lib, n, k):
    """The tcgen05 bf16 sketch (TMA-staged Omega^T, generated K tiles, TMEM
    accumulators) and the float32-core bf16 sketch compute the same
    Y_mu = K_bf16 Omega_bf16 + mu Omega up to float32 summation order, so the
    resulting R factors and tau agree to float32 rounding.  Above 152 row
    blocks of 128 (n = 20000, 25000) the stream-K sketch splits row blocks
    between two CTAs, whose parts meet in Y."""
    rr = cuda_lib
    X = W.mixture_points(n, seed=25)
    mu = 1e-3
    hs = [rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=25,
                    precision="mixed", kernel_impl=impl) for impl in (1, 2)]
    R1, R2 = (h.export("R").cpu().numpy() for h in hs)
    cond = np.linalg.cond(R1)
    # the two kernels evaluate each exponent in a different float32 order, so
    # a few entries round to neighbouring bf16 values (the per-row check of the
    # sketch against float64 is test_tensor_core_sketch_rows_vs_float64)
    assert rel(R2, R1) <= 5e-6 * cond
    assert hs[1].scalars()[0] == pytest.approx(hs[0].scalars()[0], rel=1e-3)
    b = W.gaussian_rhs(n, 1, 25)[:, 0]
    x, status, _ = hs[1].solve(dev(b), rtol=1e-8)
    assert status == rr.RR_OK
    assert O.true_rel_residual(O.GaussKernelOp(X), mu, x.cpu().numpy(), b)[0] <= 1e-8


@pytest.mark.parametrize("n,k", [(25000, 200), (20000, 500), (3001, 300)])
def test_tensor_core_sketch_rows_vs_float64(cuda_lib, n, k):
    """Rows of the tensor-core sketch Y_mu = Q R (exported factors) against
    float64 sums_j K_ij Omega_bf16[j, c] + mu Omega[i, c], on rows spread over
    the row blocks (above 152 blocks of 128 rows most of them are split between
    two CTAs of the stream-K sketch).  Each kernel entry is rounded to bf16
    (relative error uniform within 2^-9), so entry (i, c) may differ by about
    2^-9 / sqrt(3) * |K_i. o Omega_.c|_2; six of those, plus the float32
    accumulation and factor rounding, bound it.  A lost or doubled part of a row
    block would miss by about the part's sum, far above that."""
    rr = cuda_lib
    X = W.mixture_points(n, seed=26)
    mu = 1e-3
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=26,
                  precision="mixed", kernel_impl=2)
    Q = h.export("Q").cpu().numpy()
    R = h.export("R").cpu().numpy()
    nrb = (n + 127) // 128
    rows = sorted({min(n - 1, b * 128 + o) for b in range(0, nrb, max(1, nrb // 40))
                   for o in (0, 63, 127)})
    Yg = Q[rows] @ R
    op = O.GaussKernelOp(X)
    Kr = np.vstack([op.rows(i, i + 1) for i in rows])
    Om = philox.gaussian_omega(n, k, 26)
    Ob, Of = philox.round_bf16(Om), philox.round_f32(Om)
    Yr = Kr @ Ob + mu * Of[rows]
    spread = np.sqrt((Kr * Kr) @ (Ob * Ob))
    tol = 6.0 * 2.0 ** -9 / np.sqrt(3.0) * spread + 1e-5 * np.abs(Yr).max()
    assert np.all(np.abs(Yg - Yr) <= tol), float(np.max(np.abs(Yg - Yr) / tol))
    h.close()


@pytest.mark.parametrize("n,m", [(20000, 4), (12345, 2), (3001, 4), (777, 1), (1000, 2), (515, 8)])
def test_tensor_core_kernel_product(cuda_lib, n, m):
    """Float32 Gaussian-kernel product with the exponent arguments contracted
    on the tensor cores (augmented 3xTF32 split) against the float64 oracle,
    relative to sum_j |K_ij v_j|.  The exponent a_ij = xs_i.xs_j + cn_i + cn_j
    cancels terms of size |xs|^2 ~ 60 down to O(10); the split products carry
    ~2^-22 relative error and the tensor-core float32 accumulation a few
    ulps of 60, so |delta a| ~ 1e-5..4e-5 and K_ij is off by ln2 |delta a|:
    bound 1e-4 (float32 cores: 2e-5).  The restart residual is float64-accurate,
    so this only affects the inner iterations."""
    rr = cuda_lib
    X = W.mixture_points(n, seed=26)
    mu = 1e-3
    V = np.random.default_rng(3).standard_normal((n, m))
    if n > 5000:
        # sampled rows, including the last (ragged) row block, computed a few
        # rows at a time from the definition K_ij = exp(-|x_i - x_j|^2 / 2)
        idx = np.concatenate([np.random.default_rng(4).choice(n - 300, 192, replace=False),
                              np.arange(n - 64, n)])
        X64 = X.astype(np.float64)
        ref, scale = [], []
        for c in range(0, len(idx), 32):
            ii = idx[c:c + 32]
            K = np.exp(-((X64[ii, None, :] - X64[None, :, :]) ** 2).sum(-1) / 2)
            ref.append(K @ V + mu * V[ii])
            scale.append(np.abs(K) @ np.abs(V) + mu * np.abs(V[ii]))
        ref, scale = np.concatenate(ref), np.concatenate(scale)
    else:
        op = O.GaussKernelOp(X)
        ref = op.matmat(V) + mu * V
        scale = op.matmat(np.abs(V)) + mu * np.abs(V)
        idx = slice(None)
    # impl 3 also contracts K v on the tensor cores with K and v each split
    # into two bf16 parts (hi = RN(x), lo = RN(x - hi): relative error
    # <= 2^-16 each), so an entry's product is off by <= 2^-15 more: with the
    # exponent error (ln2 x 4e-5) still within 1e-4
    for impl in (1, 2, 3):
        h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, 16, "gaussian", seed=26,
                      precision="mixed", max_rhs=m, kernel_impl=impl)
        w = h.apply_operator(dev(V)).cpu().numpy().reshape(n, m)[idx]
        assert np.max(np.abs(w - ref) / scale) <= (2e-5 if impl == 1 else 1e-4), impl


@pytest.mark.parametrize("m", [1, 4])
def test_two_contraction_product_solve(cuda_lib, m):
    """Mixed-precision solves with K v on the tensor cores (kernel_impl 3):
    the float64 residual meets rtol and the inner iteration counts stay within
    a few of those with K v on the float32 cores (kernel_impl 2)."""
    rr = cuda_lib
    n, k, mu = 3001, 80, 1e-3
    X = W.mixture_points(n, seed=63)
    op = O.GaussKernelOp(X)
    B = W.gaussian_rhs(n, m, 63)
    its = []
    for impl in (2, 3):
        h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=63,
                      precision="mixed", max_rhs=m, kernel_impl=impl)
        for _ in range(2):     # the split scratch is rewritten by every product
            x, status, infos = h.solve(dev(B), rtol=1e-6)
            assert status == rr.RR_OK
            assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)
        its.append([i["inner_iters"] for i in infos])
        h.close()
    for a, b in zip(*its):
        assert abs(a - b) <= max(3, 0.05 * b)


def test_kernel_impl_out_of_range(cuda_lib):
    rr = cuda_lib
    X = W.mixture_points(300, seed=64)
    with pytest.raises(rr.RandRandError):
        rr.Handle(rr.Operator.gauss_kernel(dev(X)), 1e-3, 16, "gaussian", seed=64,
                  precision="mixed", kernel_impl=4)


# ------------------------------------------- persistent fused PCG step
@pytest.mark.parametrize("variant", ["C", "R"])
@pytest.mark.parametrize("m", [1, 3, 8])
def test_fused_step_matches_separate_kernels_fp64(cuda_lib, m, variant):
    """The persistent cooperative step (iter_impl 0: the fused PCG step of
    variant C; for variant R the two launches around the product) and the
    separate kernels (iter_impl 1) take the same iterations and reach the same
    iterate (their reductions group sums differently: rounding-level
    differences), and both match the oracle's iterate.  Variant R stops on
    |r| of plain CG on B, which is not monotone: near rtol 1e-13 a reordered
    sum can move a crossing (of the restart threshold or of rtol) by a step,
    and an extra restart adds a few; near 1e-13 its recursive residual can
    also stall at float64 rounding.  So variant R stops at rtol 1e-11, and
    there the counts agree within 10 % and the converged iterates to 1e-10."""
    rr = cuda_lib
    n, k, mu = 1025, 100, 1e-4
    P, op = dense_problem(n)
    B = W.gaussian_rhs(n, m, 61)
    rt = 1e-13 if variant == "C" else 1e-11
    out = []
    for impl in (0, 1):
        h = rr.Handle(rr.Operator.dense(dev(P.A)), mu, k, "gaussian", seed=61, max_rhs=m,
                      variant=variant, iter_impl=impl)
        for budget in (5, 40):
            x, status, infos = h.solve(dev(B), rtol=rt, maxit=budget)
            out.append((budget, x.cpu().numpy(), [i["inner_iters"] for i in infos]))
        h.close()
    for (b0, x0, i0), (b1, x1, i1) in zip(out[:2], out[2:]):
        if variant == "C" or b0 == 5:
            assert i0 == i1
            assert rel(x0, x1) <= 1e-12
        else:
            assert all(abs(a - b) <= max(2, 0.1 * b) for a, b in zip(i0, i1)), (i0, i1)
            assert rel(x0, x1) <= 1e-10
    bd = O.build(op, mu, k, "gaussian", seed=61, variant=variant)
    xo, _ = O.solve(bd, B, rtol=rt, maxit=40)
    assert rel(out[1][1], xo) <= 1e-10


@pytest.mark.parametrize("variant", ["C", "R"])
@pytest.mark.parametrize("m", [1, 4, 8])
def test_fused_step_kernel_operator_mixed(cuda_lib, m, variant):
    """Float32 iterations with the fused step on the Gaussian-kernel operator:
    same iteration counts as the separate kernels within a few, and the float64
    residual meets rtol."""
    rr = cuda_lib
    n, k, mu = 3001, 80, 1e-3
    X = W.mixture_points(n, seed=62)
    op = O.GaussKernelOp(X)
    B = W.gaussian_rhs(n, m, 62)
    its = []
    for impl in (0, 1):
        h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=62,
                      precision="mixed", max_rhs=m, variant=variant, iter_impl=impl)
        x, status, infos = h.solve(dev(B), rtol=1e-6)
        assert status == rr.RR_OK
        assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)
        its.append([i["inner_iters"] for i in infos])
        h.close()
    for a, b in zip(*its):
        assert abs(a - b) <= max(3, 0.05 * b)


# ------------------------------------------- test matrix with power q = 1
def test_power_q1_factors_fp64(cuda_lib):
    """eq:testmatrix with q = 1 (Omega = A X^T): Omega, R, G, tau and the
    power-iteration estimates equal the oracle's."""
    rr = cuda_lib
    n, k, mu = 700, 40, 1e-4
    P, op = dense_problem(n)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mu, k, "gaussian", seed=71, q=1, max_rhs=2)
    bd = O.build(op, mu, k, "gaussian", seed=71, q=1)
    assert rel(h.export("omega").cpu().numpy(), bd.Omega) <= 1e-13
    cond = np.linalg.cond(bd.R)
    assert rel(h.export("R").cpu().numpy(), bd.R) <= max(1e-12, 1e-15 * cond) * 100
    tau, nE, lmax = h.scalars()
    assert nE == pytest.approx(bd.normE, rel=1e-8)
    # lambda_max (hence tau) goes through G = (R_M R^-1)^T (R_M R^-1): with q = 1
    # cond(R) ~ 7e6 here, so the tolerance scales with u cond(R)
    assert tau == pytest.approx(bd.tau, rel=max(1e-8, 1e-15 * cond) * 100)
    B = W.gaussian_rhs(n, 2, 71)
    x, status, infos = h.solve(dev(B), rtol=1e-12)
    assert status == rr.RR_OK
    assert rel(x.cpu().numpy(), O.exact_solve(op, mu, B)) <= 1e-8


def test_power_q1_kernel_mixed(cuda_lib):
    """q = 1 on the Gaussian-kernel operator (bf16 sketch products): the solve
    meets rtol in the float64 residual and takes no more iterations than q = 0."""
    rr = cuda_lib
    n, k, mu = 3001, 60, 1e-3
    X = W.mixture_points(n, seed=72)
    op = O.GaussKernelOp(X)
    B = W.gaussian_rhs(n, 2, 72)
    its = {}
    for q in (0, 1):
        h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=72,
                      precision="mixed", max_rhs=2, q=q)
        x, status, infos = h.solve(dev(B), rtol=1e-6)
        assert status == rr.RR_OK
        assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)
        its[q] = max(i["inner_iters"] for i in infos)
        h.close()
    assert its[1] <= its[0]


def test_power_q_with_basis_less_unsupported(cuda_lib):
    rr = cuda_lib
    C = W.diffusion_csr(side=16, seed=73, corr_len=4.0)
    op = rr.Operator.csr(dev(C.rowptr), dev(C.colidx), dev(C.vals.astype(np.float64)))
    with pytest.raises(rr.RandRandError) as e:
        rr.Handle(op, 1e-4, 8, "sparse_sign", seed=73, orth="rand_cholqr", q=1)
    assert e.value.status == rr.RR_ERR_UNSUPPORTED


# ------------------------------------ the benchmark's configuration, full size
def _kernel_rows(X64, rows, V, mu):
    """(K + mu I) V and sum_j |K_ij V_j| on the given rows, from the definition
    K_ij = exp(-|x_i - x_j|^2 / 2), float64, a few rows at a time."""
    out, scale = [], []
    for c in range(0, len(rows), 32):
        ii = rows[c:c + 32]
        K = np.exp(-((X64[ii, None, :] - X64[None, :, :]) ** 2).sum(-1) / 2)
        out.append(K @ V + mu * V[ii])
        scale.append(np.abs(K) @ np.abs(V) + mu * np.abs(V[ii]))
    return np.concatenate(out), np.concatenate(scale)


def test_kernel_ridge_full_size(cuda_lib):
    """n = 20000, d = 8, k = 500, 4 right-hand sides, mu = 1e-3, mixed
    precision, rtol 1e-6 (the timed configuration, same launch path): the
    double-float restart product matches the float64 definition on sampled
    rows (including the ragged last block) to ~1e-11 of the row magnitudes,
    the solve converges, and the float64 residual on sampled rows is
    consistent with the reported |b - A_mu x| / |b| <= rtol."""
    rr = cuda_lib
    n, m, k, mu, rtol = 20000, 4, 500, 1e-3, 1e-6
    X = W.mixture_points(n, 8, 10, seed=W.SEED_KERNEL)
    B = W.gaussian_rhs(n, m, W.SEED_KERNEL)
    X64 = X.astype(np.float64)
    rows = np.concatenate([np.random.default_rng(7).choice(n - 300, 160, replace=False),
                           np.arange(n - 96, n)])
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=W.SEED_KERNEL,
                  precision="mixed", max_rhs=m)
    V = np.random.default_rng(8).standard_normal((n, m))
    w = h.matvec(dev(V)).cpu().numpy().reshape(n, m)[rows]
    ref, scale = _kernel_rows(X64, rows, V, mu)
    assert np.max(np.abs(w - ref) / scale) <= 1e-11
    x, status, infos = h.solve(dev(B), rtol=rtol)
    assert status == rr.RR_OK
    assert all(i["rel_residual"] <= rtol for i in infos)
    x = x.cpu().numpy()
    Ax, _ = _kernel_rows(X64, rows, x, mu)
    r = B[rows] - Ax
    # sampled rows estimate |r|^2 / n per column; the reported residual is the
    # full float64-accurate |r| / |b|
    est = np.sqrt((r ** 2).mean(axis=0) * n) / np.linalg.norm(B, axis=0)
    rep = np.array([i["rel_residual"] for i in infos])
    assert np.all(est <= 3 * rtol)
    assert np.all(est <= 4 * rep + 1e-9) and np.all(rep <= 4 * est + 1e-9)
    h.close()


def test_kernel_ridge_full_size_error_vs_exact_solution(cuda_lib):
    """The timed configuration (n = 20000, d = 8, k = 500, 4 right-hand sides,
    mu = 1e-3, bf16 sketch, float32 iterations, float64-accurate refinement)
    against the float64 oracle's exact solution x* = (K + mu I)^-1 b, a dense
    Cholesky solve of the materialized K.  The throughput solve (rtol 1e-6)
    has a float64 residual, over all rows, within rtol and a forward error
    within 1e-5; a parity solve to rtol 1e-9 (the refinement loop run to a
    tighter target on the same inputs) is within 1e-7 of x*."""
    rr = cuda_lib
    n, m, k, mu = 20000, 4, 500, 1e-3
    X = W.mixture_points(n, 8, 10, seed=W.SEED_KERNEL)
    B = W.gaussian_rhs(n, m, W.SEED_KERNEL)
    op = O.GaussKernelOp(X, materialize=True)
    xs = O.exact_solve(op, mu, B)
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=W.SEED_KERNEL,
                  precision="mixed", max_rhs=m)
    x, status, infos = h.solve(dev(B), rtol=1e-6)
    assert status == rr.RR_OK
    x = x.cpu().numpy()
    res = O.true_rel_residual(op, mu, x, B)
    rep = np.array([i["rel_residual"] for i in infos])
    fe = np.linalg.norm(x - xs, axis=0) / np.linalg.norm(xs, axis=0)
    print(f"rtol 1e-6: residual {res}, reported {rep}, forward error {fe}")
    assert np.all(res <= 1e-6)
    assert np.allclose(res, rep, rtol=1e-3, atol=1e-12)
    assert np.all(fe <= 1e-5)
    x, status, infos = h.solve(dev(B), rtol=1e-9)
    assert status == rr.RR_OK
    x = x.cpu().numpy()
    fe = np.linalg.norm(x - xs, axis=0) / np.linalg.norm(xs, axis=0)
    print(f"rtol 1e-9: residual {O.true_rel_residual(op, mu, x, B)}, forward error {fe}")
    assert np.all(fe <= 1e-7)
    h.close()


@pytest.mark.parametrize("m", [2, 5])
def test_variant_r_persistent_step_fp32_dense(cuda_lib, m):
    """Variant R in float32 on a dense operator: the persistent launches
    around the product and the separate kernels reach the same float32
    iterate at a fixed budget (sums in another order: float32 rounding), and
    plain float32 solve reaches a float32-level residual."""
    rr = cuda_lib
    n, k, mu = 1500, 120, 1e-3
    P, op = dense_problem(n)
    B = W.gaussian_rhs(n, m, 63)
    A32 = P.A.astype(np.float32)
    op32 = O.DenseOp(A32.astype(np.float64))
    xs, its = [], []
    for impl in (0, 1):
        h = rr.Handle(rr.Operator.dense(dev(A32)), mu, k, "gaussian", seed=63,
                      precision="fp32", variant="R", max_rhs=m, iter_impl=impl)
        x, status, infos = h.solve(dev(B), rtol=1e-14, maxit=6)
        xs.append(x.cpu().numpy())
        its.append([i["inner_iters"] for i in infos])
        x, status, infos = h.solve(dev(B), rtol=1e-4)
        assert status == rr.RR_OK
        assert np.all(O.true_rel_residual(op32, mu, x.cpu().numpy(), B) <= 2e-4)
        h.close()
    assert its[0] == its[1]
    assert rel(xs[0], xs[1]) <= 1e-4
