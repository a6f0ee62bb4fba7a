"""GPU parity of Alg. 3 (randomized Q-less QR) and of the basis-less C-RandRAND
path for sparse operators (Sec. 4.2), through the C ABI, against the float64
oracle built with orth="qless" (same Theta pattern from the same seed).

Tolerances: float64 factors and iterates 1e-10 relative (the R factor is unique
once its diagonal is positive; the GPU takes it from a Cholesky QR of the
sketch S, the oracle from Householder QR, so they agree to u * cond(S));
low-precision solves are checked by their float64 residual (oracle product).
"""
import numpy as np
import pytest

from oracle import randrand as O
from workloads import generators as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def csr_problem(side, seed, fp64=True):
    C = W.diffusion_csr(side=side, seed=seed, corr_len=4.0)
    op = O.CsrOp(C.rowptr, C.colidx, C.vals, C.n)
    vals = dev(C.vals.astype(np.float64)) if fp64 else dev(C.vals)
    return C, op, vals


def csr_handle(rr, C, vals, mu, k, sketch, seed, **kw):
    return rr.Handle(rr.Operator.csr(dev(C.rowptr), dev(C.colidx), vals), mu, k, sketch,
                     seed=seed, orth="rand_cholqr", **kw)


# ------------------------------------------------------------ Alg. 3 factors
@pytest.mark.parametrize("sketch", ["sparse_sign", "gaussian", "multilevel", "srht"])
@pytest.mark.parametrize("side,k,l_sk", [(24, 40, 0), (30, 17, 50)])
def test_alg3_basis_less_factors_fp64(cuda_lib, sketch, side, k, l_sk):
    """Basis-less build on a CSR operator: R, G, tau and the power-iteration
    estimates equal the oracle's Alg. 3 build."""
    rr = cuda_lib
    C, op, vals = csr_problem(side, 41)
    mu = 1e-4
    h = csr_handle(rr, C, vals, mu, k, sketch, 41, l_sk=l_sk, max_rhs=2)
    bd = O.build(op, mu, k, sketch, seed=41, orth="qless", l_sk=l_sk or None)
    cond = np.linalg.cond(bd.R)
    R = h.export("R").cpu().numpy()
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.all(np.diag(R) > 0)
    assert rel(R, bd.R) <= max(1e-12, 1e-15 * cond) * 100
    G = h.export("G").cpu().numpy()
    assert rel(G, bd.G) <= max(1e-12, 1e-15 * cond ** 2) * 100
    tau, nE, lmax = h.scalars()
    assert nE == pytest.approx(bd.normE, rel=1e-8)
    assert lmax == pytest.approx(bd.lam_max, rel=1e-8)
    assert tau == pytest.approx(bd.tau, rel=1e-8)
    with pytest.raises(rr.RandRandError):
        h.export("Q")          # no basis is kept


def test_alg3_explicit_basis_dense_fp64(cuda_lib):
    """Alg. 3 on a dense operator keeps Q = W chol(W^T W)^-1: Q and R equal the
    oracle's (which forms Q = Y_mu R^-1)."""
    rr = cuda_lib
    n, k, mu = 700, 60, 1e-4
    P = W.dense_power_spectrum(n, seed=W.SEED_DENSE, power=2.0)
    op = O.DenseOp(P.A)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mu, k, "gaussian", seed=7, orth="rand_cholqr")
    bd = O.build(op, mu, k, "gaussian", seed=7, orth="qless")
    cond = np.linalg.cond(bd.R)
    assert rel(h.export("R").cpu().numpy(), bd.R) <= max(1e-12, 1e-15 * cond) * 100
    Q = h.export("Q").cpu().numpy()
    assert rel(Q, bd.Q) <= max(1e-12, 1e-15 * cond) * 100
    assert np.linalg.norm(Q.T @ Q - np.eye(k)) <= 1e-13


# ------------------------------------------------------- preconditioner apply
@pytest.mark.parametrize("sketch", ["sparse_sign", "gaussian", "multilevel", "srht"])
def test_basis_less_apply_fp64(cuda_lib, sketch):
    """z = P r with Q applied through A_mu, Omega and R^-1 equals the oracle's
    P r = r - Q Q^T r + tau Q G Q^T r with its explicit Q."""
    rr = cuda_lib
    C, op, vals = csr_problem(24, 42)
    mu, k = 1e-4, 40
    h = csr_handle(rr, C, vals, mu, k, sketch, 42, max_rhs=3)
    bd = O.build(op, mu, k, sketch, seed=42, orth="qless")
    r = np.random.default_rng(1).standard_normal((C.n, 3))
    z = h.apply(dev(r)).cpu().numpy()
    cond = np.linalg.cond(bd.R)
    assert rel(z, bd.apply_P(r)) <= max(1e-12, 1e-15 * cond ** 2) * 100


# ---------------------------------------------------------------- solves
@pytest.mark.parametrize("sketch", ["sparse_sign", "gaussian", "multilevel", "srht"])
@pytest.mark.parametrize("m", [1, 3])
def test_basis_less_iteration_level_fp64(cuda_lib, sketch, m):
    """After a fixed inner budget the GPU iterate equals the oracle iterate."""
    rr = cuda_lib
    C, op, vals = csr_problem(30, 43)
    mu, k = 1e-4, 48
    B = W.gaussian_rhs(C.n, m, 43)
    h = csr_handle(rr, C, vals, mu, k, sketch, 43, max_rhs=m)
    bd = O.build(op, mu, k, sketch, seed=43, orth="qless")
    for budget in (3, 12):
        x, status, infos = h.solve(dev(B), rtol=1e-14, maxit=budget)
        xo, oinfo = O.solve(bd, B, rtol=1e-14, maxit=budget)
        assert status == rr.RR_ERR_MAXIT
        assert [i["inner_iters"] for i in infos] == [i.inner_iters for i in oinfo]
        assert rel(x.cpu().numpy(), xo) <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_basis_less_solve(cuda_lib, precision):
    """Solves to rtol 1e-6 with the float64 residual as the criterion; the float64
    path also reaches the dense Cholesky solution."""
    rr = cuda_lib
    C, op, vals = csr_problem(40, 44, fp64=(precision == "fp64"))
    mu, k = 1e-6, 32
    b = W.gaussian_rhs(C.n, 2, 44)
    h = csr_handle(rr, C, vals, mu, k, "sparse_sign", 44, precision=precision, max_rhs=2)
    if precision == "fp32":
        x, status, infos = h.solve(dev(b), rtol=1e-4, maxit=20000)
        assert status == rr.RR_OK
        assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), b) <= 2e-4)
        return
    x, status, infos = h.solve(dev(b), rtol=1e-6, maxit=20000)
    assert status == rr.RR_OK
    assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), b) <= 1e-6)
    assert all(i["matvecs"] >= 3 * i["inner_iters"] for i in infos)
    if precision == "fp64":
        x, status, infos = h.solve(dev(b), rtol=1e-12, maxit=20000)
        assert status == rr.RR_OK
        xs = O.exact_solve(op, mu, b)
        assert rel(x.cpu().numpy(), xs) <= 1e-7


@pytest.mark.parametrize("sketch", ["sparse_sign", "gaussian"])
def test_basis_less_variant_R_fp64(cuda_lib, sketch):
    """Variant R (Alg. 4) without a basis: tau = |E| and R equal the oracle's
    Alg. 3 build; B p (five products with A_mu) equals the oracle's
    (I - Pi) A_mu (I - Pi) p + tau Pi p; after fixed inner budgets the
    recovered iterate equals the oracle's."""
    rr = cuda_lib
    C, op, vals = csr_problem(24, 45)
    mu, k = 1e-4, 40
    h = csr_handle(rr, C, vals, mu, k, sketch, 45, variant="R", max_rhs=3)
    bd = O.build(op, mu, k, sketch, seed=45, orth="qless", variant="R")
    cond = np.linalg.cond(bd.R)
    assert rel(h.export("R").cpu().numpy(), bd.R) <= max(1e-12, 1e-15 * cond) * 100
    tau, nE, _ = h.scalars()
    assert nE == pytest.approx(bd.normE, rel=1e-8)
    assert tau == pytest.approx(bd.tau, rel=1e-8)
    r = np.random.default_rng(6).standard_normal((C.n, 3))
    assert rel(h.apply(dev(r)).cpu().numpy(), bd.apply_B(r)) <= max(1e-12, 1e-15 * cond ** 2) * 100
    B = W.gaussian_rhs(C.n, 3, 45)
    for budget in (3, 12):
        x, status, infos = h.solve(dev(B), rtol=1e-14, maxit=budget)
        xo, oinfo = O.solve(bd, B, rtol=1e-14, maxit=budget)
        assert [i["inner_iters"] for i in infos] == [i.inner_iters for i in oinfo]
        assert rel(x.cpu().numpy(), xo) <= 1e-9
    x, status, infos = h.solve(dev(B), rtol=1e-12, maxit=20000)
    assert status == rr.RR_OK
    assert rel(x.cpu().numpy(), O.exact_solve(op, mu, B)) <= 1e-7
    assert all(i["matvecs"] >= 5 * i["inner_iters"] for i in infos)


def test_basis_less_variant_R_mixed(cuda_lib):
    rr = cuda_lib
    C, op, vals = csr_problem(40, 46, fp64=False)
    mu, k = 1e-6, 32
    b = W.gaussian_rhs(C.n, 2, 46)
    h = csr_handle(rr, C, vals, mu, k, "sparse_sign", 46, variant="R", precision="mixed",
                   max_rhs=2)
    x, status, infos = h.solve(dev(b), rtol=1e-6, maxit=20000)
    assert status == rr.RR_OK
    assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), b) <= 1e-6)


def csr_indefinite(side, seed, after=30):
    """A CSR diffusion operator and a shift between its (after+1)-th and
    (after+2)-th largest eigenvalues, so A_mu is indefinite."""
    C, op, vals = csr_problem(side, seed)
    ev = np.sort(np.linalg.eigvalsh(op.matmat(np.eye(C.n))))[::-1]
    return C, op, vals, -0.5 * (ev[after] + ev[after + 1])


@pytest.mark.parametrize("sketch", ["sparse_sign", "srht", "multilevel"])
def test_basis_less_variant_G_fp64(cuda_lib, sketch):
    """Basis-less G-RandRAND (Sec. 3.3 eq:g_randrand with the Q of Sec. 4.2:
    P = I + A_mu Omega R^-1 (tau G - I) R^-T Omega^T A_mu) on an indefinite
    CSR system: R, G, the two norm estimates and tau equal the oracle's Alg. 3
    build with its explicit Q; restarted MINRES reaches the float64 residual
    target."""
    rr = cuda_lib
    C, op, vals, mu = csr_indefinite(24, 47)
    k = 40
    h = csr_handle(rr, C, vals, mu, k, sketch, 47, variant="G", max_rhs=2)
    bd = O.build(op, mu, k, sketch, seed=47, orth="qless", variant="G")
    cond = np.linalg.cond(bd.R)
    assert rel(h.export("R").cpu().numpy(), bd.R) <= max(1e-12, 1e-15 * cond) * 100
    assert rel(h.export("G").cpu().numpy(), bd.G) <= 1e-9
    tau, nE, lmax = h.scalars()
    assert nE == pytest.approx(bd.normE, rel=1e-7)
    assert lmax == pytest.approx(bd.lam_max, rel=1e-7)
    assert tau == pytest.approx(bd.tau, rel=1e-7)
    b = W.gaussian_rhs(C.n, 2, 47)
    x, status, infos = h.solve(dev(b), rtol=1e-10)
    assert status == rr.RR_OK
    assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), b) <= 1e-10)
    # about the oracle's number of restarted MINRES steps: over ~800 steps on
    # an indefinite system the restarts fall at rounding-dependent points (the
    # GPU's reductions sum in a different order), measured within 12 %
    _, oinfos = O.solve(bd, b, rtol=1e-10)
    for gi, oi in zip(infos, oinfos):
        assert abs(gi["inner_iters"] - oi.inner_iters) <= max(3, oi.inner_iters // 5)


def test_basis_less_variant_G_mixed(cuda_lib):
    """Basis-less G-RandRAND with float32 iterations and float64 restart
    residuals on an indefinite float32 CSR system: restarted MINRES meets
    rtol 1e-6 with the float64 residual as the criterion."""
    rr = cuda_lib
    C, op, _, mu = csr_indefinite(24, 48)
    vals32 = dev(C.vals.astype(np.float32))
    h = csr_handle(rr, C, vals32, mu, 40, "sparse_sign", 48, variant="G", precision="mixed",
                   max_rhs=4)
    b = W.gaussian_rhs(C.n, 4, 48)
    x, status, infos = h.solve(dev(b), rtol=1e-6, maxit=20000)
    assert status == rr.RR_OK
    assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), b) <= 1e-6)


def test_basis_less_variant_G_needs_room(cuda_lib):
    """The basis-less MINRES keeps two n x m temporaries in the n x k basis
    array: k < 2 m is rejected."""
    rr = cuda_lib
    C, op, vals = csr_problem(16, 45)
    with pytest.raises(rr.RandRandError):
        csr_handle(rr, C, vals, -1e-2, 8, "sparse_sign", 45, variant="G", max_rhs=8)


def test_sparse_operator_full_size(cuda_lib):
    """The 512 x 512 variable-coefficient diffusion operator (n = 262144, CSR
    float32, log-normal coefficients sigma = 1, correlation length 16),
    mu = 1e-6, k = 256, sparse-sign Omega with 8 nonzeros per row, Alg. 3 with
    l_sk = 1024, basis-less C-RandRAND PCG with float32 iterations and float64
    refinement to rtol 1e-6.  Criterion: the float64 residual of the oracle's
    product, per column."""
    rr = cuda_lib
    C = W.diffusion_csr(side=512, seed=W.SEED_CSR)
    op = O.CsrOp(C.rowptr, C.colidx, C.vals, C.n)
    mu, k = 1e-6, 256
    b = W.gaussian_rhs(C.n, 1, W.SEED_CSR)
    h = rr.Handle(rr.Operator.csr(dev(C.rowptr), dev(C.colidx), dev(C.vals)), mu, k,
                  "sparse_sign", seed=W.SEED_CSR, precision="mixed", orth="rand_cholqr",
                  l_sk=1024)
    x, status, infos = h.solve(dev(b), rtol=1e-6, maxit=50000)
    assert status == rr.RR_OK
    res = O.true_rel_residual(op, mu, x.cpu().numpy(), b)
    assert res[0] <= 1e-6
    assert infos[0]["rel_residual"] == pytest.approx(res[0], rel=1e-3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_persistent_basis_less_matches_separate_kernels(cuda_lib, precision):
    """The persistent basis-less iteration in its shared-memory window form
    (iter_impl 0) and without windows (iter_impl 2), and the separate kernels
    (iter_impl 1) agree: float64 iterates to 1e-10 at a fixed budget (an odd
    one: the window form's r and p end in their second buffers), and all
    solve to rtol with the float64 residual as the criterion."""
    rr = cuda_lib
    C, op, vals = csr_problem(40, 46, fp64=(precision == "fp64"))
    mu, k = 1e-6, 32
    B = W.gaussian_rhs(C.n, 3, 46)
    _persistent_forms_agree(rr, C, op, vals, mu, k, B, 46, precision)


def _persistent_forms_agree(rr, C, op, vals, mu, k, B, seed, precision):
    res = {}
    for impl in (0, 2, 1):
        h = csr_handle(rr, C, vals, mu, k, "sparse_sign", seed, precision=precision,
                       max_rhs=B.shape[1], iter_impl=impl)
        if precision == "fp64":
            x, status, infos = h.solve(dev(B), rtol=1e-14, maxit=25)
            assert status == rr.RR_ERR_MAXIT
            res[impl] = x.cpu().numpy()
        x, status, infos = h.solve(dev(B), rtol=1e-6, maxit=20000)
        assert status == rr.RR_OK
        assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)
        h.close()
    if precision == "fp64":
        assert rel(res[0], res[1]) <= 1e-10
        assert rel(res[2], res[1]) <= 1e-10


def random_graph_csr(n, deg, seed):
    """SPD CSR without band structure: the weighted Laplacian of a random
    graph (deg edges drawn per row, symmetrised) plus 1e-2 I, so that every
    CTA's rows read columns across the whole range."""
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(seed)
    i = np.repeat(np.arange(n), deg)
    j = rng.integers(0, n, n * deg)
    w = rng.uniform(0.5, 2.0, n * deg)
    keep = i != j
    M = sp.coo_matrix((w[keep], (i[keep], j[keep])), shape=(n, n)).tocsr()
    M = M + M.T
    A = (sp.diags(np.asarray(M.sum(axis=1)).ravel()) - M + 1e-2 * sp.eye(n)).tocsr()
    A.sort_indices()
    return W.CsrMatrix(n=n, rowptr=A.indptr.astype(np.int32), colidx=A.indices.astype(np.int32),
                       vals=A.data.astype(np.float64))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_persistent_forms_wide_and_banded_windows(cuda_lib, precision):
    """Window form against the other two where the windows differ in kind: a
    200 x 200 diffusion grid (each CTA's 264 rows read 200 rows on each side)
    and a random graph Laplacian (every CTA reads nearly all 3000 rows)."""
    rr = cuda_lib
    C, op, vals = csr_problem(200, 47, fp64=(precision == "fp64"))
    _persistent_forms_agree(rr, C, op, vals, 1e-5, 48, W.gaussian_rhs(C.n, 2, 47), 47, precision)
    G = random_graph_csr(3000, 3, 48)
    vals = dev(G.vals) if precision == "fp64" else dev(G.vals.astype(np.float32))
    opg = O.CsrOp(G.rowptr, G.colidx, G.vals, G.n)
    _persistent_forms_agree(rr, G, opg, vals, 1e-4, 40, W.gaussian_rhs(G.n, 3, 48), 48, precision)


@pytest.mark.parametrize("max_rhs,m", [(4, 2), (8, 3), (2, 1)])
def test_window_form_fewer_columns_than_handle(cuda_lib, max_rhs, m):
    """The window form computes only the solve's columns (rounded up) of a
    handle built for more: float64 iterates at a fixed budget equal the
    separate kernels', and a second solve with all columns still agrees."""
    rr = cuda_lib
    C, op, vals = csr_problem(48, 49)
    mu, k = 1e-5, 36
    B = W.gaussian_rhs(C.n, max_rhs, 49)
    out = {}
    for impl in (0, 1):
        h = csr_handle(rr, C, vals, mu, k, "sparse_sign", 49, max_rhs=max_rhs, iter_impl=impl)
        x, status, _ = h.solve(dev(B[:, :m]), rtol=1e-14, maxit=31)
        assert status == rr.RR_ERR_MAXIT
        xa, status, _ = h.solve(dev(B), rtol=1e-14, maxit=17)
        out[impl] = (x.cpu().numpy(), xa.cpu().numpy())
        h.close()
    assert rel(out[0][0], out[1][0]) <= 1e-10
    assert rel(out[0][1], out[1][1]) <= 1e-10
