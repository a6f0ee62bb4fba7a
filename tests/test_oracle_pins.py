"""Pins of the float64 oracle to facts fixed by the paper and by mathematics.

None of these re-types an oracle formula: each checks the oracle against an
independent computation (dense inverse, dense eigenvalues, a closed-form
spectrum, a textbook routine, brute force) or an invariant the paper proves.
"""
import math

import numpy as np
import pytest

from oracle import philox
from oracle import randrand as O
from workloads import generators as W


# --------------------------------------------------------------------------
# fixtures
# --------------------------------------------------------------------------
def small_dense(n=160, power=2.0, seed=11):
    P = W.dense_power_spectrum(n, seed=seed, power=power)
    return P, O.DenseOp(P.A)


def dense_inv(op, mu):
    return np.linalg.inv(op.dense() + mu * np.eye(op.n))


def sym_sqrt(M):
    w, V = np.linalg.eigh(0.5 * (M + M.T))
    return (V * np.sqrt(np.maximum(w, 0))) @ V.T


# --------------------------------------------------------------------------
# Philox streams: statistics and structure (the paper fixes no generator)
# --------------------------------------------------------------------------
def test_philox_known_answer_vectors():
    """The generator against the published Philox4x32-10 known-answer vectors."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")
    with open(path) as f:
        kat = json.load(f)["vectors"]
    for v in kat:
        ctr = np.array([[int(x, 16) for x in v["counter"]]], dtype=np.uint64)
        key = tuple(int(x, 16) for x in v["key"])
        got = philox.philox4x32_10(ctr, key)[0]
        assert [int(x) for x in got] == [int(x, 16) for x in v["words"]]


def test_philox_uniform_statistics():
    n = 1 << 18
    ctr = np.zeros((n // 4, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(n // 4)
    w = philox.philox4x32_10(ctr, philox.seed_key(12345)).ravel()
    u = philox.uniform24(w)
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5e-3 / 12 * 4
    # every bit of the 32-bit words is balanced
    bits = (w[:, None] >> np.arange(32, dtype=np.uint32)) & 1
    frac = bits.mean(axis=0)
    assert np.all(np.abs(frac - 0.5) < 5 * 0.5 / math.sqrt(n))
    # chi-square of the top byte over 256 bins
    hist = np.bincount((w >> 24).astype(np.int64), minlength=256)
    exp = n / 256
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)


def test_philox_avalanche_and_key_dependence():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(2048, 4), dtype=np.uint64)
    key = (0x1234, 0x5678)
    base = philox.philox4x32_10(ctr, key)
    for word in range(4):
        for bit in (0, 13, 31):
            c2 = ctr.copy()
            c2[:, word] ^= np.uint64(1 << bit)
            diff = philox.philox4x32_10(c2, key) ^ base
            flips = np.unpackbits(diff.view(np.uint8)).mean()
            assert abs(flips - 0.5) < 0.02
    other = philox.philox4x32_10(ctr, (0x1235, 0x5678)) ^ base
    assert abs(np.unpackbits(other.view(np.uint8)).mean() - 0.5) < 0.02


def test_gaussian_omega_moments():
    n, k = 4000, 64
    Om = philox.gaussian_omega(n, k, seed=77)
    z = Om.ravel() * math.sqrt(k)            # entries N(0, 1/k) (Sec. 2)
    N = z.size
    assert abs(z.mean()) < 5 / math.sqrt(N)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / N)
    kurt = (z ** 4).mean() / z.var() ** 2
    assert abs(kurt - 3) < 5 * math.sqrt(24 / N)
    # columns nearly orthogonal with norm^2 ~ n/k
    G = Om.T @ Om
    assert np.allclose(np.diag(G), n / k, rtol=0.15)
    # independent counters -> distinct seeds give different matrices
    assert not np.allclose(Om, philox.gaussian_omega(n, k, seed=78))


def test_sparse_sign_structure():
    n, k, gamma = 3000, 40, 8
    cols, sgn = philox.sparse_sign_pattern(n, k, gamma, seed=5, stream=philox.STREAM_OMEGA)
    assert cols.min() >= 0 and cols.max() < k
    for r in range(n):
        assert len(set(cols[r].tolist())) == gamma      # distinct per row
    assert set(np.unique(sgn)) == {-1, 1}
    assert abs(sgn.mean()) < 5 / math.sqrt(sgn.size)
    # column choice uniform: chi-square over k bins
    hist = np.bincount(cols.ravel(), minlength=k)
    exp = n * gamma / k
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < (k - 1) + 6 * math.sqrt(2 * (k - 1))
    Om = philox.sparse_sign_omega_dense(n, k, gamma, seed=5)
    assert np.allclose(np.abs(Om[Om != 0]), 1 / math.sqrt(gamma))
    assert np.all((Om != 0).sum(axis=1) == gamma)
    Th = philox.theta_dense(32, 500, 8, seed=5)
    assert np.all((Th != 0).sum(axis=0) == 8)


def test_bf16_rounding_brute_force():
    # brute force: the nearest bfloat16 (ties to even) among all candidates
    rng = np.random.default_rng(3)
    x = rng.standard_normal(2000) * 10.0 ** rng.integers(-3, 3, 2000)
    r = philox.round_bf16(x)
    x32 = x.astype(np.float32).astype(np.float64)
    for xi, ri in zip(x32, r):
        u = np.array([xi], dtype=np.float32).view(np.uint32)[0] & 0xFFFF0000
        lo = np.array([u], dtype=np.uint32).view(np.float32)[0].astype(np.float64)
        hi = np.array([u + 0x10000], dtype=np.uint32).view(np.float32)[0].astype(np.float64)
        cands = sorted([lo, hi], key=lambda c: (abs(c - xi),
                                                int(np.array([c], np.float32).view(np.uint32)[0] >> 16) & 1))
        assert ri == cands[0]


# --------------------------------------------------------------------------
# Input generators
# --------------------------------------------------------------------------
def test_dense_generator_closed_form_spectrum():
    P = W.dense_power_spectrum(300, seed=1)
    ev = np.linalg.eigvalsh(P.A)[::-1]
    assert np.max(np.abs(ev - np.arange(1, 301) ** -2.0)) < 1e-13
    assert np.allclose(P.U.T @ P.U, np.eye(300), atol=1e-13)


def test_kernel_operator_brute_force():
    X = W.mixture_points(60, seed=3)
    op = O.GaussKernelOp(X, bandwidth=1.3)
    K = op.dense()
    for i, j in [(0, 0), (0, 5), (17, 42), (59, 1)]:
        d2 = sum((float(X[i, c]) - float(X[j, c])) ** 2 for c in range(X.shape[1]))
        assert K[i, j] == pytest.approx(math.exp(-d2 / (2 * 1.3 ** 2)), rel=1e-14)
    assert np.allclose(K, K.T) and np.allclose(np.diag(K), 1.0)
    v = np.random.default_rng(0).standard_normal((60, 3))
    assert np.allclose(op.matmat(v), K @ v, rtol=1e-13, atol=1e-13)


def test_csr_generator_properties():
    C = W.diffusion_csr(side=24, seed=9, corr_len=4.0)
    assert C.nnz == 5 * C.n - 4 * 24
    D = C.to_dense()
    assert np.allclose(D, D.T)
    assert np.all(D.sum(axis=1) > -1e-5)              # weak diagonal dominance
    assert np.linalg.eigvalsh(D).min() > 0             # SPD with Dirichlet boundary
    op = O.CsrOp(C.rowptr, C.colidx, C.vals, C.n)
    v = np.random.default_rng(1).standard_normal(C.n)
    assert np.allclose(op.matmat(v), D @ v)


# --------------------------------------------------------------------------
# Projector, basis and the identity A_mu^-1 Pi = Omega (A_mu Omega)^+
# --------------------------------------------------------------------------
@pytest.mark.parametrize("sketch", ["gaussian", "sparse_sign"])
def test_projector_is_orthogonal_projector_onto_range(sketch):
    P, op = small_dense()
    k, mu = 20, 1e-3
    bd = O.build(op, mu, k, sketch, seed=3)
    Pi = bd.Pi(np.eye(op.n))
    assert np.linalg.norm(Pi @ Pi - Pi, 2) <= 1e-12          # idempotent
    assert np.linalg.norm(Pi - Pi.T, 2) <= 1e-12             # symmetric
    assert abs(np.trace(Pi) - k) < 1e-10                     # rank k
    Ymu = op.A @ bd.Omega + mu * bd.Omega                    # independent A_mu Omega
    assert np.linalg.norm(Ymu - Pi @ Ymu) <= 1e-12 * np.linalg.norm(Ymu)
    assert np.linalg.norm(bd.Q @ bd.R - Ymu) <= 1e-13 * np.linalg.norm(Ymu)
    assert np.all(np.diag(bd.R) > 0)


def test_invAPi_identity_against_dense_inverse():
    # Sec. 1.1 eq:invAPi: A_mu^-1 Pi = Omega (A_mu Omega)^+, used through
    # Omega R^-1 Q^T (eq:projector)
    P, op = small_dense()
    mu = 1e-2
    bd = O.build(op, mu, 15, "gaussian", seed=4)
    lhs = dense_inv(op, mu) @ bd.Pi(np.eye(op.n))
    rhs = bd.Ainv_Pi(np.eye(op.n))
    assert np.linalg.norm(lhs - rhs, 2) <= 1e-10 * np.linalg.norm(lhs, 2)
    pinv = bd.Omega @ np.linalg.pinv(op.A @ bd.Omega + mu * bd.Omega)
    assert np.linalg.norm(pinv - rhs, 2) <= 1e-9 * np.linalg.norm(lhs, 2)


def test_core_matrix_G_equals_QT_Ainv_Q():
    # G = R^-T (Omega^T A_mu Omega) R^-1 (eq:g_randrand_explicit) equals
    # Q^T A_mu^-1 Q by eq:invAPi; the oracle forms G as (R_M R^-1)^T (R_M R^-1)
    P, op = small_dense()
    mu = 1e-2
    bd = O.build(op, mu, 25, "gaussian", seed=5)
    ref = bd.Q.T @ dense_inv(op, mu) @ bd.Q
    assert np.linalg.norm(bd.G - ref, 2) <= 1e-9 * np.linalg.norm(ref, 2)
    assert np.linalg.eigvalsh(bd.G).min() > 0


def test_nystrom_preconditioner_is_c_randrand_at_mu_zero():
    # Sec. 1.3: for mu = 0 the Nystrom approximation
    # A_hat = A Omega (Omega^T A Omega)^-1 Omega^T A equals (Pi A^-1 Pi)^+, so
    # the Nystrom preconditioner lambda_hat_min A_hat^+ + (I - U U^T), with
    # (U, Lambda_hat) the nonzero eigenpairs of A_hat, is C-RandRAND with
    # tau = |Pi A^-1 Pi|^-1.  The Nystrom side here is the textbook route (an
    # eigendecomposition of A_hat), tau comes from a dense inverse, and
    # neither uses the oracle's R, G or power iterations.
    P, op = small_dense(n=140)
    n, k = op.n, 12
    A = op.A
    Om = np.random.default_rng(3).standard_normal((n, k))
    Y = A @ Om
    Ahat = Y @ np.linalg.solve(Om.T @ Y, Y.T)
    w, V = np.linalg.eigh(0.5 * (Ahat + Ahat.T))
    U, lam = V[:, -k:], w[-k:]
    assert lam.min() > 1e6 * abs(w[:-k]).max()          # rank k, well separated
    I = np.eye(n)
    P_nys = lam.min() * (U / lam) @ U.T + (I - U @ U.T)
    Qy = np.linalg.qr(Y)[0]
    Pi = Qy @ Qy.T
    tau = 1.0 / np.linalg.norm(Pi @ np.linalg.inv(A) @ Pi, 2)
    bd = O.build(op, 0.0, k, omega=Om, tau=tau)
    P_c = bd.apply_P(I)
    assert np.linalg.norm(P_c - P_nys, 2) <= 1e-8 * np.linalg.norm(P_nys, 2)
    # the same tau through the oracle's own factors: 1 / lambda_max(G)
    assert tau == pytest.approx(1.0 / np.linalg.eigvalsh(bd.G).max(), rel=1e-8)


# --------------------------------------------------------------------------
# Special cases with closed-form spectra
# --------------------------------------------------------------------------
@pytest.mark.parametrize("q", [0, 1])
@pytest.mark.parametrize("variant", ["C", "R"])
def test_exact_eigenvector_deflation_spectrum(variant, q):
    # X^T = U_k (exact top-k eigenvectors), Omega = A^q X^T spans the same
    # space: Pi = U_k U_k^T and both the R-RandRAND operator B (eq:APdef2)
    # and the C-RandRAND P A_mu have spectrum {tau (k times)} U
    # {lambda_i + mu, i > k}
    P, op = small_dense(n=120)
    k, mu = 10, 1e-3
    bd = O.build(op, mu, k, omega=P.U[:, :k], variant=variant, q=q)
    I = np.eye(op.n)
    if variant == "C":
        M = bd.apply_P(I) @ (op.A + mu * I)
    else:
        M = bd.apply_B(I)
    ev = np.sort(np.linalg.eigvals(M).real)
    expect = np.sort(np.concatenate([np.full(k, bd.tau), P.lam[k:] + mu]))
    assert np.allclose(ev, expect, rtol=1e-9, atol=1e-12)
    if variant == "C":
        # Pi A_mu Pi~ = Pi on range(Q): lambda_max = 1 exactly
        assert bd.lam_max == pytest.approx(1.0, rel=1e-10)
        # eq:optimal_rho with F = 1/mu: tau = sqrt(mu |E| / lambda_max)
        assert bd.tau == pytest.approx(math.sqrt(mu * bd.normE / bd.lam_max), rel=1e-14)
    # |E| = lambda_{k+1} + mu is approached from below by the power iteration
    assert bd.normE <= (P.lam[k] + mu) * (1 + 1e-12)
    assert bd.normE >= 0.5 * (P.lam[k] + mu)


def test_subspace_iteration_test_matrix():
    # eq:testmatrix with q = 1: Omega = A X^T (A, not A_mu), and the basis
    # A_mu Omega deflates the spectrum closer to the optimum lambda_{k+1} + mu
    # than q = 0 (range approximation of Sec. 4 with one power; power-law
    # spectra, same X)
    for power in (1.0, 2.0):
        P, op = small_dense(n=400, power=power)
        k, mu = 20, 1e-4
        X = O.make_omega(op.n, k, "gaussian", seed=8)
        assert np.allclose(O.make_omega(op.n, k, "gaussian", seed=8, q=1, op=op), op.A @ X,
                           rtol=0, atol=1e-14)
        ratios = []
        for q in (0, 1):
            bd = O.build(op, mu, k, "gaussian", seed=8, q=q)
            I = np.eye(op.n)
            E = (I - bd.Pi(I)) @ (op.A + mu * I) @ (I - bd.Pi(I))
            ratios.append(np.linalg.norm(E, 2) / (P.lam[k] + mu))
        assert 1.0 <= ratios[1] < ratios[0]
        assert ratios[1] <= 1.8


@pytest.mark.parametrize("variant", ["C", "R"])
def test_full_sketch_converges_in_one_iteration(variant):
    # k = n: Pi = I, P = tau A_mu^-1 (C) and B = tau I (R): one CG step
    P, op = small_dense(n=40)
    bd = O.build(op, 1e-2, 40, "gaussian", seed=6, variant=variant)
    b = W.gaussian_rhs(40, 1, 6)[:, 0]
    x, info = O.solve(bd, b, rtol=1e-10, fixed_inner=1)
    assert O.true_rel_residual(op, 1e-2, x, b)[0] < 1e-9


def test_c_randrand_eigenvalue_bracket():
    # Prop. thm:cnd_bound2 eq:c_randrand_eigenvalues:
    # (|F| + 1/tau)^-1 <= lambda_i(P^1/2 A_mu P^1/2) <= (1 + rho) |E|,
    # rho = tau lambda_max(Pi A_mu Pi A_mu^-1 Pi) / |E|; all from dense algebra
    P, op = small_dense(n=150, power=1.5)
    mu = 1e-3
    bd = O.build(op, mu, 12, "gaussian", seed=7)
    I = np.eye(op.n)
    Amu = op.A + mu * I
    Pi = bd.Pi(I)
    E = (I - Pi) @ Amu @ (I - Pi)
    F = (I - Pi) @ np.linalg.inv(Amu) @ (I - Pi)
    nE, nF = np.linalg.norm(E, 2), np.linalg.norm(F, 2)
    lmax = np.max(np.linalg.eigvals(Pi @ Amu @ Pi @ np.linalg.inv(Amu) @ Pi).real)
    rho = bd.tau * lmax / nE
    Pm = bd.apply_P(I)
    S = sym_sqrt(Pm)
    ev = np.linalg.eigvalsh(S @ Amu @ S)
    assert ev.min() >= (nF + 1 / bd.tau) ** -1 * (1 - 1e-9)
    assert ev.max() <= (1 + rho) * nE * (1 + 1e-9)
    # power-iteration estimates: |E| (symmetric E) from below; lambda_max of
    # the product of two SPD factors (not normal: the norm ratio may overshoot)
    assert bd.normE <= nE * (1 + 1e-12) and bd.normE >= 0.8 * nE
    assert abs(bd.lam_max - lmax) <= 0.05 * lmax
    # Prop. thm:cnd_bound2_ext eq:c_randrand_eigenvalues2_ext
    Ainv = np.linalg.inv(Amu)
    N = Pi @ Ainv @ Pi
    w, V = np.linalg.eigh(0.5 * (N + N.T))
    keep = w > 1e-12 * w.max()
    Nh = (V[:, keep] * np.sqrt(w[keep])) @ V[:, keep].T
    Nmh = (V[:, keep] / np.sqrt(w[keep])) @ V[:, keep].T
    C1 = (I - Pi) @ Ainv @ Pi @ Nmh
    C2 = (I - Pi) @ Amu @ Pi @ Nh
    lmin = np.linalg.eigvalsh(Amu).min()
    lo = (max(1 / lmin, 1 / bd.tau) + bd.tau ** -0.5 * np.linalg.norm(C1 + C1.T, 2)) ** -1
    hi = max(nE, lmax) + bd.tau ** 0.5 * np.linalg.norm(C2 + C2.T, 2)
    assert ev.min() >= lo * (1 - 1e-9) and ev.max() <= hi * (1 + 1e-9)


@pytest.mark.parametrize("seed", range(6))
def test_power_estimate_of_E_within_five_percent_from_below(seed):
    # |E| = |(I - Pi) A_mu (I - Pi)| by 20 power iterations (Alg. 7 step 2,
    # the count fixed at 20): on the lambda_i = i^-2 spectrum the norm-ratio
    # estimate of a symmetric PSD matrix never exceeds the 2-norm and is
    # within 5% of the dense value
    n, k, mu = 400, 30, 1e-4
    P = W.dense_power_spectrum(n, seed=W.SEED_DENSE, power=2.0)
    op = O.DenseOp(P.A)
    bd = O.build(op, mu, k, "gaussian", seed=seed)
    I = np.eye(n)
    Pi = bd.Pi(I)
    nE = np.linalg.norm((I - Pi) @ (P.A + mu * I) @ (I - Pi), 2)
    assert 0.95 * nE <= bd.normE <= nE * (1 + 1e-12)


def test_r_randrand_condition_bound():
    # Prop. thm:cnd_bound eq:cnd_bound: for lambda_min <= tau <= |E| the
    # spectrum of B lies in [lambda_min(A_mu), |E|] (rho = 1)
    P, op = small_dense(n=150, power=1.5)
    mu = 1e-3
    bd = O.build(op, mu, 12, "gaussian", seed=8, variant="R")
    I = np.eye(op.n)
    Amu = op.A + mu * I
    Pi = bd.Pi(I)
    nE = np.linalg.norm((I - Pi) @ Amu @ (I - Pi), 2)
    lmin = np.linalg.eigvalsh(Amu).min()
    assert lmin <= bd.tau <= nE * (1 + 1e-12)
    ev = np.linalg.eigvalsh(0.5 * (bd.apply_B(I) + bd.apply_B(I).T))
    assert ev.min() >= min(bd.tau, lmin) * (1 - 1e-9)
    assert ev.max() <= max(bd.tau, nE) * (1 + 1e-9)
    # B P^-1 = A_mu (the recovery is exact): x = P y solves A_mu x = B y
    y = np.random.default_rng(0).standard_normal(op.n)
    assert np.allclose(Amu @ bd.recover_R(y), bd.apply_B(y[:, None])[:, 0], rtol=1e-9, atol=1e-12)


def test_iteration_count_within_convergence_bound():
    # Prop. thm:conv_bound: |y - y_t|_B <= 2 exp(-2t/T) |y - y_0|_B with
    # T = (|E| / (lambda_n + mu))^1/2.  Since |r_t| / |r_0| <= cond(B)^1/2
    # times the B-norm ratio and cond(B) <= T^2 here, reaching |r_t| <= u |r_0|
    # takes at most t = ceil(T/2 (log(2T) + log(1/u))) CG steps (exact |E|).
    P, op = small_dense(n=200, power=2.0)
    mu, u = 1e-4, 1e-8
    bd = O.build(op, mu, 20, "gaussian", seed=9, variant="R")
    I = np.eye(op.n)
    Pi = bd.Pi(I)
    nE = np.linalg.norm((I - Pi) @ (op.A + mu * I) @ (I - Pi), 2)
    T = math.sqrt(nE / (P.lam[-1] + mu))
    b = W.gaussian_rhs(op.n, 1, 9)[:, 0]
    y, it = O.pcg(bd.apply_B, b, lambda v: v, u * np.linalg.norm(b), 10 * op.n)
    assert it <= math.ceil(T / 2 * (math.log(2 * T) + math.log(1 / u)))
    assert it > 0


# --------------------------------------------------------------------------
# Solutions against the dense Cholesky solve
# --------------------------------------------------------------------------
@pytest.mark.parametrize("variant", ["C", "R"])
@pytest.mark.parametrize("sketch", ["gaussian", "sparse_sign"])
def test_solution_matches_dense_cholesky(variant, sketch):
    P, op = small_dense(n=300)
    mu, rtol = 1e-4, 1e-10
    bd = O.build(op, mu, 30, sketch, seed=10, variant=variant)
    B = W.gaussian_rhs(op.n, 3, 10)
    X, infos = O.solve(bd, B, rtol)
    Xs = O.exact_solve(op, mu, B)
    cond = (1 + mu) / (P.lam[-1] + mu)
    assert all(i.converged for i in infos)
    assert np.all(O.true_rel_residual(op, mu, X, B) <= rtol)
    err = np.linalg.norm(X - Xs, axis=0) / np.linalg.norm(Xs, axis=0)
    assert np.all(err <= cond * rtol)


def test_kernel_system_solution():
    X = W.mixture_points(400, seed=12)
    op = O.GaussKernelOp(X)
    mu = 1e-3
    bd = O.build(op, mu, 40, "gaussian", seed=12)
    B = W.gaussian_rhs(400, 2, 12)
    Xs = O.exact_solve(op, mu, B)
    Xo, infos = O.solve(bd, B, 1e-10)
    assert np.allclose(Xo, Xs, rtol=0, atol=1e-7 * np.abs(Xs).max())


# --------------------------------------------------------------------------
# Alg. 3 (randomised Q-less preconditioned Cholesky QR)
# --------------------------------------------------------------------------
def test_qless_R_matches_householder():
    P, op = small_dense(n=400, power=1.0)
    mu, k = 1e-6, 30
    Om = O.make_omega(op.n, k, "sparse_sign", 13)
    Ymu = op.A @ Om + mu * Om
    Th = philox.theta_dense(4 * k, op.n, 8, 13)
    R3 = O.fast_q_less_precond_chol_qr(Ymu, Th)
    _, Rh = O.householder_qr(Ymu)
    c = np.linalg.cond(Ymu)
    assert np.linalg.norm(R3 - Rh) <= 1e3 * c * 1e-16 * np.linalg.norm(Rh)
    # orthogonality of Q = Y R^-1 scales with u cond (Sec. 4.2), not u cond^2
    Q = O.right_solve_upper(Ymu, R3)
    assert np.linalg.norm(Q.T @ Q - np.eye(k), 2) <= 1e3 * c * 1e-16
    # the embedding makes W = Y R_sk^-1 well conditioned (eq:epsilon_embedding)
    _, Rsk = O.householder_qr(Th @ Ymu)
    assert np.linalg.cond(O.right_solve_upper(Ymu, Rsk)) < 10


def test_qless_G_variant_matches_householder_on_indefinite_csr():
    """G-RandRAND through Alg. 3 (the oracle route the basis-less GPU form is
    compared with) equals the Householder route on an indefinite CSR system:
    the same unique R, the same G = (R^-T Omega^T Omega R^-1)^(1/2), the two
    norm estimates and tau; and P is symmetric positive definite."""
    C = W.diffusion_csr(side=16, seed=11, corr_len=4.0)
    op = O.CsrOp(C.rowptr, C.colidx, C.vals, C.n)
    A = op.matmat(np.eye(C.n))
    ev = np.sort(np.linalg.eigvalsh(A))[::-1]
    mu = -0.5 * (ev[20] + ev[21])                       # A_mu indefinite
    k = 30
    hq = O.build(op, mu, k, "sparse_sign", seed=11, variant="G", orth="qless")
    hh = O.build(op, mu, k, "sparse_sign", seed=11, variant="G", orth="householder")
    c = np.linalg.cond(hh.R)
    assert np.linalg.norm(hq.R - hh.R) <= 1e3 * c * 1e-16 * np.linalg.norm(hh.R)
    assert np.allclose(hq.G, hh.G, rtol=0, atol=1e-9 * np.abs(hh.G).max())
    assert hq.normE == pytest.approx(hh.normE, rel=1e-8)
    assert hq.lam_max == pytest.approx(hh.lam_max, rel=1e-8)
    assert hq.tau == pytest.approx(hh.tau, rel=1e-8)
    Pm = hq.apply_P(np.eye(C.n))
    assert np.allclose(Pm, Pm.T, atol=1e-10)
    assert np.linalg.eigvalsh(0.5 * (Pm + Pm.T)).min() > 0


# --------------------------------------------------------------------------
# Lemma thm:apriori_gen00: expected projection error with l = 2k+2
# --------------------------------------------------------------------------
@pytest.mark.slow
def test_gaussian_range_approximation_expectation():
    n, kk = 256, 8
    l = 2 * kk + 2
    P = W.dense_power_spectrum(n, seed=21, power=1.0)
    mu = 1e-3
    Amu = P.A + mu * np.eye(n)
    sig = P.lam + mu
    sr = (sig[kk - 1:] ** 2).sum() / sig[kk - 1] ** 2
    bound = (2 + math.sqrt(2) * math.e * math.sqrt(sr / kk)) * sig[kk - 1]
    errs = []
    for s in range(40):
        Om = philox.gaussian_omega(n, l, seed=1000 + s)
        Q, _ = np.linalg.qr(Amu @ Om)
        errs.append(np.linalg.norm(Amu - Q @ (Q.T @ Amu), 2))
    assert np.mean(errs) <= bound


# --------------------------------------------------------------------------
# Planted mistakes: each pin above must catch a plausible slip in the oracle
# --------------------------------------------------------------------------
def test_pins_catch_planted_mistakes(monkeypatch):
    P, op = small_dense(n=80)
    mu, k = 1e-3, 8
    I = np.eye(op.n)

    def spectrum_ok(bd):
        M = bd.apply_P(I) @ (op.A + mu * I)
        ev = np.sort(np.linalg.eigvals(M).real)
        expect = np.sort(np.concatenate([np.full(k, bd.tau), P.lam[k:] + mu]))
        return np.allclose(ev, expect, rtol=1e-9, atol=1e-12)

    good = O.build(op, mu, k, omega=P.U[:, :k])
    assert spectrum_ok(good)

    # (1) dropped "- Q Q^T V" term in P
    monkeypatch.setattr(O.Build, "apply_P",
                        lambda self, V: V + self.tau * (self.Q @ (self.G @ (self.Q.T @ V))))
    assert not spectrum_ok(good)
    monkeypatch.undo()

    # (2) transposed R in A_mu^-1 Pi
    bd = O.build(op, mu, k, "gaussian", seed=1)
    lhs = dense_inv(op, mu) @ bd.Pi(I)
    monkeypatch.setattr(O.Build, "Ainv_Pi",
                        lambda self, V: self.Omega @ O.solve_upper(self.R.T.copy(), self.Q.T @ V))
    assert np.linalg.norm(lhs - bd.Ainv_Pi(I), 2) > 1e-6 * np.linalg.norm(lhs, 2)
    monkeypatch.undo()

    # (3) wrong sign of the shift in the basis
    orig = O.shifted
    bad = O.build(op, -mu, k, "gaussian", seed=1)
    assert np.linalg.norm((op.A + mu * I) @ bad.Omega - bad.Q @ bad.R) > 1e-8
    assert orig is O.shifted


# ------------------------------------------------ multiple shifts (Sec. 5.1)
def test_shift_gram_separation_matches_direct_gram():
    """The Gram separation of the parameter-free projections equals the Gram
    of Y_mu formed directly, for several shifts (A symmetric)."""
    P = W.dense_power_spectrum(300, seed=81, power=2.0)
    op = O.DenseOp(P.A)
    sk = O.shift_sketch(op, 24, "gaussian", seed=81)
    for mu in (0.0, 1e-4, 0.3, 5.0):
        Ymu = P.A @ sk.Omega + mu * sk.Omega
        direct = Ymu.T @ Ymu
        sep = O.shifted_gram(sk, mu)
        assert np.linalg.norm(sep - direct) <= 1e-12 * np.linalg.norm(direct)
        # its Cholesky factor is the R of Y_mu = Q R (unique with a positive
        # diagonal), as the Householder QR of Y_mu gives it
        R = np.linalg.cholesky(sep).T
        _, Rh = O.householder_qr(Ymu)
        assert np.allclose(R, Rh, rtol=0, atol=1e-9 * np.abs(Rh).max())


def test_recycled_sketch_build_equals_fresh_build():
    """A build from the recycled A Omega (Sec. 5.1) equals a fresh build at
    the same shift with the same Omega: R, G, tau and the solution."""
    P = W.dense_power_spectrum(300, seed=82, power=2.0)
    op = O.DenseOp(P.A)
    sk = O.shift_sketch(op, 24, "gaussian", seed=82)
    B = W.gaussian_rhs(300, 2, 82)
    for mu in (1e-3, 0.2):
        fresh = O.build(op, mu, 24, "gaussian", seed=82, omega=sk.Omega)
        rec = O.build(op, mu, 24, "gaussian", seed=82, omega=sk.Omega, a_omega=sk.AOmega)
        assert np.allclose(rec.R, fresh.R, rtol=1e-12, atol=1e-12 * np.abs(fresh.R).max())
        assert np.allclose(rec.G, fresh.G, rtol=1e-10, atol=1e-10 * np.abs(fresh.G).max())
        assert rec.tau == pytest.approx(fresh.tau, rel=1e-10)
        x, info = O.solve(rec, B, rtol=1e-12)
        assert np.linalg.norm(x - O.exact_solve(op, mu, B)) <= 1e-8 * np.linalg.norm(x)


def test_joint_basis_qr_matches_direct_qr():
    """The joint basis of Sec. 5.1: Q_joint Q_red and R from qr(C1 + mu C2)
    are the unique (positive-diagonal) QR factors of A Omega + mu Omega
    computed directly, for several shifts including an ill-conditioned
    basis; dropping the mu C2 term (a plausible slip) fails at mu > 0."""
    P = W.dense_power_spectrum(300, seed=83, power=3.0)
    op = O.DenseOp(P.A)
    sk = O.shift_sketch(op, 24, "gaussian", seed=83)
    jb = O.joint_basis(sk)
    assert jb.Qj.shape == (300, 48) and jb.C1.shape == (48, 24) and jb.C2.shape == (48, 24)
    assert np.linalg.norm(jb.Qj.T @ jb.Qj - np.eye(48), 2) <= 1e-13
    for mu in (0.0, 1e-6, 1e-3, 0.4):
        Ymu = P.A @ sk.Omega + mu * sk.Omega
        Qh, Rh = O.householder_qr(Ymu)
        Q, R = O.joint_qr(jb, mu)
        scale = np.abs(Rh).max()
        assert np.allclose(R, Rh, rtol=0, atol=1e-11 * scale)
        # two backward-stable QRs: Q agrees to O(u cond(Y_mu))
        assert np.linalg.norm(Q - Qh, 2) <= 1e3 * 2.2e-16 * np.linalg.cond(Ymu)
        assert np.linalg.norm(Q @ R - Ymu) <= 1e-12 * np.linalg.norm(Ymu)
    bad = O.JointBasis(Qj=jb.Qj, C1=jb.C1, C2=np.zeros_like(jb.C2))
    _, Rb = O.joint_qr(bad, 0.4)
    _, Rh = O.householder_qr(P.A @ sk.Omega + 0.4 * sk.Omega)
    assert np.abs(Rb - Rh).max() > 1e-3 * np.abs(Rh).max()


# ------------------------------------------------------------ SRHT (Sec. 2)
def test_srht_subsampling_is_a_permutation():
    """The keyed Feistel permutation (with cycle-walking for odd log2 s) maps
    0..s-1 onto 0..s-1, so the k kept rows are distinct."""
    for s in (1, 2, 4, 8, 16, 32, 64, 256, 512, 2048):
        rows = philox.srht_rows(s, s, seed=17)
        assert np.array_equal(np.sort(rows), np.arange(s))
    assert philox.srht_size(20000) == 32768 and philox.srht_size(256) == 256


def test_srht_hadamard_entries_match_library():
    """H[r][i] = (-1)^popcount(r & i) is the Sylvester Walsh-Hadamard matrix
    of the library routine."""
    sp = pytest.importorskip("scipy.linalg")
    s = 64
    H = sp.hadamard(s)
    r = np.arange(s)[:, None]
    i = np.arange(s)[None, :]
    assert np.array_equal(np.where(np.bitwise_count(r & i) & 1, -1, 1), H)


def test_srht_columns_orthogonal_for_power_of_two():
    """With n = s the k columns of Omega are distinct rows of D H / sqrt(k)
    (H^T H = s I): Omega^T Omega = (s / k) I, off-diagonal entries exactly 0."""
    n, k = 256, 32
    Om = philox.srht_omega(n, k, seed=23)
    assert np.all(np.abs(Om) == 1.0 / math.sqrt(k))
    S = np.rint(Om * math.sqrt(k)).astype(np.int64)     # the +-1 pattern, exactly
    assert np.array_equal(S.T @ S, n * np.eye(k, dtype=np.int64))


def test_srht_build_solves():
    """An SRHT test matrix gives a working preconditioner: the PCG solution
    reaches the exact solution."""
    P = W.dense_power_spectrum(300, seed=84, power=2.0)
    op = O.DenseOp(P.A)
    B = W.gaussian_rhs(300, 1, 84)
    bd = O.build(op, 1e-4, 40, "srht", seed=84)
    x, info = O.solve(bd, B, rtol=1e-12)
    assert np.linalg.norm(x - O.exact_solve(op, 1e-4, B)) <= 1e-8 * np.linalg.norm(x)


# ------------------------------------------ multi-level embedding (Sec. 2 eq:multilevelose)
def test_multilevel_x1_is_a_sparse_random_operator():
    """X1 has exactly gamma1 nonzeros +-1/sqrt(gamma1) in each column, in
    distinct rows, so every column has unit norm (Sec. 2 definition of a
    sparse random operator); rows of X1 are hit about n gamma1 / l1 times."""
    n, k = 3000, 40
    l1, g1 = philox.multilevel_defaults(n, k)
    assert (l1, g1) == (9 * 40, 9)
    cols, sgn, X2T = philox.multilevel_parts(n, k, l1, g1, seed=31)
    X1 = philox.multilevel_x1(n, l1, g1, cols, sgn).toarray()
    assert X1.shape == (l1, n) and X2T.shape == (l1, k)
    assert np.all((X1 != 0).sum(axis=0) == g1)
    assert np.allclose(np.abs(X1[X1 != 0]), 1.0 / math.sqrt(g1), rtol=0, atol=1e-15)
    assert np.allclose((X1 * X1).sum(axis=0), 1.0, rtol=0, atol=1e-14)
    hits = (X1 != 0).sum(axis=1)
    assert abs(hits.mean() - n * g1 / l1) < 1e-9 and hits.min() > 0
    # the signs are balanced
    assert abs(np.mean(sgn)) < 0.05


def test_multilevel_omega_rows_are_signed_sums_of_x2_columns():
    """Row i of Omega = X1^T X2^T, taken the other way round: the signed sum
    of the gamma1 rows of X2^T that column i of X1 selects, and the dense
    product (X2 X1)^T."""
    n, k, l1, g1 = 500, 24, 120, 5
    Om = philox.multilevel_omega(n, k, seed=32, l1=l1, gamma1=g1)
    cols, sgn, X2T = philox.multilevel_parts(n, k, l1, g1, seed=32)
    for i in (0, 1, 77, 499):
        row = np.zeros(k)
        for t in range(g1):
            row += sgn[i, t] * X2T[cols[i, t]]
        assert np.allclose(Om[i], row / math.sqrt(g1), rtol=0, atol=1e-14)
    X1 = philox.multilevel_x1(n, l1, g1, cols, sgn).toarray()
    assert np.allclose(Om, (X2T.T @ X1).T, rtol=0, atol=1e-13)


def test_multilevel_embedding_is_isotropic_and_embeds_subspaces():
    """E[X^T X] = I_n (E[X2^T X2] = I_l1 and the columns of X1 have unit
    norm), so the mean squared row norm of Omega is 1; and X embeds a fixed
    d-dimensional subspace: the singular values of X U lie near 1."""
    n, k = 4000, 200
    Om = philox.multilevel_omega(n, k, seed=33)
    assert abs(np.mean(np.sum(Om * Om, axis=1)) - 1.0) < 0.02
    U, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((n, 4)))
    sv = np.linalg.svd(Om.T @ U, compute_uv=False)
    assert sv.min() > 0.7 and sv.max() < 1.3


def test_multilevel_build_solves_like_gaussian():
    """A multi-level test matrix gives a working preconditioner: PCG reaches
    the exact solution, in about the iterations of the Gaussian sketch of
    the same size (the range guarantees are alike)."""
    P = W.dense_power_spectrum(400, seed=85, power=2.0)
    op = O.DenseOp(P.A)
    B = W.gaussian_rhs(400, 1, 85)
    its = {}
    for sk in ("multilevel", "gaussian"):
        bd = O.build(op, 1e-4, 40, sk, seed=85)
        x, info = O.solve(bd, B, rtol=1e-12)
        assert np.linalg.norm(x - O.exact_solve(op, 1e-4, B)) <= 1e-8 * np.linalg.norm(x)
        its[sk] = info[0].inner_iters
    assert its["multilevel"] <= 1.5 * its["gaussian"] + 3


def test_multilevel_full_sketch_converges_in_one_iteration():
    # k = n: Omega square and nonsingular, Pi = I, P = tau A_mu^-1
    P, op = small_dense(n=40)
    bd = O.build(op, 1e-2, 40, "multilevel", seed=7)
    b = W.gaussian_rhs(40, 1, 7)[:, 0]
    x, info = O.solve(bd, b, rtol=1e-10, fixed_inner=1)
    assert O.true_rel_residual(op, 1e-2, x, b)[0] < 1e-9


# ------------------------------------------ refined projector (Sec. 4.3 eq:accurate_proj)
def _perturbed_basis(n, k, eps, seed):
    rng = np.random.default_rng(seed)
    Q0, _ = np.linalg.qr(rng.standard_normal((n, k)))
    F = rng.standard_normal((k, k))
    return Q0 @ (np.eye(k) + eps * F)        # a basis of range(Q0), |I - Q^T Q| ~ eps


def test_neumann_projector_error_is_second_order():
    """For a nearly orthonormal Q, Q Q^T is off the orthogonal projector onto
    range(Q) by O(|I - Q^T Q|) and Q T Q^T by O(|I - Q^T Q|^2) (the claim after
    eq:accurate_proj).  The exact projector comes from a Householder QR."""
    n, k = 300, 20
    errs = {}
    for eps in (1e-3, 1e-4):
        Q = _perturbed_basis(n, k, eps, seed=61)
        U, _ = np.linalg.qr(Q)
        Pex = U @ U.T
        plain = np.linalg.norm(Q @ Q.T - Pex, 2)
        refined = np.linalg.norm(Q @ O.neumann_T(Q) @ Q.T - Pex, 2)
        errs[eps] = (plain, refined)
        d = np.linalg.norm(np.eye(k) - Q.T @ Q, 2)
        assert 0.3 * d <= plain <= 1.5 * d
        assert refined <= 2.0 * d * d
    # first order vs second order in eps
    assert 5 < errs[1e-3][0] / errs[1e-4][0] < 20
    assert 50 < errs[1e-3][1] / errs[1e-4][1] < 200


def test_neumann_T_is_two_refinement_steps():
    """eq:accurate_proj_2: v_1 = Q^T u, v_(i+1) = v_i + Q^T (u - Q v_i).  Two
    steps give T Q^T u exactly; many steps reach the least-squares solution
    Q^+ u of the library solver."""
    Q = _perturbed_basis(200, 12, 1e-2, seed=62)
    u = np.random.default_rng(63).standard_normal(200)
    v = Q.T @ u
    v2 = v + Q.T @ (u - Q @ v)
    assert np.allclose(v2, O.neumann_T(Q) @ (Q.T @ u), rtol=0, atol=1e-13)
    for _ in range(60):
        v = v + Q.T @ (u - Q @ v)
    assert np.allclose(v, np.linalg.lstsq(Q, u, rcond=None)[0], rtol=0, atol=1e-12)


def test_refined_build_equals_plain_for_orthonormal_basis_and_solves():
    """With the Householder basis (orthonormal to rounding) T = I to rounding:
    the refined preconditioner equals the plain one, and the solve is exact."""
    P, op = small_dense(n=200)
    mu, k = 1e-4, 24
    plain = O.build(op, mu, k, "gaussian", seed=64)
    ref = O.build(op, mu, k, "gaussian", seed=64, refine=True)
    assert np.linalg.norm(ref.Tref - np.eye(k)) <= 1e-13
    V = np.random.default_rng(65).standard_normal((200, 3))
    assert np.allclose(ref.apply_P(V), plain.apply_P(V), rtol=0, atol=1e-10 * np.abs(plain.apply_P(V)).max())
    b = W.gaussian_rhs(200, 1, 64)
    x, info = O.solve(ref, b, rtol=1e-12)
    assert np.linalg.norm(x - O.exact_solve(op, mu, b)) <= 1e-8 * np.linalg.norm(x)
    with pytest.raises(ValueError):
        O.build(op, mu, k, "gaussian", seed=64, variant="R", refine=True)


def test_refined_preconditioner_restores_the_spectrum():
    """Exact eigenvector deflation with a non-orthonormal basis of the same
    range: the plain P = I + Q (tau G - I) Q^T loses the closed-form spectrum
    {tau (k times), lambda_i + mu (i > k)} of P A_mu at first order in
    |I - Q^T Q|, the refined one at second order."""
    P, op = small_dense(n=120)
    mu, k = 1e-3, 10
    good = O.build(op, mu, k, omega=P.U[:, :k])
    expect = np.sort(np.concatenate([np.full(k, good.tau), P.lam[k:] + mu]))
    Amu = P.A + mu * np.eye(op.n)
    rng = np.random.default_rng(66)
    Mp = np.eye(k) + 1e-4 * rng.standard_normal((k, k))
    Qp = good.Q @ Mp
    # the core matrix of that basis, G = Q^T A_mu^-1 Q (what the build forms
    # from its own Q = A_mu Omega R^-1), here from the dense inverse
    Gp = Qp.T @ np.linalg.solve(Amu, Qp)
    dev_ = {}
    for name, Tref in (("plain", None), ("refined", O.neumann_T(Qp))):
        bd = O.Build(op=op, mu=mu, k=k, variant="C", Omega=good.Omega, Ymu=good.Ymu, Q=Qp,
                     R=np.linalg.solve(Mp, good.R), G=Gp, normE=good.normE,
                     lam_max=good.lam_max, tau=good.tau, rho=good.rho, Tref=Tref)
        ev = np.sort(np.linalg.eigvals(bd.apply_P(np.eye(op.n)) @ Amu).real)
        dev_[name] = np.max(np.abs(ev - expect) / expect)
    assert dev_["plain"] > 1e-6
    assert dev_["refined"] < 1e-2 * dev_["plain"]


# ------------------------------------------ G-RandRAND and MINRES (Sec. 3.3, 6.3)
def _indefinite(n=200, seed=86, after=20):
    P = W.dense_power_spectrum(n, seed=seed, power=2.0)
    ev = np.sort(np.linalg.eigvalsh(P.A))[::-1]
    mu = -0.5 * (ev[after] + ev[after + 1])      # a shift between two eigenvalues
    return P.A, mu


def test_minres_matches_library_minres():
    """The oracle's preconditioned MINRES takes the library routine's iterates
    (same Krylov method, same SPD preconditioner) on an indefinite system."""
    spl = pytest.importorskip("scipy.sparse.linalg")
    A, mu = _indefinite()
    n = A.shape[0]
    Amu = A + mu * np.eye(n)
    rng = np.random.default_rng(3)
    Mh = rng.standard_normal((n, n))
    Pm = np.eye(n) + 0.1 * Mh @ Mh.T / n        # an SPD preconditioner
    b = rng.standard_normal(n)
    # iterates to rounding over the first steps; later the Lanczos recurrences
    # of the two formulations drift apart by rounding on this ill-conditioned
    # system, so the residual norms are compared there
    for m in (1, 2, 3, 12):
        x, it = O.minres(lambda v: Amu @ v, b, lambda v: Pm @ v, 0.0, m)
        assert it == m
        xs, _ = spl.minres(Amu, b, M=spl.aslinearoperator(Pm), maxiter=m, rtol=1e-300)
        if m <= 3:
            assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)
        else:
            r, rs = np.linalg.norm(b - Amu @ x), np.linalg.norm(b - Amu @ xs)
            assert abs(r - rs) <= 1e-6 * rs


def test_g_randrand_core_and_eigenvalue_bounds():
    """G^2 = R^-T Omega^T Omega R^-1; P is SPD although A_mu is indefinite; with
    tau from eq:g_randrand_tau on the exact norms, the singular values of P A_mu
    obey eq:c_randrand_eigenvalues2."""
    A, mu = _indefinite()
    n = A.shape[0]
    op = O.DenseOp(A)
    Amu = A + mu * np.eye(n)
    assert np.linalg.eigvalsh(Amu).min() < 0 < np.linalg.eigvalsh(Amu).max()
    bd = O.build(op, mu, 40, "gaussian", seed=86, variant="G", q=1)
    Ri = np.linalg.inv(bd.R)
    MG = Ri.T @ (bd.Omega.T @ bd.Omega) @ Ri
    assert np.linalg.norm(bd.G @ bd.G - MG) <= 1e-10 * np.linalg.norm(MG)
    I = np.eye(n)
    Pi = bd.Q @ bd.Q.T
    Pt = bd.Q @ bd.G @ bd.Q.T
    n1 = np.linalg.norm((I - Pi) @ Amu, 2)
    n2 = np.linalg.norm(Pt @ Amu, 2)
    rho = 0.5
    tau = math.sqrt(rho) * n1 / n2
    bt = O.build(op, mu, 40, "gaussian", seed=86, variant="G", q=1, tau=tau)
    Pm = bt.apply_P(I)
    assert np.allclose(Pm, Pm.T, atol=1e-12)
    assert np.linalg.eigvalsh(0.5 * (Pm + Pm.T)).min() > 0.0
    s = np.linalg.svd(Pm @ Amu, compute_uv=False)
    lo = 1.0 / (np.linalg.norm((I - Pi) @ np.linalg.inv(Amu), 2) ** 2 + tau ** -2)
    assert s.min() ** 2 >= lo * (1 - 1e-8)
    assert s.max() ** 2 <= (1 + rho) * n1 ** 2 * (1 + 1e-8)


def test_g_randrand_minres_solves_indefinite():
    """Restarted MINRES with the G-RandRAND preconditioner (q = 1) reaches the
    exact solution of an indefinite system, in fewer iterations than plain
    MINRES."""
    A, mu = _indefinite(n=300, seed=87)
    op = O.DenseOp(A)
    B = W.gaussian_rhs(300, 2, 87)
    bd = O.build(op, mu, 60, "gaussian", seed=87, variant="G", q=1)
    x, infos = O.solve(bd, B, rtol=1e-10)
    xs = np.linalg.solve(A + mu * np.eye(300), B)
    assert np.linalg.norm(x - xs) <= 1e-7 * np.linalg.norm(xs)
    _, plain = O.minres(lambda v: A @ v + mu * v, B[:, 0], lambda v: v, 1e-10, 5000)
    assert infos[0].inner_iters < plain


# --------------------------------------------------------------------------
# Core-matrix jitter ladder (App. C): alpha = the smallest of 10^-14 |M|,
# ..., 10^-1 |M| for which M + alpha I factors, |M| the spectral norm
# --------------------------------------------------------------------------
def test_jitter_ladder_matches_brute_force_scan():
    from ladder_cases import ladder_core, ladder_rung
    k = 40
    M = ladder_core(k)
    ev = np.linalg.eigvalsh(M)
    nrm2 = np.abs(ev).max()
    assert nrm2 == pytest.approx(np.linalg.svd(M, compute_uv=False)[0], rel=1e-12)
    expected = ladder_rung(M, nrm2)
    # the fixture decides every rung far from rounding: the rung below fails
    # and the chosen one succeeds by margins well above k u |M|
    assert expected is not None and expected > 0
    margin = 1e4 * k * np.finfo(float).eps * nrm2
    assert ev.min() + expected > margin
    assert ev.min() + expected / 10 < -margin
    RM, alpha = O.chol_upper_jitter(M)
    assert alpha == pytest.approx(expected, rel=1e-12)
    assert np.allclose(RM.T @ RM, M + alpha * np.eye(k), rtol=0, atol=1e-13 * nrm2)
    assert np.all(np.diag(RM) > 0) and np.allclose(RM, np.triu(RM))
    # the largest-diagonal reading of |M| lands on another rung here, so a
    # ladder scaled by that reading fails this test
    alt = ladder_rung(M, np.abs(np.diag(M)).max())
    assert alt is not None and not np.isclose(alt, expected, rtol=0.5)
    # an SPD matrix factors without jitter; one far from SPD exhausts the ladder
    _, a0 = O.chol_upper_jitter(M + 1e-6 * nrm2 * np.eye(k))
    assert a0 == 0.0
    with pytest.raises(np.linalg.LinAlgError):
        O.chol_upper_jitter(M - 0.5 * nrm2 * np.eye(k))


def test_build_takes_the_jitter_ladder_for_an_indefinite_core():
    """A dense A with Omega^T A_mu Omega = M (one slightly negative eigenvalue)
    sends the C build through the ladder: G = R^-T (M + alpha I) R^-1 with the
    brute-force alpha, and A_mu Omega = Q R stays well conditioned."""
    from ladder_cases import ladder_core, ladder_rung, operator_with_core
    n, k, mu, seed = 400, 40, 1e-3, 21
    Om = O.make_omega(n, k, "sparse_sign", seed, gamma=8)
    M = ladder_core(k)
    A = operator_with_core(Om, M, mu)
    assert np.allclose(A, A.T)
    assert np.allclose(Om.T @ (A + mu * np.eye(n)) @ Om, M, rtol=0, atol=1e-11)
    b = O.build(O.DenseOp(A), mu, k, "sparse_sign", seed, gamma=8)
    assert np.linalg.cond(b.Ymu) < 1e4
    expected = ladder_rung(M, np.abs(np.linalg.eigvalsh(M)).max())
    assert b.jitter == pytest.approx(expected, rel=1e-9)
    Rinv = np.linalg.inv(b.R)
    G_def = Rinv.T @ (M + b.jitter * np.eye(k)) @ Rinv
    assert np.allclose(b.G, G_def, rtol=0, atol=1e-10 * np.abs(G_def).max())


def test_projector_refinement_recurrence_converges_to_pseudoinverse():
    """eq:accurate_proj_2: v_1 = Q^T u, v_{i+1} = v_i + Q^T (u - Q v_i) is the
    Neumann series of (Q^T Q)^-1 applied to Q^T u: for a nearly orthonormal Q
    its error against the least-squares Q^+ u (library lstsq) falls like
    |I - Q^T Q|^s, its first refinement equals the Neumann T = 2 I - Q^T Q of
    eq:accurate_proj, and the refined P keeps the spectrum that exact
    eigenvector deflation fixes."""
    rng = np.random.default_rng(31)
    n, k = 300, 25
    Q0, _ = np.linalg.qr(rng.standard_normal((n, k)))
    Q = Q0 + 1e-3 * rng.standard_normal((n, k))            # |I - Q^T Q| ~ 1e-2
    eps = np.linalg.norm(np.eye(k) - Q.T @ Q, 2)
    u = rng.standard_normal((n, 2))
    vstar = np.linalg.lstsq(Q, u, rcond=None)[0]
    b = O.Build(op=None, mu=0.0, k=k, variant="C", Omega=None, Ymu=None, Q=Q, R=np.eye(k),
                G=np.eye(k), normE=1.0, lam_max=1.0, tau=1.0, rho=1.0)
    errs = []
    for s in range(0, 5):
        b.refine_steps = s
        v = b.refined_coeffs(u)
        errs.append(np.linalg.norm(v - vstar) / np.linalg.norm(vstar))
        if s == 1:
            assert np.allclose(v, O.neumann_T(Q) @ (Q.T @ u), rtol=0, atol=1e-13)
    for s in range(1, 5):
        assert errs[s] <= 3 * eps ** (s + 1)
        assert errs[s] < errs[s - 1]
    # the left refinement is the same polynomial in Q^T Q on a k-vector
    w = rng.standard_normal((k, 2))
    b.refine_steps = 3
    E = np.eye(k) - Q.T @ Q
    Tpoly = np.eye(k) + E + E @ E + E @ E @ E
    assert np.allclose(b.refined_left(w), Tpoly @ w, rtol=0, atol=1e-12)
    assert np.allclose(b.refined_coeffs(u), Tpoly @ (Q.T @ u), rtol=0, atol=1e-12)


def test_refined_recurrence_build_solves_and_is_symmetric():
    """A build with the eq:accurate_proj_2 refinement (3 steps beyond the
    first) gives a symmetric P (checked on the dense matrix of the operator)
    and solves to the dense Cholesky solution."""
    P_, op = small_dense(n=200, seed=13)
    mu, k = 1e-3, 30
    bd = O.build(op, mu, k, "gaussian", seed=13, refine=3)
    assert bd.refine_steps == 3
    Pm = bd.apply_P(np.eye(200))
    assert np.allclose(Pm, Pm.T, rtol=0, atol=1e-12 * np.abs(Pm).max())
    B = W.gaussian_rhs(200, 2, 13)
    X, infos = O.solve(bd, B, rtol=1e-12)
    xs = np.linalg.solve(op.dense() + mu * np.eye(200), B)
    assert np.linalg.norm(X - xs) / np.linalg.norm(xs) <= 1e-9


# ------------------------------------------------- Sec. 5.2 Newton sketch
def _newton_problem(n=600, k=20, seed=91):
    rng = np.random.default_rng(seed)
    # A_mu Omega with spread column scales (cond ~ 1e3), a generic right side
    U, _ = np.linalg.qr(rng.standard_normal((n, k)))
    V, _ = np.linalg.qr(rng.standard_normal((k, k)))
    Y = U @ np.diag(np.logspace(0, -3, k)) @ V.T
    u = rng.standard_normal(n)
    return Y, u


def test_newton_sketch_exact_sketch_solves_in_one_step():
    """With Theta = I (S = Y) D is the normal matrix Y^T Y: the first step of
    eq:iterative_refinement from v = 0 is the least-squares solution."""
    Y, u = _newton_problem()
    v, info = O.newton_sketch_lstsq(Y, Y, u, steps=1)
    ref = np.linalg.lstsq(Y, u, rcond=None)[0]
    assert np.linalg.norm(v - ref) <= 1e-9 * np.linalg.norm(ref)
    assert info.rel_normal_residual[0] <= 1e-9


def test_newton_sketch_contracts_by_the_spectrum_of_d_inverse_normal_matrix():
    """The error e_t = v_t - v* obeys e_{t+1} = (I - D^-1 Y^T Y) e_t, so its
    Y^T Y-energy norm contracts each step by at most rho = max |1 - lambda|
    over the eigenvalues of D^-1 Y^T Y; with a sparse-sign Theta of l_sk =
    16 k rows (an epsilon-embedding) rho < 1 and the iteration reaches the
    least-squares solution geometrically (O(log 1/u) steps)."""
    Y, u = _newton_problem()
    n, k = Y.shape
    Th = philox.theta_dense(16 * k, n, 8, 92)
    S = Th @ Y
    lam = np.linalg.eigvals(np.linalg.solve(S.T @ S, Y.T @ Y)).real
    rho = float(np.max(np.abs(1.0 - lam)))
    assert rho < 1.0
    ref = np.linalg.lstsq(Y, u, rcond=None)[0]
    A = Y.T @ Y
    enorm = lambda e: float(np.sqrt(e @ A @ e))
    steps = int(math.ceil(math.log(1e-11) / math.log(rho)))   # O(log 1/u) steps
    assert steps <= 80
    v, info = O.newton_sketch_lstsq(Y, S, u, steps=steps)
    for t in (1, 2, 5, steps // 2):
        vt, _ = O.newton_sketch_lstsq(Y, S, u, steps=t)
        assert enorm(vt - ref) <= rho ** t * enorm(ref) * (1 + 1e-6) + 1e-12 * enorm(ref)
    assert enorm(v - ref) <= 1e-10 * enorm(ref)


def test_newton_sketch_with_inner_cg_matches_exact_inner_solve():
    """D^-1 by CG on D (matvec S^T S x) to 1e-13 gives the same iterates as a
    direct solve, and its iteration count grows like sqrt(cond(D))."""
    Y, u = _newton_problem()
    n, k = Y.shape
    S = philox.theta_dense(16 * k, n, 8, 93) @ Y
    v1, _ = O.newton_sketch_lstsq(Y, S, u, steps=8)
    v2, info = O.newton_sketch_lstsq(Y, S, u, steps=8, inner_tol=1e-13)
    assert np.linalg.norm(v2 - v1) <= 1e-8 * np.linalg.norm(v1)
    cond = np.linalg.cond(S.T @ S)
    assert all(0 < it <= 4 * np.sqrt(cond) * math.log(2e13) for it in info.inner_iters)


def test_cg_spd_is_exact_in_n_steps_on_small_systems():
    rng = np.random.default_rng(94)
    B = rng.standard_normal((12, 12))
    D = B @ B.T + 12 * np.eye(12)
    rhs = rng.standard_normal(12)
    x, it = O.cg_spd(lambda z: D @ z, rhs, 1e-14, 100)
    assert it <= 14
    assert np.linalg.norm(D @ x - rhs) <= 1e-12 * np.linalg.norm(rhs)
