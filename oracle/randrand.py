"""ORACLE (test infrastructure only) -- plain FP64 RandRAND on the CPU.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA
library: it is a slow, direct transcription of the method in float64 numpy,
written so that each step can be checked against the paper by eye.

What it computes (paper: Balabanov, Derezinski, Mahoney et al., "RandRAND",
arXiv 2509.19747):

* the shifted system (A + mu I) x = b, A symmetric PSD (Sec. 1, eq:initsys);
* the test matrix Omega = A^q X^T (eq:testmatrix), X Gaussian, sparse sign,
  SRHT or the multi-level embedding X2 X1 (Sec. 2), drawn by ``oracle.philox``;
* the basis Y_mu = A_mu Omega and its orthogonalisation A_mu Omega = Q R
  (Sec. 4.1 eq:Rdef) by Householder QR (library ``numpy.linalg.qr``), or
  the randomised Q-less preconditioned Cholesky QR (Sec. 4.2, Alg. 3);
* the projector Pi u = Q Q^T u and A_mu^-1 Pi u = Omega R^-1 Q^T u
  (Sec. 4.1 eq:projector; Sec. 1.1 eq:invAPi);
* C-RandRAND: P = I - Q Q^T + tau Q G Q^T with G = R^-T (Omega^T A_mu Omega)
  R^-1 (Sec. 4.1 eq:g_randrand_explicit) in the SPD-preserving form
  G = (R_M R^-1)^T (R_M R^-1), R_M^T R_M = Omega^T A_mu Omega (remark after
  Alg. 7); tau = rho |E| / lambda_max(Pi A_mu Pi~) (Sec. 3.2
  eq:c_randrand_tau) with rho from eq:optimal_rho, F = 1/mu;
* R-RandRAND: CG on B y = r, B = (I - Pi) A_mu (I - Pi) + tau Pi (Sec. 3.1
  eq:APdef2), recovery x = Omega R^-1 Q^T (tau y - A_mu (I - Pi) y) +
  (I - Pi) y (eq:APdef3), tau = |E| (Alg. 4 step 2);
* |E| and lambda_max by power iterations (Alg. 4 step 2, Alg. 7 step 3);
* PCG / CG with restarts after each residual reduction by eta = 1e-2
  (Sec. 7 experimental setup; Alg. 4 step 9, Alg. 7 step 10), the restart
  residual b - A_mu x recomputed in float64;
* the exact solution x* = A_mu^-1 b by a dense Cholesky solve;
* G-RandRAND (Sec. 3.3 eq:g_randrand): P = (I - Pi) + tau Q G Q^T with
  G = (R^-T Omega^T Omega R^-1)^(1/2), tau = rho^(1/2) |(I - Pi) A_mu| /
  |Pi~ A_mu| (eq:g_randrand_tau, the Sec. 6.3 estimates), and restarted
  preconditioned MINRES (Paige and Saunders), also for indefinite A_mu
  (mu < 0);
* the refined projector of eq:accurate_proj: Pi ~ Q T Q^T with the Neumann
  T = 2 I - Q^T Q, and Pi A_mu^-1 Pi ~ Q T G T Q^T (the symmetric reading of
  the re-orthogonalized C-RandRAND, eq:c_randrand_reorth);
* the factorization-free least-squares solve of Sec. 5.2
  (eq:iterative_refinement): v <- v + D^-1 (A_mu Omega)^T (u - A_mu Omega v),
  D = (Theta A_mu Omega)^T (Theta A_mu Omega), D^-1 by a library solve or by
  CG on D (used to measure that form against the factored build; the library
  factors R);
* several shifts from one sketch (Sec. 5.1): A Omega computed once, Y_mu =
  A Omega + mu Omega per shift, and the Gram separation (A Omega + mu
  Omega)^T (A Omega + mu Omega) = Omega^T A^T A Omega + 2 mu Omega^T A Omega
  + mu^2 Omega^T Omega of the parameter-free projections; and the joint basis
  (Sec. 5.1): Q_joint from qr([Omega, A Omega]), C1 = Q_joint^T A Omega,
  C2 = Q_joint^T Omega, then per shift qr(C1 + mu C2) = Q_red R and
  Q = Q_joint Q_red.

Readings where the paper is silent: for G-RandRAND rho = 0.5 a priori (the
optimal rho of eq:rho_g_rand_rand needs |A_mu^-1|), the norms as square
roots of power-iteration estimates of the largest eigenvalues of A_mu (I -
Pi) A_mu and A_mu Pi~^2 A_mu, and the MINRES inner stop as the same
relative reduction of |r|_P = sqrt(r^T P r), the norm MINRES tracks.  Also:
20 power iterations from seeded start
vectors, estimate = |w_20| (norm of the last image of a unit vector); the
inner stop max(eta |r_0|, 0.5 rtol |b|); R = R_chol R_sk as the product
order in Alg. 3 (the only order with R^T R = Y_mu^T Y_mu); l_sk = 4k and
gamma_sk = 8 for Theta.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import philox

VARIANT_C = "C"
VARIANT_R = "R"
VARIANT_G = "G"
MAX_RESTARTS = 400      # restarts per column, as in the library


# ==========================================================================
# Operators: u -> A u (Sec. 1: access to A through matvecs only)
# ==========================================================================
class DenseOp:
    def __init__(self, A: np.ndarray):
        self.A = np.asarray(A, dtype=np.float64)
        self.n = self.A.shape[0]

    def matmat(self, V: np.ndarray) -> np.ndarray:
        return self.A @ V

    def dense(self) -> np.ndarray:
        return self.A


class CsrOp:
    def __init__(self, rowptr, colidx, vals, n: int):
        import scipy.sparse as sp
        self.n = int(n)
        self.M = sp.csr_matrix((np.asarray(vals, dtype=np.float64),
                                np.asarray(colidx), np.asarray(rowptr)), shape=(n, n))

    def matmat(self, V: np.ndarray) -> np.ndarray:
        return self.M @ V

    def dense(self) -> np.ndarray:
        return self.M.toarray()


class GaussKernelOp:
    """K_ij = exp(-|x_i - x_j|^2 / (2 h^2)) evaluated in float64 from the
    given (float32) coordinates, never stored whole (Sec. 7.2.2 eq:kernel,
    with the kernel matrix itself as A)."""

    def __init__(self, points: np.ndarray, bandwidth: float = 1.0, block: int = 2048,
                 materialize: bool = False):
        self.X = np.asarray(points, dtype=np.float64)
        self.n = self.X.shape[0]
        self.h = float(bandwidth)
        self.block = block
        # materialize=True keeps the dense K (n^2 float64) so that repeated
        # products are plain matrix products; same values as the blockwise path
        self.K = self.rows(0, self.n) if materialize else None

    def rows(self, lo: int, hi: int) -> np.ndarray:
        diff2 = ((self.X[lo:hi, None, :] - self.X[None, :, :]) ** 2).sum(-1) \
            if (hi - lo) * self.n * self.X.shape[1] <= 4_000_000 else None
        if diff2 is None:
            xi = self.X[lo:hi]
            diff2 = np.zeros((hi - lo, self.n))
            for c in range(self.X.shape[1]):
                diff2 += (xi[:, c:c + 1] - self.X[None, :, c]) ** 2
        return np.exp(-diff2 / (2.0 * self.h * self.h))

    def matmat(self, V: np.ndarray) -> np.ndarray:
        V = np.asarray(V, dtype=np.float64)
        if self.K is not None:
            return self.K @ V
        out = np.empty((self.n,) + V.shape[1:])
        for lo in range(0, self.n, self.block):
            hi = min(self.n, lo + self.block)
            out[lo:hi] = self.rows(lo, hi) @ V
        return out

    def dense(self) -> np.ndarray:
        return self.K if self.K is not None else self.rows(0, self.n)


def shifted(op, mu: float):
    """u -> A_mu u = A u + mu u (Sec. 1)."""
    return lambda V: op.matmat(V) + mu * V


# ==========================================================================
# Small helpers
# ==========================================================================
def householder_qr(Y: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Economic QR with diag(R) > 0 (makes Q, R unique for full column rank)."""
    Q, R = np.linalg.qr(Y)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s, R * s[:, None]


def chol_upper(M: np.ndarray) -> np.ndarray:
    """Upper-triangular R with R^T R = M (raises LinAlgError if not SPD)."""
    return np.linalg.cholesky(M).T


def chol_upper_jitter(M: np.ndarray) -> tuple[np.ndarray, float]:
    """Cholesky with the jitter ladder of App. C: on failure add alpha I with
    alpha the smallest of 1e-14 |M|, ..., 1e-1 |M| that succeeds."""
    try:
        return chol_upper(M), 0.0
    except np.linalg.LinAlgError:
        pass
    nrm = np.linalg.norm(M, 2)
    for e in range(-14, 0):
        alpha = 10.0 ** e * nrm
        try:
            return chol_upper(M + alpha * np.eye(M.shape[0])), alpha
        except np.linalg.LinAlgError:
            continue
    raise np.linalg.LinAlgError("matrix not SPD even with the jitter ladder")


def solve_upper(R: np.ndarray, B: np.ndarray) -> np.ndarray:
    import scipy.linalg as sl
    return sl.solve_triangular(R, B, lower=False)


def right_solve_upper(Y: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Y R^-1 for upper-triangular R."""
    import scipy.linalg as sl
    return sl.solve_triangular(R, Y.T, trans="T", lower=False).T


# ==========================================================================
# Build: Alg. 7 steps 1-4 (C) / Alg. 4 steps 1-2 (R)
# ==========================================================================
@dataclasses.dataclass
class Build:
    op: object
    mu: float
    k: int
    variant: str
    Omega: np.ndarray        # n x k test matrix
    Ymu: np.ndarray          # A_mu Omega
    Q: np.ndarray            # orthonormal basis of range(A_mu Omega)
    R: np.ndarray            # A_mu Omega = Q R
    G: np.ndarray | None     # C-RandRAND core matrix
    normE: float
    lam_max: float
    tau: float
    rho: float
    jitter: float = 0.0
    Tref: np.ndarray | None = None   # refined projector, eq:accurate_proj (refine=True)
    refine_steps: int = 0            # eq:accurate_proj_2: refinement steps beyond the first

    # --- projector and preconditioner applications (Sec. 4.1 eq:projector)
    def Pi(self, V):
        return self.Q @ (self.Q.T @ V)

    def Ainv_Pi(self, V):
        """A_mu^-1 Pi V = Omega R^-1 Q^T V (eq:projector with eq:invAPi)."""
        return self.Omega @ solve_upper(self.R, self.Q.T @ V)

    def refined_coeffs(self, V):
        """eq:accurate_proj_2: T(u, Q^T u) = v_s, v_1 = Q^T u,
        v_{i+1} = v_i + Q^T (u - Q v_i), s = 1 + refine_steps."""
        v = self.Q.T @ V
        for _ in range(self.refine_steps):
            v = v + self.Q.T @ (V - self.Q @ v)
        return v

    def refined_left(self, W):
        """The same refinement for the outer projector of Pi A_mu^-1 Pi, whose
        argument y = A_mu^-1 Pi u enters the recurrence only through
        Q^T y = G c (a k-vector w): y_1 = w, y_{i+1} = y_i + w - Q^T (Q y_i)."""
        y = W
        for _ in range(self.refine_steps):
            y = y + W - self.Q.T @ (self.Q @ y)
        return y

    def apply_P(self, V):
        """C-RandRAND: P V = V - Q Q^T V + tau Q G Q^T V (eq:g_randrand_explicit).
        With the refined projector (eq:accurate_proj) Pi is replaced by
        Q T Q^T and Pi A_mu^-1 Pi by Q T G T Q^T, T = 2 I - Q^T Q; with
        refine_steps >= 2 (eq:accurate_proj_2) the coefficients come from the
        refinement recurrence on each vector."""
        if self.refine_steps >= 2:
            c = self.refined_coeffs(V)
            return V - self.Q @ c + self.tau * (self.Q @ self.refined_left(self.G @ c))
        t = self.Q.T @ V
        if self.Tref is not None:
            Tt = self.Tref @ t
            return V - self.Q @ Tt + self.tau * (self.Q @ (self.Tref @ (self.G @ Tt)))
        return V - self.Q @ t + self.tau * (self.Q @ (self.G @ t))

    def apply_B(self, V):
        """R-RandRAND operator B = (I - Pi) A_mu (I - Pi) + tau Pi (eq:APdef2)."""
        Amu = shifted(self.op, self.mu)
        U = V - self.Pi(V)
        W = Amu(U)
        return W - self.Pi(W) + self.tau * self.Pi(V)

    def recover_R(self, Yv):
        """x = Omega R^-1 Q^T (tau y - A_mu (I - Pi) y) + (I - Pi) y (eq:APdef3)."""
        Amu = shifted(self.op, self.mu)
        U = Yv - self.Pi(Yv)
        return self.Ainv_Pi(self.tau * Yv - Amu(U)) + U


def make_omega(n: int, k: int, sketch: str, seed: int, gamma: int = 8,
               precision: str = "fp64", q: int = 0, op=None, ml_l1: int = 0,
               ml_gamma: int = 0) -> np.ndarray:
    """Test matrix Omega = A^q X^T (eq:testmatrix, A symmetric), rounded to the
    working precision of the sketch (float64, float32 or bfloat16).  X^T is
    the Gaussian or sparse-sign draw; with q >= 1 it is multiplied by A (not
    A_mu: Omega does not depend on the shift) q times before the rounding.
    X^T may also be an SRHT (Sec. 2, fast randomized transforms) or the
    multi-level embedding X = X2 X1 of eq:multilevelose (sparse X1 with
    ml_l1 rows and ml_gamma nonzeros per column, Gaussian X2), whose float64
    product is rounded once."""
    if sketch == "gaussian":
        Om = philox.gaussian_omega(n, k, seed)
    elif sketch == "sparse_sign":
        Om = philox.sparse_sign_omega_dense(n, k, gamma, seed)
    elif sketch == "srht":
        Om = philox.srht_omega(n, k, seed)
    elif sketch == "multilevel":
        Om = philox.multilevel_omega(n, k, seed, ml_l1, ml_gamma)
    else:
        raise ValueError(sketch)
    if q > 0:
        if precision == "bf16":
            Om = philox.round_bf16(Om)
        elif precision == "fp32":
            Om = philox.round_f32(Om)
        for _ in range(q):
            Om = op.matmat(Om)
    if precision == "bf16":
        Om = philox.round_bf16(Om)
    elif precision == "fp32":
        Om = philox.round_f32(Om)
    return Om


def power_iteration(apply, v0: np.ndarray, iters: int) -> float:
    """|w_iters| where v_0 = v0/|v0|, w_i = apply(v_{i-1}), v_i = w_i/|w_i|."""
    v = v0 / np.linalg.norm(v0)
    lam = 0.0
    for _ in range(iters):
        w = apply(v)
        lam = float(np.linalg.norm(w))
        if lam == 0.0:
            return 0.0
        v = w / lam
    return lam


def orthogonalize_householder(Ymu):
    return householder_qr(Ymu)


def fast_q_less_precond_chol_qr(Ymu: np.ndarray, Theta: np.ndarray) -> np.ndarray:
    """Alg. 3: S = Theta A_mu Omega; R_sk = qr(S); G = R_sk^-T Y^T Y R_sk^-1
    formed as W^T W with W = Y R_sk^-1; R_chol = chol(G); R = R_chol R_sk."""
    S = Theta @ Ymu
    _, Rsk = householder_qr(S)
    W = right_solve_upper(Ymu, Rsk)
    Rchol = chol_upper(W.T @ W)
    return Rchol @ Rsk


def build(op, mu: float, k: int, sketch: str = "gaussian", seed: int = 0,
          variant: str = VARIANT_C, omega: np.ndarray | None = None,
          omega_precision: str = "fp64", orth: str = "householder",
          gamma: int = 8, l_sk: int | None = None, gamma_sk: int = 8,
          power_iters: int = 20, rho: float | None = None,
          tau: float | None = None, q: int = 0,
          a_omega: np.ndarray | None = None, ml_l1: int = 0, ml_gamma: int = 0,
          refine: int = 0) -> Build:
    """a_omega: A Omega computed once for several shifts (Sec. 5.1): then
    omega must be the Omega it was computed from, and Y_mu = a_omega + mu
    Omega replaces the product.  refine (variants C and G): 1 (or True) the
    Neumann-refined projector of eq:accurate_proj; s >= 2 the refinement
    recurrence of eq:accurate_proj_2 with s steps beyond the first."""
    n = op.n
    if not (1 <= k <= n):
        raise ValueError("need 1 <= k <= n")
    if omega is None:
        Om = make_omega(n, k, sketch, seed, gamma, omega_precision, q=q, op=op, ml_l1=ml_l1,
                        ml_gamma=ml_gamma)
    else:
        # a given X^T: Omega = A^q X^T (eq:testmatrix)
        Om = np.asarray(omega, dtype=np.float64)
        for _ in range(q):
            Om = op.matmat(Om)
    # Alg. 7 step 1 / Alg. 4 step 1: Y_mu = A Omega + mu Omega (A Omega
    # recycled across shifts when given, Sec. 5.1)
    if a_omega is not None:
        if omega is None:
            raise ValueError("a_omega needs the omega it was computed from")
        Ymu = np.asarray(a_omega, dtype=np.float64) + mu * Om
    else:
        Ymu = op.matmat(Om) + mu * Om
    if orth == "householder":
        Q, R = orthogonalize_householder(Ymu)
    elif orth == "qless":
        Theta = philox.theta_dense(l_sk or 4 * k, n, gamma_sk, seed)
        R = fast_q_less_precond_chol_qr(Ymu, Theta)
        Q = right_solve_upper(Ymu, R)       # Q u = A_mu Omega R^-1 u (eq:implicit)
    else:
        raise ValueError(orth)

    b = Build(op=op, mu=mu, k=k, variant=variant, Omega=Om, Ymu=Ymu, Q=Q, R=R,
              G=None, normE=0.0, lam_max=0.0, tau=0.0, rho=0.0)
    Amu = shifted(op, mu)

    # |E|, E = (I - Pi) A_mu (I - Pi): Alg. 4 step 2 / Alg. 7 step 3
    def E_apply(v):
        u = v - b.Pi(v)
        w = Amu(u)
        return w - b.Pi(w)
    if variant != VARIANT_G:
        b.normE = power_iteration(E_apply, philox.power_start(n, 0, seed), power_iters)
    # For k < n, interlacing gives |E| >= lambda_min(A_mu) >= mu (the
    # eigenvalues of E on the complement of range(Y_mu) are not below those
    # of A_mu).  Clamping the estimate at mu changes nothing then, and keeps
    # tau > 0 in the degenerate case k = n, where E = 0 up to rounding.
    nE = max(b.normE, mu)

    if variant == VARIANT_C:
        # Alg. 7 step 2 with the SPD-preserving form of G
        M = Om.T @ Ymu
        M = 0.5 * (M + M.T)
        RM, b.jitter = chol_upper_jitter(M)
        T = right_solve_upper(RM, R)        # R_M R^-1
        b.G = T.T @ T
        # lambda_max(Pi A_mu Pi~), Pi~ = Q G Q^T: Alg. 7 step 3
        b.lam_max = power_iteration(lambda v: b.Pi(Amu(b.Q @ (b.G @ (b.Q.T @ v)))),
                                    philox.power_start(n, 1, seed), power_iters)
        if tau is not None:
            b.tau = float(tau)
            b.rho = b.tau * b.lam_max / nE
        else:
            if rho is None or rho <= 0:
                # eq:optimal_rho with F = 1/mu; rho = 0.5 a priori when mu = 0
                b.rho = math.sqrt(mu * b.lam_max / nE) if mu > 0 else 0.5
            else:
                b.rho = float(rho)
            b.tau = b.rho * nE / b.lam_max           # eq:c_randrand_tau
            if b.tau <= 0.0:                         # mu = 0 and k = n
                b.tau = 1.0 / b.lam_max
    elif variant == VARIANT_G:
        # G-RandRAND (Sec. 3.3 eq:g_randrand): P = (I - Pi) + tau Pi~ with
        # Pi~ = Q G Q^T, G = (R^-T (Omega^T Omega) R^-1)^(1/2) (the symmetric
        # square root, by an eigendecomposition)
        Ri = solve_upper(R, np.eye(k))
        MG = Ri.T @ (Om.T @ Om) @ Ri
        MG = 0.5 * (MG + MG.T)
        wv, V = np.linalg.eigh(MG)
        b.G = (V * np.sqrt(np.maximum(wv, 0.0))) @ V.T
        Pt = lambda v: b.Q @ (b.G @ (b.Q.T @ v))
        # |(I - Pi) A_mu| and |Pi~ A_mu| as square roots of the largest
        # eigenvalues of A_mu (I - Pi) A_mu and A_mu Pi~^2 A_mu (the G-RandRAND
        # MINRES estimates of Sec. 6.3)
        def EA(v):                       # A_mu (I - Pi) A_mu v
            u = Amu(v)
            return Amu(u - b.Pi(u))
        b.normE = math.sqrt(power_iteration(EA, philox.power_start(n, 0, seed), power_iters))
        b.lam_max = math.sqrt(power_iteration(lambda v: Amu(Pt(Pt(Amu(v)))),
                                              philox.power_start(n, 1, seed), power_iters))
        # eq:g_randrand_tau; rho = 0.5 a priori (the optimal rho of
        # eq:rho_g_rand_rand needs |A_mu^-1|, unknown for an indefinite A_mu)
        b.rho = float(rho) if (rho is not None and rho > 0) else 0.5
        b.tau = math.sqrt(b.rho) * b.normE / b.lam_max if tau is None else float(tau)
    elif variant == VARIANT_R:
        if refine:
            raise ValueError("the refined projector is applied to variants C and G")
        b.rho = 1.0
        b.tau = nE if tau is None else float(tau)        # Alg. 4 step 2
        if b.tau <= 0.0:                                  # mu = 0 and k = n
            b.tau = 1.0
    else:
        raise ValueError(variant)
    if refine:
        if int(refine) >= 2:
            b.refine_steps = int(refine)        # eq:accurate_proj_2
        else:
            b.Tref = neumann_T(b.Q)             # eq:accurate_proj
    return b


def neumann_T(Q: np.ndarray) -> np.ndarray:
    """T = 2 I - Q^T Q, the Neumann approximation of (Q^T Q)^-1 for a nearly
    orthonormal Q (Sec. 4.3 eq:accurate_proj): Q T Q^T u approximates the
    orthogonal projection Q (Q^T Q)^-1 Q^T u to second order in
    |I - Q^T Q|."""
    return 2.0 * np.eye(Q.shape[1]) - Q.T @ Q


# ==========================================================================
# Multiple shifts (Sec. 5.1): the parameter-free pieces of one sketch
# ==========================================================================
@dataclasses.dataclass
class ShiftSketch:
    """Omega, A Omega and the parameter-free Gram matrices of Sec. 5.1:
    P2 = (A Omega)^T (A Omega), M0 = Omega^T A Omega (symmetrized), S0 =
    Omega^T Omega."""
    Omega: np.ndarray
    AOmega: np.ndarray
    P2: np.ndarray
    M0: np.ndarray
    S0: np.ndarray


def shift_sketch(op, k: int, sketch: str = "gaussian", seed: int = 0, gamma: int = 8,
                 omega_precision: str = "fp64") -> ShiftSketch:
    Om = make_omega(op.n, k, sketch, seed, gamma, omega_precision)
    AOm = op.matmat(Om)
    M0 = Om.T @ AOm
    return ShiftSketch(Omega=Om, AOmega=AOm, P2=AOm.T @ AOm, M0=0.5 * (M0 + M0.T),
                       S0=Om.T @ Om)


def shifted_gram(sk: ShiftSketch, mu: float) -> np.ndarray:
    """(A Omega + mu Omega)^T (A Omega + mu Omega) from the parameter-free
    projections (the Gram separation of Sec. 5.1; A symmetric)."""
    return sk.P2 + 2.0 * mu * sk.M0 + mu * mu * sk.S0


@dataclasses.dataclass
class JointBasis:
    """The joint basis of Sec. 5.1 for several shifts: Q_joint with
    range(Q_joint) = range([Omega, A Omega]) and the 2k x k projections
    C1 = Q_joint^T A Omega and C2 = Q_joint^T Omega."""
    Qj: np.ndarray
    C1: np.ndarray
    C2: np.ndarray


def joint_basis(sk: ShiftSketch) -> JointBasis:
    """[Q_joint, ~] = qr([Omega, A Omega]) (Householder), then the two
    projections."""
    Qj, _ = householder_qr(np.hstack([sk.Omega, sk.AOmega]))
    return JointBasis(Qj=Qj, C1=Qj.T @ sk.AOmega, C2=Qj.T @ sk.Omega)


def joint_qr(jb: JointBasis, mu: float) -> tuple[np.ndarray, np.ndarray]:
    """For one shift: [Q_red, R] = qr(C1 + mu C2) (2k x k, Householder,
    diag(R) > 0) and Q = Q_joint Q_red, the QR factors of A Omega + mu Omega
    (Sec. 5.1)."""
    Qr, R = householder_qr(jb.C1 + mu * jb.C2)
    return jb.Qj @ Qr, R


# ==========================================================================
# Solve: Alg. 7 steps 5-11 (PCG) / Alg. 4 steps 3-9 (CG on B) with restarts
# ==========================================================================
@dataclasses.dataclass
class SolveInfo:
    inner_iters: int = 0
    outer_iters: int = 0
    rel_residual: float = math.inf
    converged: bool = False
    history: list = dataclasses.field(default_factory=list)


def pcg(Aop, b, Pop, stop: float, maxit: int):
    """Textbook preconditioned CG (Saad, Iterative Methods, Alg. 9.1), x0 = 0.
    Stops when the recursive residual norm is <= stop or after maxit steps."""
    x = np.zeros_like(b)
    r = b.copy()
    it = 0
    if np.linalg.norm(r) <= stop:
        return x, it
    z = Pop(r)
    p = z.copy()
    rz = float(r @ z)
    while it < maxit:
        w = Aop(p)
        alpha = rz / float(p @ w)
        x += alpha * p
        r -= alpha * w
        it += 1
        if np.linalg.norm(r) <= stop:
            break
        z = Pop(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


def minres(Aop, b, Pop, stop_rel: float, maxit: int):
    """Preconditioned MINRES (Paige and Saunders 1975, in the Lanczos /
    Givens form with an SPD preconditioner P ~ A^-1), x0 = 0.  Works with the
    unnormalised Lanczos vectors v_j and z_j = P v_j; eta carries the
    P-norm of the residual, |r_j|_P = sqrt(r_j^T P r_j).  Stops when |eta| <=
    stop_rel |eta_0| or after maxit steps."""
    x = np.zeros_like(b)
    v_prev = np.zeros_like(b)
    v = b.copy()
    z = Pop(v)
    zv = float(z @ v)
    it = 0
    if not (zv > 0.0 and math.isfinite(zv)):     # r = 0, or P not SPD in rounding
        return x, it
    gamma = math.sqrt(zv)
    eta = eta0 = gamma
    gamma_prev = 1.0
    c_prev = c = 1.0
    s_prev = s = 0.0
    w_prev = np.zeros_like(b)
    w = np.zeros_like(b)
    while it < maxit:
        z = z / gamma
        Az = Aop(z)
        delta = float(Az @ z)
        v_next = Az - (delta / gamma) * v - (gamma / gamma_prev) * v_prev
        z_next = Pop(v_next)
        zv = float(z_next @ v_next)
        if not (math.isfinite(zv) and math.isfinite(delta)):
            break                                  # breakdown: keep the iterate so far
        gamma_next = math.sqrt(max(zv, 0.0))
        # the new column of the tridiagonal matrix through the previous
        # rotations, then the rotation that annihilates gamma_next
        a0 = c * delta - c_prev * s * gamma
        a1 = math.hypot(a0, gamma_next)
        a2 = s * delta + c_prev * c * gamma
        a3 = s_prev * gamma
        c_next, s_next = a0 / a1, gamma_next / a1
        w_next = (z - a3 * w_prev - a2 * w) / a1
        x += c_next * eta * w_next
        eta = -s_next * eta
        it += 1
        v_prev, v = v, v_next
        z = z_next
        gamma_prev, gamma = gamma, gamma_next
        c_prev, c = c, c_next
        s_prev, s = s, s_next
        w_prev, w = w, w_next
        if abs(eta) <= stop_rel * eta0 or gamma == 0.0:
            break
    return x, it


def solve(b_: Build, B: np.ndarray, rtol: float, maxit: int = 20000,
          eta: float = 1e-2, x0: np.ndarray | None = None,
          fixed_inner: int | None = None):
    """Solve A_mu X = B column by column.  Returns (X, [SolveInfo]).

    Outer loop = the paper's restarting (Alg. 7 step 10 / Alg. 4 step 9):
    r = b - A_mu x in float64; stop when |r| <= rtol |b| or when the inner
    iterations reach maxit; otherwise run PCG (C), CG on B (R) or MINRES with
    the G-RandRAND preconditioner (G, Sec. 6.3) to the inner target
    max(eta |r|, 0.5 rtol |b|) (for MINRES the same reduction of the P-norm of
    the residual) and add the correction to x.

    fixed_inner: if set, run exactly that many inner iterations once (no
    restart), for iteration-level comparisons.
    """
    Amu = shifted(b_.op, b_.mu)
    B = np.asarray(B, dtype=np.float64)
    one = B.ndim == 1
    B2 = B[:, None] if one else B
    X = np.zeros_like(B2) if x0 is None else np.array(x0, dtype=np.float64).reshape(B2.shape)
    infos = []
    for c in range(B2.shape[1]):
        bc = B2[:, c]
        x = X[:, c]
        info = SolveInfo()
        nb = float(np.linalg.norm(bc))
        if nb == 0.0:
            x[:] = 0.0
            info.rel_residual = 0.0
            info.converged = True
            infos.append(info)
            continue
        while True:
            r = bc - Amu(x)
            rel = float(np.linalg.norm(r)) / nb
            info.history.append(rel)
            info.rel_residual = rel
            if fixed_inner is None and rel <= rtol:
                info.converged = True
                break
            if fixed_inner is not None and info.outer_iters == 1:
                break
            budget = maxit - info.inner_iters if fixed_inner is None else fixed_inner
            if budget <= 0:
                break
            stop = max(eta * rel * nb, 0.5 * rtol * nb) if fixed_inner is None else 0.0
            if b_.variant == VARIANT_C:
                e, it = pcg(Amu, r, b_.apply_P, stop, budget)
            elif b_.variant == VARIANT_G:
                # the same inner target relative to |r|, in the P-norm
                # MINRES tracks: |r_j|_P <= max(eta, 0.5 rtol |b| / |r|) |r_0|_P
                srel = max(eta, 0.5 * rtol * nb / (rel * nb)) if fixed_inner is None else 0.0
                e, it = minres(Amu, r, b_.apply_P, srel, budget)
            else:
                y, it = pcg(b_.apply_B, r, lambda v: v, stop, budget)
                e = b_.recover_R(y)
            x += e
            info.inner_iters += it
            info.outer_iters += 1
            if it == 0 or info.outer_iters >= MAX_RESTARTS:
                break                              # no progress (breakdown) or too many restarts
        infos.append(info)
    return (X[:, 0] if one else X), infos


# ==========================================================================
# Factorization-free least squares (Sec. 5.2 eq:iterative_refinement)
@dataclasses.dataclass
class NewtonSketchInfo:
    steps: int
    rel_normal_residual: list       # |Y^T (u - Y v_t)| / |Y^T u| after each step
    inner_iters: list               # CG iterations on D per step (0: exact solve)


def cg_spd(matvec, rhs: np.ndarray, tol: float, maxit: int) -> tuple[np.ndarray, int]:
    """Plain conjugate gradients for an SPD operator from x = 0, stopping at
    |rhs - D x| <= tol |rhs| (textbook Hestenes-Stiefel recurrences)."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    p = r.copy()
    rr = float(r @ r)
    stop = (tol * np.linalg.norm(rhs)) ** 2
    it = 0
    while it < maxit and rr > stop:
        Dp = matvec(p)
        alpha = rr / float(p @ Dp)
        x += alpha * p
        r -= alpha * Dp
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def newton_sketch_lstsq(Y: np.ndarray, S: np.ndarray, u: np.ndarray, steps: int,
                        inner_tol: float | None = None, inner_maxit: int = 100000):
    """v = argmin |Y v - u| for Y = A_mu Omega (n x k) without factoring:
    from v = 0, v <- v + D^-1 Y^T (u - Y v) with D = S^T S, S = Theta Y the
    two-sided sketch (Sec. 5.2 eq:iterative_refinement, the Newton-sketch
    iteration with the R factor taken as the identity).  D^-1 is applied by
    a library solve of the k x k system (inner_tol None) or, as the paper
    proposes, by CG on D (matvec S^T (S x)) to a relative residual inner_tol,
    whose iteration counts are returned."""
    Y = np.asarray(Y, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    D = S.T @ S
    v = np.zeros(Y.shape[1])
    g0 = np.linalg.norm(Y.T @ u)
    info = NewtonSketchInfo(steps=0, rel_normal_residual=[], inner_iters=[])
    for _ in range(steps):
        g = Y.T @ (u - Y @ v)
        if inner_tol is None:
            dv = np.linalg.solve(D, g)
            info.inner_iters.append(0)
        else:
            dv, it = cg_spd(lambda x: S.T @ (S @ x), g, inner_tol, inner_maxit)
            info.inner_iters.append(it)
        v = v + dv
        info.steps += 1
        info.rel_normal_residual.append(float(np.linalg.norm(Y.T @ (u - Y @ v)) / g0))
    return v, info


def exact_solve(op, mu: float, B: np.ndarray) -> np.ndarray:
    """x* = (A + mu I)^-1 b by a dense Cholesky solve (library routine)."""
    import scipy.linalg as sl
    A = op.dense() + mu * np.eye(op.n)
    return sl.cho_solve(sl.cho_factor(A, lower=True), B)


def true_rel_residual(op, mu: float, X: np.ndarray, B: np.ndarray) -> np.ndarray:
    R = np.asarray(B) - shifted(op, mu)(np.asarray(X))
    R = R.reshape(R.shape[0], -1)
    Bn = np.asarray(B).reshape(R.shape)
    return np.linalg.norm(R, axis=0) / np.linalg.norm(Bn, axis=0)
