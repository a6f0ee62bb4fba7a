"""Inputs that drive the core-matrix jitter ladder (App. C) on purpose.

The C-RandRAND core matrix M = sym(Omega^T A_mu Omega) is positive definite
in exact arithmetic for an SPD A_mu; the ladder only runs when rounding (for
instance a bf16 sketch) makes it indefinite.  To reach that branch with a
known answer, these helpers build a symmetric M with one slightly negative
eigenvalue, and a symmetric dense A with Omega^T (A + mu I) Omega = M for a
given Omega while A_mu Omega stays well conditioned.
"""
import numpy as np


def ladder_core(k=40, lam_neg=-5e-8, top=100.0, seed=5):
    """Symmetric k x k M: eigenvalue `top` along ones/sqrt(k), one eigenvalue
    `lam_neg` < 0, the others uniform in [1, 2].  The dominant direction is
    spread over every coordinate, so |M|_2 = top is far above the largest
    diagonal entry (~ top / k + 2): the two readings of |M| pick different
    rungs of the ladder."""
    rng = np.random.default_rng(seed)
    V, _ = np.linalg.qr(np.column_stack([np.ones(k), rng.standard_normal((k, k - 1))]))
    lam = np.concatenate([[top], rng.uniform(1.0, 2.0, k - 2), [lam_neg]])
    M = (V * lam) @ V.T
    return 0.5 * (M + M.T)


def operator_with_core(Om, M, mu, seed=6):
    """Dense symmetric A (n x n) with Omega^T (A + mu I) Omega = M.

    With U = [U1 U2] orthonormal, U1 spanning range(Omega) (Omega = U1 S),
    A_mu = U [[A11, A21^T], [A21, A22]] U^T where A11 = S^-T M S^-1 fixes the
    core matrix, A21 = [I_k; 0] keeps A_mu Omega = (U1 A11 + U2 A21) S of
    full rank however singular M is, and A22 = diag(d), d in [0.5, 3]."""
    n, k = Om.shape
    assert n >= 2 * k
    rng = np.random.default_rng(seed)
    U, S = np.linalg.qr(Om, mode="complete")
    S = S[:k]
    Si = np.linalg.inv(S)
    A11 = Si.T @ M @ Si
    A21 = np.zeros((n - k, k))
    A21[:k] = np.eye(k)
    A22 = np.diag(rng.uniform(0.5, 3.0, n - k))
    Amu = np.block([[A11, A21.T], [A21, A22]])
    Amu = U @ Amu @ U.T
    Amu = 0.5 * (Amu + Amu.T)
    return Amu - mu * np.eye(n)


def ladder_rung(M, scale):
    """Brute force over the App. C set: the smallest 10^e scale (e = -14..-1)
    with lambda_min(M) + 10^e scale > 0, by dense eigenvalues; None if none."""
    lmin = np.linalg.eigvalsh(M).min()
    if lmin > 0:
        return 0.0
    for e in range(-14, 0):
        a = 10.0 ** e * scale
        if lmin + a > 0:
            return a
    return None
