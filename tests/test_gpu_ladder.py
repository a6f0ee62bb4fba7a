"""GPU parity of the core-matrix jitter ladder (App. C) through the C ABI.

A dense float64 operator whose core matrix M = sym(Omega^T A_mu Omega) has one
slightly negative eigenvalue makes both the library's and the oracle's C
builds take the ladder: R_M = chol(M + alpha I), alpha the smallest of
10^-14 |M|, ..., 10^-1 |M| that factors, |M| the spectral norm.  The sparse
sign Omega is integer work and bit for bit the oracle's, so M agrees to
float64 rounding and both sides must land on the same rung; then G, tau and
the power-iteration estimates agree to the float64 path's 1e-10 (1e-9 for
the estimates, whose 20 steps run in a different summation order).
"""
import numpy as np
import pytest

from oracle import randrand as O
from ladder_cases import ladder_core, ladder_rung, operator_with_core

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,lam_neg", [(40, -5e-8), (64, -3e-11)])
def test_core_matrix_jitter_ladder_matches_oracle(cuda_lib, k, lam_neg):
    rr = cuda_lib
    n, mu, seed = 10 * k, 1e-3, 21
    Om = O.make_omega(n, k, "sparse_sign", seed, gamma=8)
    M = ladder_core(k, lam_neg=lam_neg)
    A = operator_with_core(Om, M, mu)
    ref = O.build(O.DenseOp(A), mu, k, "sparse_sign", seed, gamma=8)
    expected = ladder_rung(M, np.abs(np.linalg.eigvalsh(M)).max())
    assert ref.jitter == pytest.approx(expected, rel=1e-9) and expected > 0

    h = rr.Handle(rr.Operator.dense(torch.from_numpy(A).cuda()), mu, k, "sparse_sign",
                  seed=seed, gamma=8, precision="fp64")
    assert np.array_equal(h.export("omega").cpu().numpy(), ref.Omega)
    # the library's |M| is a 30-step power estimate; here the dominant
    # eigenvalue is isolated, so it matches the spectral norm to rounding
    assert h.core_jitter() == pytest.approx(ref.jitter, rel=1e-10)
    G = h.export("G").cpu().numpy()
    R = h.export("R").cpu().numpy()
    assert np.max(np.abs(R - ref.R)) <= 1e-10 * np.abs(ref.R).max()
    assert np.max(np.abs(G - ref.G)) <= 1e-10 * np.abs(ref.G).max()
    # R^T G R = M + alpha I: the smallest eigenvalue moved by exactly the rung
    lam = np.linalg.eigvalsh(R.T @ G @ R)
    assert lam.min() == pytest.approx(lam_neg + expected, rel=1e-3, abs=1e-12)
    tau, normE, lam_max = h.scalars()
    assert normE == pytest.approx(ref.normE, rel=1e-9)
    assert lam_max == pytest.approx(ref.lam_max, rel=1e-9)
    assert tau == pytest.approx(ref.tau, rel=1e-9)
