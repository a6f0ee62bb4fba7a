"""GPU parity of the SRHT test matrix (Sec. 2, fast randomized transforms):
Omega bit for bit against the oracle's draw (same Philox streams, same keyed
Feistel subsampling), float64 factors against the oracle build, a mixed
precision kernel solve checked by the float64 residual, and the basis-less CSR
form, which applies Omega and Omega^T by fast Walsh-Hadamard transforms (one
shared-memory pass, or two when s exceeds the block)."""
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


@pytest.mark.parametrize("n,k", [(300, 40), (1024, 64), (3001, 100)])
def test_srht_omega_fp64_exact(cuda_lib, n, k):
    """n ragged (s = 512, 4096) and a power of two: the drawn Omega equals the
    oracle's exactly.  (n just above a power of two is avoided here: the
    zero-padded SRHT then keeps Hadamard rows r and r ^ s/2 that agree on all
    but n - s/2 of the n coordinates, and drawing both makes A_mu Omega
    numerically rank-deficient; the build reports RR_ERR_NOT_SPD.)"""
    rr = cuda_lib
    P = W.dense_power_spectrum(n, seed=95, power=2.0)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), 1e-3, k, "srht", seed=95)
    assert np.array_equal(h.export("omega").cpu().numpy(), philox.srht_omega(n, k, 95))


def test_srht_omega_bf16_exact(cuda_lib):
    rr = cuda_lib
    n, k = 3001, 80
    X = W.mixture_points(n, seed=96)
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), 1e-3, k, "srht", seed=96, precision="mixed")
    ref = philox.round_bf16(philox.srht_omega(n, k, 96))
    assert np.array_equal(h.export("omega").cpu().numpy(), ref)


def test_srht_factors_fp64(cuda_lib):
    rr = cuda_lib
    n, k, mu = 700, 60, 1e-4
    P = W.dense_power_spectrum(n, seed=W.SEED_DENSE, power=2.0)
    op = O.DenseOp(P.A)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mu, k, "srht", seed=97, max_rhs=2)
    bd = O.build(op, mu, k, "srht", seed=97)
    cond = np.linalg.cond(bd.R)
    assert rel(h.export("R").cpu().numpy(), bd.R) <= max(1e-12, 1e-15 * cond) * 100
    assert rel(h.export("G").cpu().numpy(), bd.G) <= max(1e-12, 1e-15 * cond ** 2) * 100
    tau, nE, lmax = h.scalars()
    assert tau == pytest.approx(bd.tau, rel=1e-8)
    B = W.gaussian_rhs(n, 2, 97)
    x, status, infos = h.solve(dev(B), rtol=1e-12)
    assert status == rr.RR_OK
    assert rel(x.cpu().numpy(), O.exact_solve(op, mu, B)) <= 1e-8


def test_srht_kernel_mixed_solve(cuda_lib):
    rr = cuda_lib
    n, k, mu = 3001, 80, 1e-3
    X = W.mixture_points(n, seed=98)
    op = O.GaussKernelOp(X)
    B = W.gaussian_rhs(n, 4, 98)
    h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "srht", seed=98, precision="mixed",
                  max_rhs=4)
    x, status, infos = h.solve(dev(B), rtol=1e-6)
    assert status == rr.RR_OK
    assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_srht_basis_less_fwht(cuda_lib, precision):
    """n = 9216 (s = 16384: two transform passes, zero padding): the float64
    preconditioner apply and fixed-budget iterates equal the oracle's (which
    applies the dense Omega); the mixed solve meets rtol by the float64
    residual."""
    rr = cuda_lib
    C = W.diffusion_csr(side=96, seed=99, corr_len=4.0)
    op = O.CsrOp(C.rowptr, C.colidx, C.vals, C.n)
    fp64 = precision == "fp64"
    vals = dev(C.vals.astype(np.float64)) if fp64 else dev(C.vals)
    mu, k = 1e-6, 48
    h = rr.Handle(rr.Operator.csr(dev(C.rowptr), dev(C.colidx), vals), mu, k, "srht", seed=99,
                  orth="rand_cholqr", precision=precision, max_rhs=2)
    B = W.gaussian_rhs(C.n, 2, 99)
    if fp64:
        bd = O.build(op, mu, k, "srht", seed=99, orth="qless")
        r = np.random.default_rng(5).standard_normal((C.n, 2))
        cond = np.linalg.cond(bd.R)
        assert rel(h.apply(dev(r)).cpu().numpy(), bd.apply_P(r)) <= max(1e-12, 1e-15 * cond ** 2) * 100
        x, status, infos = h.solve(dev(B), rtol=1e-14, maxit=6)
        xo, oinfo = O.solve(bd, B, rtol=1e-14, maxit=6)
        assert [i["inner_iters"] for i in infos] == [i.inner_iters for i in oinfo]
        assert rel(x.cpu().numpy(), xo) <= 1e-9
    x, status, infos = h.solve(dev(B), rtol=1e-6, maxit=20000)
    assert status == rr.RR_OK
    assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)
