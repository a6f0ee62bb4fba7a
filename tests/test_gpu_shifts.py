"""GPU parity of several shifts from one sketch (Sec. 5.1): a handle built
with keep_sketch keeps A Omega and the shift-free projections, and
randrand_set_mu rebuilds the preconditioner for another mu.  The oracle is a
fresh float64 build at that mu with the same Omega (R is unique once its
diagonal is positive, so the Gram separation and the Householder QR give it
to rounding)."""
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


def check_factors(h, bd):
    cond = np.linalg.cond(bd.R)
    assert rel(h.export("R").cpu().numpy(), bd.R) <= max(1e-12, 1e-15 * cond) * 100
    assert rel(h.export("G").cpu().numpy(), bd.G) <= max(1e-12, 1e-15 * cond ** 2) * 100
    tau, nE, lmax = h.scalars()
    assert nE == pytest.approx(bd.normE, rel=1e-8)
    assert lmax == pytest.approx(bd.lam_max, rel=1e-8)
    assert tau == pytest.approx(bd.tau, rel=1e-8)


def test_set_mu_matches_fresh_builds_fp64(cuda_lib):
    """Dense float64: the kept-sketch build and two later shifts equal fresh
    oracle builds at those shifts; solves reach the exact solution; going back
    to the first shift reproduces its factors exactly."""
    rr = cuda_lib
    n, k, seed = 700, 60, 91
    P = W.dense_power_spectrum(n, seed=W.SEED_DENSE, power=2.0)
    op = O.DenseOp(P.A)
    B = W.gaussian_rhs(n, 2, seed)
    mus = (1e-4, 1e-2, 0.5)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mus[0], k, "gaussian", seed=seed, max_rhs=2,
                  keep_sketch=True)
    R0 = h.export("R").cpu().numpy()
    for i, mu in enumerate(mus):
        if i > 0:
            h.set_mu(mu)
        check_factors(h, O.build(op, mu, k, "gaussian", seed=seed))
        x, status, infos = h.solve(dev(B), rtol=1e-12)
        assert status == rr.RR_OK
        assert rel(x.cpu().numpy(), O.exact_solve(op, mu, B)) <= 1e-8
    h.set_mu(mus[0])
    assert np.array_equal(h.export("R").cpu().numpy(), R0)


def test_set_mu_kernel_mixed(cuda_lib):
    """Gaussian kernel, bf16 tensor-core sketch and float32 iterations: along a
    shift path each solve meets rtol with the float64 residual as the criterion,
    in about the iterations of a fresh build at that shift."""
    rr = cuda_lib
    n, k, seed = 3001, 80, 92
    X = W.mixture_points(n, seed=seed)
    op = O.GaussKernelOp(X)
    B = W.gaussian_rhs(n, 4, seed)
    Xd = dev(X)
    path = rr.Handle(rr.Operator.gauss_kernel(Xd), 1e-3, k, "gaussian", seed=seed,
                     precision="mixed", max_rhs=4, keep_sketch=True)
    for i, mu in enumerate((1e-3, 1e-2, 1e-4)):
        if i > 0:
            path.set_mu(mu)
        x, status, infos = path.solve(dev(B), rtol=1e-6)
        assert status == rr.RR_OK
        assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)
        fresh = rr.Handle(rr.Operator.gauss_kernel(Xd), mu, k, "gaussian", seed=seed,
                          precision="mixed", max_rhs=4)
        _, fstatus, finfos = fresh.solve(dev(B), rtol=1e-6)
        assert fstatus == rr.RR_OK
        for a, b in zip([j["inner_iters"] for j in infos], [j["inner_iters"] for j in finfos]):
            assert abs(a - b) <= max(3, 0.05 * b)
        fresh.close()


def test_keep_sketch_options(cuda_lib):
    rr = cuda_lib
    n = 300
    P = W.dense_power_spectrum(n, seed=93, power=2.0)
    A = rr.Operator.dense(dev(P.A))
    with pytest.raises(rr.RandRandError):          # variant R keeps no Gram of A Omega
        rr.Handle(A, 1e-3, 16, "gaussian", seed=93, variant="R", keep_sketch=True)
    with pytest.raises(rr.RandRandError):          # q >= 1 is not recycled
        rr.Handle(A, 1e-3, 16, "gaussian", seed=93, q=1, keep_sketch=True)
    h = rr.Handle(A, 1e-3, 16, "gaussian", seed=93)
    with pytest.raises(rr.RandRandError):          # built without keep_sketch
        h.set_mu(1e-2)
    h2 = rr.Handle(A, 1e-3, 16, "gaussian", seed=93, keep_sketch=True)
    with pytest.raises(rr.RandRandError):
        h2.set_mu(-1.0)
    with pytest.raises(rr.RandRandError):
        h2.set_mu(float("nan"))


# ------------------------------------------------ joint basis (Sec. 5.1)
def test_joint_basis_matches_oracle_fp64(cuda_lib):
    """keep_sketch = 2 (the joint basis): the factors at the build shift and
    at two later shifts equal the oracle's joint QR and a fresh float64 build
    (R unique with a positive diagonal), and the solves reach the exact
    solution."""
    rr = cuda_lib
    n, k, seed = 700, 60, 93
    P = W.dense_power_spectrum(n, seed=W.SEED_DENSE, power=2.0)
    op = O.DenseOp(P.A)
    B = W.gaussian_rhs(n, 2, seed)
    mus = (1e-4, 1e-2, 0.5)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mus[0], k, "gaussian", seed=seed, max_rhs=2,
                  keep_sketch=2)
    Om = h.export("omega").cpu().numpy()
    jb = O.joint_basis(O.ShiftSketch(Omega=Om, AOmega=P.A @ Om, P2=None, M0=None, S0=None))
    for i, mu in enumerate(mus):
        if i > 0:
            h.set_mu(mu)
        _, Rj = O.joint_qr(jb, mu)
        Rg = h.export("R").cpu().numpy()
        assert rel(Rg, Rj) <= max(1e-12, 1e-15 * np.linalg.cond(Rj)) * 100
        check_factors(h, O.build(op, mu, k, "gaussian", seed=seed))
        Q = h.export("Q").cpu().numpy()
        assert np.linalg.norm(Q.T @ Q - np.eye(k), 2) <= 1e-12
        x, status, infos = h.solve(dev(B), rtol=1e-12)
        assert status == rr.RR_OK
        assert rel(x.cpu().numpy(), O.exact_solve(op, mu, B)) <= 1e-8


def test_joint_basis_kernel_mixed(cuda_lib):
    """Gaussian kernel with float32 iterations: along a shift path the joint
    basis gives solves that meet rtol with the float64 residual as the criterion,
    and an orthonormal float32 basis whose Q R reproduces Y_mu = A Omega +
    mu Omega of the oracle (same bf16-rounded Omega; the sketch products are
    bf16 tensor-core products, hence 1e-2)."""
    rr = cuda_lib
    n, k, seed = 3001, 80, 94
    X = W.mixture_points(n, seed=seed)
    op = O.GaussKernelOp(X)
    B = W.gaussian_rhs(n, 4, seed)
    Xd = dev(X)
    joint = rr.Handle(rr.Operator.gauss_kernel(Xd), 1e-3, k, "gaussian", seed=seed,
                      precision="mixed", max_rhs=4, keep_sketch=2)
    Om = joint.export("omega").cpu().numpy().astype(np.float64)
    AOm = op.matmat(Om)
    for i, mu in enumerate((1e-3, 1e-2, 1e-4)):
        if i > 0:
            joint.set_mu(mu)
        Q = joint.export("Q").cpu().numpy().astype(np.float64)
        assert np.linalg.norm(Q.T @ Q - np.eye(k), 2) <= 2e-5
        assert rel(Q @ joint.export("R").cpu().numpy(), AOm + mu * Om) <= 1e-2
        x, status, infos = joint.solve(dev(B), rtol=1e-6)
        assert status == rr.RR_OK
        assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)


def test_joint_basis_rejects_unsupported(cuda_lib):
    """keep_sketch = 2 needs the C variant with an explicit basis."""
    rr = cuda_lib
    P = W.dense_power_spectrum(200, seed=W.SEED_DENSE, power=2.0)
    with pytest.raises(rr.RandRandError):
        rr.Handle(rr.Operator.dense(dev(P.A)), 1e-3, 20, "gaussian", seed=1, variant="R",
                  keep_sketch=2)
