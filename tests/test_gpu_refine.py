"""GPU parity of the refined projector (Sec. 4.3 eq:accurate_proj and
eq:accurate_proj_2): P = I + Q (tau T G T - T) Q^T with T = 2 I - Q^T Q of
the stored basis, or the polynomial T of the refinement recurrence, against
the oracle's refined build (float64), and its effect in the float32 paths,
where the stored basis is orthonormal only to float32 rounding."""
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


@pytest.mark.parametrize("refine", [1, 3])
@pytest.mark.parametrize("variant", ["C", "G"])
def test_refined_apply_and_iterates_fp64(cuda_lib, variant, refine):
    """refine = 1: the Neumann T of eq:accurate_proj; refine = 3: the
    eq:accurate_proj_2 recurrence with three steps beyond the first (the
    library folds it into a k x k polynomial at build, the oracle runs the
    recurrence on every vector)."""
    rr = cuda_lib
    n, k = 600, 50
    P = W.dense_power_spectrum(n, seed=111, power=2.0)
    if variant == "G":
        ev = np.sort(np.linalg.eigvalsh(P.A))[::-1]
        mu = -0.5 * (ev[20] + ev[21])
    else:
        mu = 1e-4
    op = O.DenseOp(P.A)
    h = rr.Handle(rr.Operator.dense(dev(P.A)), mu, k, "gaussian", seed=111, variant=variant,
                  q=1 if variant == "G" else 0, max_rhs=2, refine=refine)
    bd = O.build(op, mu, k, "gaussian", seed=111, variant=variant, q=1 if variant == "G" else 0,
                 refine=refine)
    r = np.random.default_rng(2).standard_normal((n, 2))
    cond = np.linalg.cond(bd.R)
    assert rel(h.apply(dev(r)).cpu().numpy(), bd.apply_P(r)) <= max(1e-12, 1e-15 * cond ** 2) * 100
    B = W.gaussian_rhs(n, 2, 111)
    for budget in (3, 9):
        x, status, infos = h.solve(dev(B), rtol=1e-14, maxit=budget)
        xo, oinfo = O.solve(bd, B, rtol=1e-14, maxit=budget)
        assert [i["inner_iters"] for i in infos] == [i.inner_iters for i in oinfo]
        assert rel(x.cpu().numpy(), xo) <= 1e-9
    x, status, infos = h.solve(dev(B), rtol=1e-11, maxit=20000)
    assert status == rr.RR_OK
    assert rel(x.cpu().numpy(), np.linalg.solve(P.A + mu * np.eye(n), B)) <= 1e-6


def test_refined_kernel_mixed_solve(cuda_lib):
    """bf16 sketch, float32 basis: T differs from I at float32 rounding, the
    refined P from the plain one at about that level; both solves meet rtol
    with the float64 residual as the criterion, in about the same iterations."""
    rr = cuda_lib
    n, k, mu = 3001, 80, 1e-3
    X = W.mixture_points(n, seed=112)
    op = O.GaussKernelOp(X)
    B = W.gaussian_rhs(n, 4, 112)
    r = np.random.default_rng(3).standard_normal((n, 4))
    its, z = {}, {}
    for refine in (False, True):
        h = rr.Handle(rr.Operator.gauss_kernel(dev(X)), mu, k, "gaussian", seed=112,
                      precision="mixed", max_rhs=4, refine=refine)
        z[refine] = h.apply(dev(r)).cpu().numpy()
        x, status, infos = h.solve(dev(B), rtol=1e-6)
        assert status == rr.RR_OK
        assert np.all(O.true_rel_residual(op, mu, x.cpu().numpy(), B) <= 1e-6)
        its[refine] = max(i["inner_iters"] for i in infos)
    d = rel(z[True], z[False])
    assert 0.0 < d < 1e-3
    assert abs(its[True] - its[False]) <= max(3, 0.05 * its[False])


def test_refine_options(cuda_lib):
    rr = cuda_lib
    P = W.dense_power_spectrum(200, seed=113, power=2.0)
    A = rr.Operator.dense(dev(P.A))
    with pytest.raises(rr.RandRandError):          # variant R keeps B's projector plain
        rr.Handle(A, 1e-3, 20, "gaussian", seed=113, variant="R", refine=True)
    with pytest.raises(rr.RandRandError):          # at most 8 refinement steps
        rr.Handle(A, 1e-3, 20, "gaussian", seed=113, refine=9)
    h = rr.Handle(A, 1e-3, 20, "gaussian", seed=113, refine=True, keep_sketch=True)
    h.set_mu(1e-2)                                 # the shift path rebuilds the refined H
    bd = O.build(O.DenseOp(P.A), 1e-2, 20, "gaussian", seed=113, refine=True)
    r = np.random.default_rng(4).standard_normal((200, 1))
    assert rel(h.apply(dev(r)).cpu().numpy(), bd.apply_P(r)) <= 1e-9
