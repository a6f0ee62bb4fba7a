"""Shared rounds (randrand_solve_group): several built systems' PCG iterations
advanced together, one grouped tensor-core product and one grouped
persistent step per round, through the C ABI.

Each system solved in the group is checked against the same system solved
alone (randrand_solve) and against the float64 oracle: the float64 residual
over all rows meets rtol, the solution agrees with the solo solution to
the forward error both have, and at a tight rtol with the dense Cholesky
solution x*.  Only the summation order of the product's split sums and of
the step's Q^T r differs between the two schedules (float32 rounding), so
iteration counts agree within a few steps.
"""
import numpy as np
import pytest

from oracle import randrand as O
from workloads import generators as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (n, mu, k): uneven sizes, shifts and sketch dimensions, all below one
# persistent grid's worth of work items
SPECS = [(2000, 1e-3, 50), (3001, 1e-4, 75), (5000, 1e-2, 125), (1500, 1e-5, 37)]


def _systems(rr, m, seed0):
    out = []
    for i, (n, mu, k) in enumerate(SPECS):
        X = W.mixture_points(n, seed=seed0 + i)
        B = W.gaussian_rhs(n, m, seed0 + i)
        h = rr.Handle(rr.Operator.gauss_kernel(torch.from_numpy(X).cuda()), mu, k, "gaussian",
                      seed=seed0 + i, precision="mixed", max_rhs=m)
        out.append((X, B, mu, h))
    return out


@pytest.mark.parametrize("m", [4, 8])
def test_group_solves_match_solo_solves(cuda_lib, m):
    rr = cuda_lib
    sys = _systems(rr, m, 300 + m)
    solo = []
    for X, B, mu, h in sys:
        x, st, infos = h.solve(torch.from_numpy(B).cuda(), rtol=1e-6)
        assert st == rr.RR_OK
        solo.append((x.cpu().numpy(), [i["inner_iters"] for i in infos]))
    st, xs, infos = rr.solve_group([h for *_, h in sys], [torch.from_numpy(B).cuda() for _, B, _, _ in sys],
                                   rtol=1e-6, stream=torch.cuda.Stream())
    assert st == rr.RR_OK, infos
    for (X, B, mu, h), (xs0, it0), x, inf in zip(sys, solo, xs, infos):
        x = x.cpu().numpy()
        op = O.GaussKernelOp(X)
        res = O.true_rel_residual(op, mu, x, B)
        assert np.all(res <= 1e-6), res
        rep = np.array([i["rel_residual"] for i in inf])
        assert np.allclose(res, rep, rtol=1e-3, atol=1e-12)
        it = [i["inner_iters"] for i in inf]
        assert all(abs(a - b) <= max(3, 0.05 * b) for a, b in zip(it, it0)), (it, it0)
        # both solutions are within ~rtol of x* (relative residual ~ relative
        # forward error here); they agree to a few times that
        d = np.linalg.norm(x - xs0, axis=0) / np.linalg.norm(xs0, axis=0)
        assert np.all(d <= 1e-5), d
    for *_, h in sys:
        h.close()


def test_group_tight_rtol_matches_exact_solution(cuda_lib):
    rr = cuda_lib
    m = 4
    sys = _systems(rr, m, 410)
    st, xs, infos = rr.solve_group([h for *_, h in sys], [torch.from_numpy(B).cuda() for _, B, _, _ in sys],
                                   rtol=1e-10, stream=torch.cuda.Stream())
    assert st == rr.RR_OK, infos
    for (X, B, mu, h), x in zip(sys, xs):
        xs_ = O.exact_solve(O.GaussKernelOp(X), mu, B)
        err = np.linalg.norm(x.cpu().numpy() - xs_) / np.linalg.norm(xs_)
        assert err <= 1e-5, err
        h.close()


def test_group_rejects_unsupported_handles(cuda_lib):
    rr = cuda_lib
    n = 500
    A = torch.from_numpy(W.dense_power_spectrum(n, seed=3).A).cuda()
    h = rr.Handle(rr.Operator.dense(A), 1e-3, 20, "gaussian", seed=3)      # float64 dense
    with pytest.raises(rr.RandRandError):
        rr.solve_group([h], [torch.zeros(n, dtype=torch.float64, device="cuda")], rtol=1e-6,
                       stream=torch.cuda.Stream())
    h.close()
