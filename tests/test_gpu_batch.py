"""Many systems on one GPU: randrand_solve_batch and the serving loop.

Each system's result must not depend on what else runs beside it: a system
solved inside a batch or a server mix equals the same system solved alone
through randrand_build + randrand_solve (same seeds; the kernels of the
Gaussian-kernel and dense paths reduce in a fixed order, so the iterates agree
to rounding-free equality of the iteration counts and 1e-12 in x), and every
solution meets its rtol in the float64 residual of the oracle's product.
"""
import numpy as np
import pytest

from oracle import randrand as O
from workloads import generators as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def kernel_system(rr, i, n, m=3):
    X = W.mixture_points(n, seed=W.SEED_BATCH + i)
    mu = 10.0 ** (-5 + 3 * ((i * 0.37) % 1.0))
    k = max(n // 40, 8)
    B = W.gaussian_rhs(n, m, W.SEED_BATCH + i)
    return dict(X=X, op=rr.Operator.gauss_kernel(dev(X)), mu=mu, k=k, B=B, seed=W.SEED_BATCH + i,
                oracle=O.GaussKernelOp(X))


def alone(rr, s, rtol, precision="mixed", sketch="gaussian", orth="cholqr2"):
    m = s["B"].shape[1]
    h = rr.Handle(s["op"], s["mu"], s["k"], sketch, seed=s["seed"], precision=precision,
                  max_rhs=m, orth=orth)
    x, status, infos = h.solve(dev(s["B"]), rtol=rtol)
    h.close()
    return x.cpu().numpy(), status, infos


def test_batch_equals_systems_solved_alone(cuda_lib):
    rr = cuda_lib
    sizes = [600, 2000, 900, 1500, 1200, 777]
    systems = [kernel_system(rr, i, n) for i, n in enumerate(sizes)]
    rtol = 1e-6
    reqs = [rr.Request(s["op"], s["mu"], s["k"], dev(s["B"]), rtol, seed=s["seed"]) for s in systems]
    st, res = rr.solve_batch(reqs, workers=4)
    assert st == rr.RR_OK
    for s, q, r in zip(systems, reqs, res):
        assert r["status"] == rr.RR_OK
        xb = q.x.cpu().numpy()
        xa, sa, ia = alone(rr, s, rtol)
        assert sa == rr.RR_OK
        assert [i["inner_iters"] for i in r["info"]] == [i["inner_iters"] for i in ia]
        assert rel(xb, xa) <= 1e-12
        assert np.all(O.true_rel_residual(s["oracle"], s["mu"], xb, s["B"]) <= rtol)
        assert r["end_ms"] >= r["start_ms"] >= r["submit_ms"]
        assert r["build_ms"] > 0 and r["solve_ms"] > 0


def test_batch_mixed_operator_kinds(cuda_lib):
    """Dense, Gaussian-kernel and basis-less CSR systems in one batch."""
    rr = cuda_lib
    rtol = 1e-6
    P = W.dense_power_spectrum(500, seed=W.SEED_DENSE, power=2.0)
    C = W.diffusion_csr(side=48, seed=51, corr_len=4.0)
    kern = kernel_system(rr, 9, 1100, m=2)
    bd = W.gaussian_rhs(500, 1, 52)
    bc = W.gaussian_rhs(C.n, 2, 53)
    csr_op = rr.Operator.csr(dev(C.rowptr), dev(C.colidx), dev(C.vals))
    reqs = [
        rr.Request(rr.Operator.dense(dev(P.A)), 1e-4, 50, dev(bd), rtol, seed=5, precision="fp64"),
        rr.Request(kern["op"], kern["mu"], kern["k"], dev(kern["B"]), rtol, seed=kern["seed"]),
        rr.Request(csr_op, 1e-6, 32, dev(bc), rtol, sketch="sparse_sign", seed=53,
                   orth="rand_cholqr"),
    ]
    st, res = rr.solve_batch(reqs, workers=3)
    assert st == rr.RR_OK, res
    xd = reqs[0].x.cpu().numpy()
    assert O.true_rel_residual(O.DenseOp(P.A), 1e-4, xd, bd)[0] <= rtol
    xk = reqs[1].x.cpu().numpy()
    assert np.all(O.true_rel_residual(kern["oracle"], kern["mu"], xk, kern["B"]) <= rtol)
    xc = reqs[2].x.cpu().numpy()
    op = O.CsrOp(C.rowptr, C.colidx, C.vals, C.n)
    assert np.all(O.true_rel_residual(op, 1e-6, xc, bc) <= rtol)
    # the dense float64 system alone gives the same iterate
    h = rr.Handle(rr.Operator.dense(dev(P.A)), 1e-4, 50, "gaussian", seed=5)
    xa, sa, _ = h.solve(dev(bd), rtol=rtol)
    assert rel(xd, xa.cpu().numpy()) <= 1e-12


def test_batch_new_test_matrices_and_options(cuda_lib):
    """Multi-level and SRHT test matrices (the SRHT applied by fast
    Walsh-Hadamard transforms in the basis-less CSR form) and the refined
    projector inside one batch: every system meets rtol by the float64
    residual, in the iterations it takes alone."""
    rr = cuda_lib
    rtol = 1e-6
    C = W.diffusion_csr(side=40, seed=54, corr_len=4.0)
    csr_op = rr.Operator.csr(dev(C.rowptr), dev(C.colidx), dev(C.vals))
    bc = W.gaussian_rhs(C.n, 1, 54)
    k1 = kernel_system(rr, 11, 1500, m=2)
    k2 = kernel_system(rr, 12, 1300, m=2)
    specs = [
        (k1["op"], k1["mu"], k1["k"], k1["B"], dict(sketch="multilevel", seed=k1["seed"])),
        (k2["op"], k2["mu"], k2["k"], k2["B"], dict(sketch="srht", seed=k2["seed"], refine=True)),
        (csr_op, 1e-6, 32, bc, dict(sketch="srht", seed=54, orth="rand_cholqr")),
        (csr_op, 1e-6, 32, bc, dict(sketch="multilevel", seed=55, orth="rand_cholqr")),
    ]
    reqs = [rr.Request(op, mu, k, dev(B), rtol, **kw) for op, mu, k, B, kw in specs]
    st, res = rr.solve_batch(reqs, workers=4)
    assert st == rr.RR_OK, res
    oracles = [k1["oracle"], k2["oracle"], O.CsrOp(C.rowptr, C.colidx, C.vals, C.n),
               O.CsrOp(C.rowptr, C.colidx, C.vals, C.n)]
    for (op, mu, k, B, kw), q, r, orc in zip(specs, reqs, res, oracles):
        assert r["status"] == rr.RR_OK
        x = q.x.cpu().numpy()
        assert np.all(O.true_rel_residual(orc, mu, x, B) <= rtol)
        h = rr.Handle(op, mu, k, kw["sketch"], seed=kw["seed"], precision="mixed",
                      max_rhs=B.shape[1], orth=kw.get("orth", "cholqr2"),
                      refine=kw.get("refine", False))
        _, sa, ia = h.solve(dev(B), rtol=rtol)
        h.close()
        assert sa == rr.RR_OK
        # float32 iterations with atomic scatter sums: run-to-run rounding
        # differences move long CSR solves by a few iterations
        for a, b in zip([i["inner_iters"] for i in r["info"]], [i["inner_iters"] for i in ia]):
            assert abs(a - b) <= max(3, 0.02 * b)


def test_server_alone_vs_mix_and_admission(cuda_lib):
    """Requests submitted while others run complete with the results they
    have alone; a budget that holds one workspace at a time serialises them
    and the arena's peak never exceeds it."""
    rr = cuda_lib
    rtol = 1e-6
    systems = [kernel_system(rr, 20 + i, n, m=1) for i, n in enumerate([800, 1600, 1000, 1300])]
    reqs = [rr.Request(s["op"], s["mu"], s["k"], dev(s["B"]), rtol, seed=s["seed"]) for s in systems]
    ws = [q.workspace_bytes() for q in reqs]
    # roomy budget, 3 workers: requests overlap
    srv = rr.Server(budget_bytes=sum(w + 256 for w in ws), workers=3)
    tickets = [srv.submit(q) for q in reqs]
    res = [srv.poll(t, wait=True) for t in tickets]
    peak = srv.peak_running()
    srv.close()
    # at least two requests were resident (admitted, not completed) at once
    assert peak >= 2
    spans = sorted((r["start_ms"], r["end_ms"]) for r in res)
    assert any(s1 < e0 for (s0, e0), (s1, e1) in zip(spans, spans[1:]))
    for s, q, r in zip(systems, reqs, res):
        assert r["status"] == rr.RR_OK
        xa, sa, ia = alone(rr, s, rtol)
        assert r["info"][0]["inner_iters"] == ia[0]["inner_iters"]
        assert rel(q.x.cpu().numpy(), xa) <= 1e-12
    # tight budget: only one workspace fits at a time
    budget = max(ws) + 256
    reqs2 = [rr.Request(s["op"], s["mu"], s["k"], dev(s["B"]), rtol, seed=s["seed"]) for s in systems]
    srv = rr.Server(budget_bytes=budget, workers=4)
    tickets = [srv.submit(q) for q in reqs2]
    srv.drain()
    res2 = [srv.poll(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert stats["peak_bytes"] <= budget
    spans = sorted((r["start_ms"], r["end_ms"]) for r in res2)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-6          # no two requests resident at once
    for q, q2 in zip(reqs, reqs2):
        assert torch.equal(q.x, q2.x)


def test_server_rejects_request_larger_than_budget(cuda_lib):
    rr = cuda_lib
    s = kernel_system(rr, 30, 1000, m=1)
    q = rr.Request(s["op"], s["mu"], s["k"], dev(s["B"]), 1e-6, seed=s["seed"])
    srv = rr.Server(budget_bytes=q.workspace_bytes() // 2, workers=1)
    with pytest.raises(rr.RandRandError) as e:
        srv.submit(q)
    assert e.value.status == rr.RR_ERR_WORKSPACE
    srv.close()


def _rounds_check(rr, systems, reqs, res, rtol):
    for s, q, r in zip(systems, reqs, res):
        assert r["status"] == rr.RR_OK
        assert r["rounds"] == 1                     # iterated in the shared rounds
        x = q.x.cpu().numpy()
        assert np.all(O.true_rel_residual(s["oracle"], s["mu"], x, s["B"]) <= rtol)
        xa, sa, ia = alone(rr, s, rtol)
        assert sa == rr.RR_OK
        # the grouped product and step sum in another order (float32
        # rounding): iteration counts within a few steps, solutions within
        # the forward error both solves have at this rtol
        for a, b in zip([i["inner_iters"] for i in r["info"]], [i["inner_iters"] for i in ia]):
            assert abs(a - b) <= max(3, 0.05 * b)
        assert rel(x, xa) <= 1e-5


def test_batch_in_shared_rounds_equals_systems_solved_alone(cuda_lib):
    rr = cuda_lib
    sizes = [600, 2000, 900, 1500, 1200, 777, 2600, 1000]
    systems = [kernel_system(rr, 40 + i, n) for i, n in enumerate(sizes)]
    rtol = 1e-6
    reqs = [rr.Request(s["op"], s["mu"], s["k"], dev(s["B"]), rtol, seed=s["seed"]) for s in systems]
    st, res = rr.solve_batch(reqs, workers=4, rounds=rr.batch_rounds_opts(reqs))
    assert st == rr.RR_OK, res
    _rounds_check(rr, systems, reqs, res, rtol)


def test_server_shared_rounds_continuous_batching(cuda_lib):
    """Requests that arrive while others iterate join the running rounds:
    at least two are resident in the rounds at once, and each result is the
    one the system has alone (within the stated tolerance)."""
    import time
    rr = cuda_lib
    rtol = 1e-6
    sizes = [1800, 700, 1300, 2200, 900, 1600]
    systems = [kernel_system(rr, 60 + i, n) for i, n in enumerate(sizes)]
    reqs = [rr.Request(s["op"], s["mu"], s["k"], dev(s["B"]), rtol, seed=s["seed"]) for s in systems]
    ws = sum(q.workspace_bytes() + 256 for q in reqs)
    srv = rr.Server(budget_bytes=ws, workers=3, rounds=rr.batch_rounds_opts(reqs))
    tickets = []
    for i, q in enumerate(reqs):
        tickets.append(srv.submit(q))
        if i == 2:
            time.sleep(0.05)                        # later arrivals join running rounds
    res = [srv.poll(t, wait=True) for t in tickets]
    peak = srv.peak_running()
    srv.close()
    assert peak >= 2
    spans = sorted((r["start_ms"], r["end_ms"]) for r in res)
    assert any(s1 < e0 for (s0, e0), (s1, e1) in zip(spans, spans[1:]))
    _rounds_check(rr, systems, reqs, res, rtol)
