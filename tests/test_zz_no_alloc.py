"""The allocation-free kernel product (randrand_kernel_matvec_noalloc).

It serves callers that cannot allocate device memory where they call the
library (a plugin inside a framework that owns all device memory, a serving
loop that bans allocator calls): its scratch is a fixed static device array.
Checked through the C ABI against the float64 definition of (K + mu I) V and
against the existing float64-accurate product of a mixed-precision handle
(randrand_matvec), on calls in a row with different sizes, because the
static array keeps the previous call's contents: a large call that has to
use fewer column splits to fit the array, then a small one, then the large
one again.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from workloads import generators as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def kernel_rows_f64(X, rows, V, mu, bw):
    """(K + mu I) V and sum_j |K_ij V_j| on the given rows, K_ij =
    exp(-|x_i - x_j|^2 / (2 bw^2)) in float64 from the float32 points."""
    X = X.astype(np.float64)
    out, scale = [], []
    for c in range(0, len(rows), 16):
        ii = rows[c:c + 16]
        K = np.exp(-((X[ii, None, :] - X[None, :, :]) ** 2).sum(-1) / (2 * bw * bw))
        out.append(K @ V + mu * V[ii])
        scale.append(np.abs(K) @ np.abs(V) + mu * np.abs(V[ii]))
    return np.concatenate(out), np.concatenate(scale)


# (n, m, bandwidth): 150000 points with 8 columns need fewer column splits
# than the default to fit the 32 MiB array; 3001 points use the default
CASES = [(150_000, 8, 1.0), (3001, 3, 1.2), (150_000, 8, 1.0)]


def test_noalloc_kernel_product_matches_definition_and_handle(cuda_lib):
    rr = cuda_lib
    mu = 1e-3
    stream = torch.cuda.current_stream()
    for call, (n, m, bw) in enumerate(CASES):
        Xh = W.mixture_points(n, seed=41 + n)
        X = torch.from_numpy(Xh).cuda()
        V = np.random.default_rng(100 + call).standard_normal((n, m))
        Vc = torch.from_numpy(np.ascontiguousarray(V.T)).cuda()        # column-major n x m
        Wn = torch.full_like(Vc, float("nan"))
        s = rr.randrand_kernel_matvec_noalloc(X.data_ptr(), n, X.shape[1], bw, mu, Vc.data_ptr(),
                                              Wn.data_ptr(), m, n, stream.cuda_stream)
        assert s == rr.RR_OK
        stream.synchronize()
        got = Wn.t().cpu().numpy()
        assert np.all(np.isfinite(got))
        # the float64 definition: every row when small, else sampled rows and
        # the ragged last block
        rows = (np.arange(n) if n <= 4000 else
                np.concatenate([np.random.default_rng(call).choice(n - 300, 96, replace=False),
                                np.arange(n - 64, n)]))
        # double-float accumulation: ~1e-11 of the row magnitude at a few
        # thousand terms, a few times that over 150000 terms
        tol = 1e-11 if n <= 4000 else 5e-11
        ref, scale = kernel_rows_f64(Xh, rows, V, mu, bw)
        assert np.max(np.abs(got[rows] - ref) / scale) <= tol
        # the existing entry point: the handle's float64-accurate product, on
        # every row; each side is within tol of the row magnitude
        # sum_j K_ij |v_j| + mu |v_i| (K >= 0: the product of |V|)
        h = rr.Handle(rr.Operator.gauss_kernel(X, bw), mu, 16, "gaussian", seed=41,
                      precision="mixed", max_rhs=m)
        ref_h = h.matvec(torch.from_numpy(V).cuda()).cpu().numpy()
        mag = h.matvec(torch.from_numpy(np.abs(V)).cuda()).cpu().numpy()
        h.close()
        assert np.max(np.abs(got - ref_h) / mag) <= 2 * tol


def test_noalloc_rejects_sizes_beyond_the_static_array(cuda_lib):
    rr = cuda_lib
    n = 400_000                       # 8 columns need > 32 MiB of scratch
    X = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    V = torch.zeros((8, n), dtype=torch.float64, device="cuda")
    s = rr.randrand_kernel_matvec_noalloc(X.data_ptr(), n, 8, 1.0, 0.0, V.data_ptr(), V.data_ptr(),
                                          8, n, torch.cuda.current_stream().cuda_stream)
    assert s == rr.RR_ERR_WORKSPACE
    s = rr.randrand_kernel_matvec_noalloc(X.data_ptr(), n, 8, -1.0, 0.0, V.data_ptr(), V.data_ptr(),
                                          1, n, torch.cuda.current_stream().cuda_stream)
    assert s == rr.RR_ERR_INVALID_ARG
