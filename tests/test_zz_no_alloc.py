"""The allocation-free kernel product (randrand_kernel_matvec_noalloc).

It serves callers that cannot allocate device memory where they call the
library (a plugin inside a framework that owns all device memory, a serving
loop that bans allocator calls): its scratch is a fixed static device array.
Checked through the C ABI against the existing float64-accurate product of a
mixed-precision handle (randrand_matvec), on two calls in a row, because the
static array keeps the previous call's contents.  This file is collected
last on purpose.
"""
import numpy as np
import pytest

from workloads import generators as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_kernel_product_matches_handle_product(cuda_lib):
    rr = cuda_lib
    n, m, mu, bw = 3001, 3, 1e-3, 1.2
    X = torch.from_numpy(W.mixture_points(n, seed=41)).cuda()
    h = rr.Handle(rr.Operator.gauss_kernel(X, bw), mu, 16, "gaussian", seed=41,
                  precision="mixed", max_rhs=m)
    stream = torch.cuda.current_stream()
    for call in range(2):
        V = np.random.default_rng(100 + call).standard_normal((n, m))
        Vc = torch.from_numpy(np.ascontiguousarray(V.T)).cuda()        # column-major n x m
        Wn = torch.full_like(Vc, float("nan"))
        s = rr.randrand_kernel_matvec_noalloc(X.data_ptr(), n, X.shape[1], bw, mu, Vc.data_ptr(),
                                              Wn.data_ptr(), m, n, stream.cuda_stream)
        assert s == rr.RR_OK
        stream.synchronize()
        ref = h.matvec(torch.from_numpy(V).cuda()).cpu().numpy()
        got = Wn.t().cpu().numpy()
        scale = np.abs(ref).max()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= 1e-11 * scale


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
