"""Host-side arithmetic of the benchmark line (no GPU): the roofline of each
dominant kernel and the launch count it claims.

The units are fixed by what each kernel computes: the tensor-core kernel
product evaluates each of the n^2 entries of the Gaussian kernel with exactly
one exponential, the symmetric double-float residual visits n (n + 1) / 2
distinct entries, and the kernel sketch is a dense n x n x k product (2 n^2 k
flops)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_matvec_roofline_counts_one_exponential_per_entry():
    # 200 launches in 19.36 ms (96.8 us each) at n = 20000 and a 2070 MHz
    # maximum clock: 4.0e8 exponentials per 96.8 us against 152 x 32 per clock
    r = bench.roofline("matvec", (200, 19.36), {"sm_max_mhz": 2070.0})
    assert r["kernel"] == "k_kernel_mv_tc" and r["bound"] == "alu"
    assert r["avg_us"] == pytest.approx(96.8)
    assert r["achieved"] == pytest.approx(4.0e8 / 96.8e-6 / 1e9)
    assert r["peak"] == pytest.approx(152 * 32 * 2.07e9 / 1e9)
    assert r["frac"] == pytest.approx(0.4104, abs=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # the power iterations run the same kernel: same units
    assert bench.roofline("power", (200, 19.36), {"sm_max_mhz": 2070.0})["frac"] == r["frac"]


def test_residual_roofline_counts_the_distinct_entries_of_symmetric_K():
    n, m = bench.WORKLOAD["n"], bench.WORKLOAD["nrhs"]
    r = bench.roofline("residual", (3, 5.49), {"sm_max_mhz": 2070.0})
    assert r["kernel"] == "k_kernel_mv_df2s"
    entries = n * (n + 1) // 2
    assert entries == 200010000
    ops = entries * (142 + 24 * m)
    assert r["achieved"] == pytest.approx(ops / 1.83e-3 / 1e9)
    assert r["peak"] == pytest.approx(152 * 128 * 2.07e9 / 1e9)
    assert 0.0 < r["frac"] < 1.0


def test_sketch_roofline_is_a_dense_contraction_against_measured_bf16():
    n, k = bench.WORKLOAD["n"], bench.WORKLOAD["k"]
    r = bench.roofline("sketch", (1, 0.58), {"sm_max_mhz": 2070.0})
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(2.0 * n * n * k / 0.58e-3 / 1e12)
    assert r["peak"] == pytest.approx(bench._peaks()["bf16"])
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_missing_clock_sample_falls_back_to_the_maximum_clock():
    a = bench.roofline("matvec", (10, 1.0), {})
    b = bench.roofline("matvec", (10, 1.0), {"sm_max_mhz": 2070.0})
    assert a["peak"] == pytest.approx(b["peak"])


def test_launch_estimate_per_solve():
    # one solve: 180 PCG products, 40 power-iteration products, 3 restart
    # residuals, one sketch launch
    p = {"matvec": (180, 0.0), "power": (40, 0.0), "residual": (3, 0.0), "sketch": (1, 0.0)}
    assert bench.estimate_launches([(p, [])]) == 180 * 2 + 40 * 3 + 3 * 4 + 150 + 1
    assert bench.estimate_launches([(p, [])], variant="R") == 180 * 3 + 40 * 3 + 3 * 4 + 150 + 1
    assert bench.estimate_launches([(p, []), (p, [])]) == 2 * (180 * 2 + 40 * 3 + 3 * 4 + 150 + 1)


def test_json_line_carries_the_contract_keys():
    class A:
        steps, warmup = 20, 3

    line = bench._line(A, 1, bench.METRIC, 25.3, "solves/s", 39.5, {"workload": "w"},
                       roofline={"frac": 0.41})
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in line
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["roofline"] == {"frac": 0.41}


def test_sparse_iteration_bytes_of_the_diffusion_stencil():
    # 512 x 512 five-point stencil: n = 262144 rows, 5 n - 4 * 512 nonzeros
    # (the boundary rows miss one neighbour per edge they touch); gamma = 8
    side = 512
    n = side * side
    nnz = 5 * n - 4 * side
    product = 8 * nnz + 4 * (n + 1) + 2 * 4 * n        # values+indices, rowptr, v in, w out
    patterns = 2 * 5 * 8 * n                            # Omega^T and Omega: 8 x (4 + 1) B per row
    vectors = 10 * 4 * n
    expect = 3 * product + patterns + vectors
    assert expect == 72302604
    assert bench.sparse_iteration_bytes(nnz, n, 8, 1) == pytest.approx(expect, rel=0, abs=0)
    # the generator's matrix has that many nonzeros
    from workloads import generators as W
    C = W.diffusion_csr(side=64, seed=0x52523)
    assert len(C.vals) == 5 * 64 * 64 - 4 * 64
