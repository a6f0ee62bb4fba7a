"""The C-ABI library builds, loads and exports every symbol the header
declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "randrand.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(\w+)\s*\(", src, flags=re.M)
    return sorted({n for n in names if n.startswith(("randrand_", "rr_"))})


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_19747_gb300 as rr
    return rr


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("randrand_build", "randrand_solve", "randrand_workspace_bytes", "randrand_free",
                 "randrand_status_str", "rr_build_opts_default"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    cdll = lib.load_library()
    for name in declared_functions():
        assert hasattr(cdll, name), f"{name} declared in randrand.h but not exported"


def test_struct_layouts_match_header(lib):
    # sizes the C compiler gives the header structs (checked by a tiny host program)
    import subprocess
    import tempfile
    src = r'''
    #include <stdio.h>
    #include <stddef.h>
    #include "randrand.h"
    int main(void){
      printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(rr_operator), sizeof(rr_build_opts),
             sizeof(rr_solve_info), offsetof(rr_operator, bandwidth), offsetof(rr_build_opts, rho),
             sizeof(rr_request), sizeof(rr_result), offsetof(rr_request, rtol),
             offsetof(rr_result, info));
      return 0; }
    '''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = list(map(int, out))
    assert sizes[0] == ctypes.sizeof(lib.rr_operator)
    assert sizes[1] == ctypes.sizeof(lib.rr_build_opts)
    assert sizes[2] == ctypes.sizeof(lib.rr_solve_info)
    assert sizes[3] == lib.rr_operator.bandwidth.offset
    assert sizes[4] == lib.rr_build_opts.rho.offset
    assert sizes[5] == ctypes.sizeof(lib.rr_request)
    assert sizes[6] == ctypes.sizeof(lib.rr_result)
    assert sizes[7] == lib.rr_request.rtol.offset
    assert sizes[8] == lib.rr_result.info.offset


def test_defaults_and_status_strings(lib):
    o = lib.rr_build_opts_default()
    assert (o.gamma, o.power_iters, o.max_rhs, o.restart_eta) == (8, 20, 1, 1e-2)
    assert lib.randrand_status_str(lib.RR_OK) == "ok"
    assert "invalid" in lib.randrand_status_str(lib.RR_ERR_INVALID_ARG)
    assert lib.randrand_status_str(999) == "unknown status"


def test_workspace_query_and_argument_checks(lib):
    # host-only entry point: works without a GPU, touches no device memory
    op = lib.rr_operator(kind=lib.RR_OP_GAUSS_KERNEL, dtype=1, n=20000, points=0x1000, dim=8,
                         bandwidth=1.0)
    o = lib.rr_build_opts_default()
    o.precision = lib.RR_PREC_MIXED
    o.max_rhs = 4
    nbytes = lib.randrand_workspace_bytes(op, 500, o)
    # at least Omega, Y and Q in float32 plus the k x k float64 work matrices
    assert nbytes >= 3 * 20000 * 500 * 4 + 12 * 500 * 500 * 8
    for bad_k in (0, 20001):
        with pytest.raises(lib.RandRandError) as e:
            lib.randrand_workspace_bytes(op, bad_k, o)
        assert e.value.status == lib.RR_ERR_INVALID_ARG
    o.max_rhs = 9
    with pytest.raises(lib.RandRandError):
        lib.randrand_workspace_bytes(op, 10, o)
    o.max_rhs = 1
    bad = lib.rr_operator(kind=lib.RR_OP_GAUSS_KERNEL, dtype=1, n=100, points=0, dim=8, bandwidth=1.0)
    with pytest.raises(lib.RandRandError):
        lib.randrand_workspace_bytes(bad, 10, o)
    dense = lib.rr_operator(kind=lib.RR_OP_DENSE, dtype=0, n=100, dense=0x1000, ld=50)
    with pytest.raises(lib.RandRandError):
        lib.randrand_workspace_bytes(dense, 10, o)


def test_build_rejects_bad_arguments_before_any_launch(lib):
    op = lib.rr_operator(kind=lib.RR_OP_DENSE, dtype=0, n=100, dense=0x1000, ld=100)
    o = lib.rr_build_opts_default()
    for mu in (-1.0, float("nan"), float("inf")):
        with pytest.raises(lib.RandRandError) as e:
            lib.randrand_build(op, mu, 10, 0, 1, o, 0x100000, 1 << 30, 0)
        assert e.value.status == lib.RR_ERR_INVALID_ARG
    with pytest.raises(lib.RandRandError) as e:     # misaligned workspace
        lib.randrand_build(op, 0.0, 10, 0, 1, o, 0x100001, 1 << 30, 0)
    assert e.value.status == lib.RR_ERR_INVALID_ARG
    with pytest.raises(lib.RandRandError) as e:     # workspace too small
        lib.randrand_build(op, 0.0, 10, 0, 1, o, 0x100000, 16, 0)
    assert e.value.status == lib.RR_ERR_WORKSPACE
    with pytest.raises(lib.RandRandError) as e:     # unknown sketch kind
        lib.randrand_build(op, 0.0, 10, 7, 1, o, 0x100000, 1 << 30, 0)
    assert e.value.status == lib.RR_ERR_INVALID_ARG


def test_multilevel_options_on_the_host(lib):
    """rr_multilevel_defaults gives the paper's sparse + Gaussian sizes (the
    same reading as the oracle); the factors enlarge the workspace; a
    multi-level build without them, or with sizes out of range, is rejected
    before any launch."""
    from oracle import philox
    op = lib.rr_operator(kind=lib.RR_OP_GAUSS_KERNEL, dtype=1, n=20000, points=0x1000, dim=8,
                         bandwidth=1.0)
    o = lib.rr_build_opts_default()
    o.precision = lib.RR_PREC_MIXED
    assert (o.ml_l1, o.ml_gamma) == (0, 0)
    base = lib.randrand_workspace_bytes(op, 500, o)
    for n, k in ((20000, 500), (3001, 80), (262144, 256), (2, 1), (10 ** 9, 100)):
        lib.set_multilevel(o, "multilevel", n, k)
        assert (o.ml_l1, o.ml_gamma) == philox.multilevel_defaults(n, k)
    lib.set_multilevel(o, "multilevel", 20000, 500)
    assert lib.randrand_workspace_bytes(op, 500, o) >= base + 5000 * 500 * 8
    plain = lib.rr_build_opts_default()
    dense = lib.rr_operator(kind=lib.RR_OP_DENSE, dtype=0, n=100, dense=0x1000, ld=100)
    with pytest.raises(lib.RandRandError) as e:      # nothing reserved for the factors
        lib.randrand_build(dense, 0.0, 10, lib.RR_SKETCH_MULTILEVEL, 1, plain, 0x100000, 1 << 30, 0)
    assert e.value.status == lib.RR_ERR_INVALID_ARG
    for l1, g in ((5, 2), (100, 0), (100, 17), (8, 9)):   # l1 < k, gamma1 outside 1..16 or > l1
        bad = lib.rr_build_opts_default()
        bad.ml_l1, bad.ml_gamma = l1, g
        with pytest.raises(lib.RandRandError) as e:
            lib.randrand_workspace_bytes(dense, 8 if l1 == 8 else 10, bad)
        assert e.value.status == lib.RR_ERR_INVALID_ARG


def test_refine_option_checks(lib):
    dense = lib.rr_operator(kind=lib.RR_OP_DENSE, dtype=0, n=100, dense=0x1000, ld=100)
    o = lib.rr_build_opts_default()
    assert o.refine == 0
    o.refine = 1
    assert lib.randrand_workspace_bytes(dense, 10, o) > 0
    o.refine = 8                     # eq:accurate_proj_2 with 8 refinement steps
    assert lib.randrand_workspace_bytes(dense, 10, o) > 0
    for bad in (9, -1):
        o.refine = bad
        with pytest.raises(lib.RandRandError) as e:
            lib.randrand_workspace_bytes(dense, 10, o)
        assert e.value.status == lib.RR_ERR_INVALID_ARG
    o.refine, o.variant = 1, lib.RR_VARIANT_R
    with pytest.raises(lib.RandRandError) as e:
        lib.randrand_workspace_bytes(dense, 10, o)
    assert e.value.status == lib.RR_ERR_UNSUPPORTED


def test_shift_and_variant_G_option_checks(lib):
    """keep_sketch (Sec. 5.1: 1 = Gram separation, 2 = joint basis) and the
    basis-less G-RandRAND form are checked on the host, before any launch."""
    n, k = 100, 10
    dense = lib.rr_operator(kind=lib.RR_OP_DENSE, dtype=0, n=n, dense=0x1000, ld=n)
    o = lib.rr_build_opts_default()
    ws = {}
    for ks in (0, 1, 2):
        o.keep_sketch = ks
        ws[ks] = lib.randrand_workspace_bytes(dense, k, o)
    # the joint basis keeps Q_joint (n x 2k) beyond what the Gram separation keeps
    assert ws[2] >= ws[1] + n * 2 * k * 8 and ws[1] > ws[0]
    for bad in (-1, 3):
        o.keep_sketch = bad
        with pytest.raises(lib.RandRandError) as e:
            lib.randrand_workspace_bytes(dense, k, o)
        assert e.value.status == lib.RR_ERR_INVALID_ARG
    for ks in (1, 2):
        for field, value in (("variant", lib.RR_VARIANT_R), ("orth", lib.RR_ORTH_RAND_CHOLQR),
                             ("q", 1)):
            o = lib.rr_build_opts_default()
            o.keep_sketch = ks
            setattr(o, field, value)
            with pytest.raises(lib.RandRandError) as e:
                lib.randrand_workspace_bytes(dense, k, o)
            assert e.value.status == lib.RR_ERR_UNSUPPORTED, (ks, field)
    # G-RandRAND with Alg. 3: only basis-less (CSR), with room for its
    # MINRES temporaries (2 x padded columns) in the unused basis array
    g = lib.rr_build_opts_default()
    g.variant, g.orth = lib.RR_VARIANT_G, lib.RR_ORTH_RAND_CHOLQR
    with pytest.raises(lib.RandRandError) as e:
        lib.randrand_workspace_bytes(dense, k, g)
    assert e.value.status == lib.RR_ERR_UNSUPPORTED
    csr = lib.rr_operator(kind=lib.RR_OP_CSR, dtype=0, n=n, rowptr=0x1000, colidx=0x2000,
                          vals=0x3000, nnz=3 * n)
    g.max_rhs = 4                                   # 4 columns: k >= 8 needed
    assert lib.randrand_workspace_bytes(csr, 8, g) > 0
    with pytest.raises(lib.RandRandError) as e:
        lib.randrand_workspace_bytes(csr, 7, g)
    assert e.value.status == lib.RR_ERR_UNSUPPORTED


def test_oracle_not_imported_by_product():
    # the product path never imports the oracle
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2509_19747_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_arena_first_fit_and_coalescing(lib):
    """The serving loop's HBM-budget allocator (host only)."""
    a = lib.Arena(10 * 256 + 100)             # usable: 10 blocks of 256 bytes
    assert a.stats() == (0, 2560)
    o1 = a.alloc(256)
    o2 = a.alloc(300)                          # rounds up to 512
    o3 = a.alloc(256)
    assert (o1, o2, o3) == (0, 256, 768)
    assert a.stats() == (1024, 1536)
    assert a.alloc(2000) is None               # larger than any free block
    a.free(o2)
    assert a.alloc(512) == 256                 # first fit reuses the hole
    a.free(256)
    a.free(o1)                                 # coalesces with the hole after it
    assert a.stats() == (256, 1536)
    assert a.alloc(768) == 0
    a.free(0)
    a.free(o3)                                 # everything merges back
    assert a.stats() == (0, 2560)
    with pytest.raises(lib.RandRandError):
        a.free(12345)                          # not an allocated offset
    a.close()


def test_arena_random_sequence_matches_model(lib):
    """Random alloc/free sequences against a plain list model of first fit."""
    import random
    rng = random.Random(7)
    nblk = 64
    a = lib.Arena(nblk * 256)
    owner = [None] * nblk                      # model: which allocation holds each block
    live = {}
    for step in range(2000):
        if live and rng.random() < 0.45:
            off = rng.choice(list(live))
            a.free(off)
            for b in range(off // 256, off // 256 + live.pop(off)):
                owner[b] = None
        else:
            want = rng.randint(1, 8)
            got = a.alloc(want * 256 - rng.randint(0, 255))
            exp = None
            for s in range(nblk - want + 1):
                if all(owner[b] is None for b in range(s, s + want)):
                    exp = s
                    break
            assert (got is None) == (exp is None)
            if got is not None:
                assert got == exp * 256
                for b in range(exp, exp + want):
                    owner[b] = got
                live[got] = want
        used, largest = a.stats()
        assert used == 256 * sum(live.values())
    a.close()


def test_server_rejects_bad_arguments_without_gpu_work(lib):
    import ctypes as C
    s = C.c_void_p(None)
    cdll = lib.load_library()
    assert cdll.rr_server_create(None, 1 << 20, 2, C.byref(s)) == lib.RR_ERR_INVALID_ARG
    assert cdll.rr_server_create(C.c_void_p(0x100001), 1 << 20, 2, C.byref(s)) == lib.RR_ERR_INVALID_ARG
    assert cdll.rr_server_create(C.c_void_p(0x100000), 1 << 20, 0, C.byref(s)) == lib.RR_ERR_INVALID_ARG
    res = (lib.rr_result * 1)()
    assert cdll.randrand_solve_batch(None, 1, C.c_void_p(0x100000), 1 << 20, 1, res) == lib.RR_ERR_INVALID_ARG
