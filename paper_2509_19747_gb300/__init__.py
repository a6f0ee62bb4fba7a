"""Python binding of the GB300 RandRAND-PCG library (include/randrand.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``lib/librandrand.so``.  PyTorch provides device memory and streams; the
binding passes raw pointers through the C ABI.  The functions named
``randrand_*`` / ``rr_*`` mirror the C entry points one to one; ``Operator``
and ``Handle`` are small conveniences on top of them.

Importing this package loads the compiled library and raises if it is missing:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

from .build import lib_path

__all__ = [
    "RR_OK", "RR_ERR_INVALID_ARG", "RR_ERR_WORKSPACE", "RR_ERR_NOT_SPD", "RR_ERR_BREAKDOWN",
    "RR_ERR_MAXIT", "RR_ERR_TIMEOUT", "RR_ERR_CUDA", "RR_ERR_UNSUPPORTED", "RR_PENDING",
    "RR_OP_DENSE", "RR_OP_CSR", "RR_OP_GAUSS_KERNEL", "RR_SKETCH_GAUSSIAN",
    "RR_SKETCH_SPARSE_SIGN", "RR_SKETCH_SRHT", "RR_SKETCH_MULTILEVEL", "RR_PREC_FP64", "RR_PREC_FP32", "RR_PREC_MIXED", "RR_VARIANT_C",
    "RR_VARIANT_R", "RR_VARIANT_G", "rr_operator", "rr_build_opts", "rr_solve_info", "rr_profile", "RandRandError",
    "load_library", "Operator", "Handle", "rr_request", "rr_result", "Arena", "Server",
    "Request", "solve_batch",
]

RR_OK, RR_ERR_INVALID_ARG, RR_ERR_WORKSPACE, RR_ERR_NOT_SPD, RR_ERR_BREAKDOWN = 0, 1, 2, 3, 4
RR_ERR_MAXIT, RR_ERR_TIMEOUT, RR_ERR_CUDA, RR_ERR_UNSUPPORTED, RR_PENDING = 5, 6, 7, 8, 9
RR_OP_DENSE, RR_OP_CSR, RR_OP_GAUSS_KERNEL = 0, 1, 2
RR_SKETCH_GAUSSIAN, RR_SKETCH_SPARSE_SIGN, RR_SKETCH_SRHT, RR_SKETCH_MULTILEVEL = 0, 1, 2, 3
RR_PREC_FP64, RR_PREC_FP32, RR_PREC_MIXED = 0, 1, 2
RR_VARIANT_C, RR_VARIANT_R, RR_VARIANT_G = 0, 1, 2
RR_ORTH_CHOLQR2, RR_ORTH_RAND_CHOLQR = 0, 1

SKETCHES = {"gaussian": RR_SKETCH_GAUSSIAN, "sparse_sign": RR_SKETCH_SPARSE_SIGN,
            "srht": RR_SKETCH_SRHT, "multilevel": RR_SKETCH_MULTILEVEL}
PRECISIONS = {"fp64": RR_PREC_FP64, "fp32": RR_PREC_FP32, "mixed": RR_PREC_MIXED}
VARIANTS = {"C": RR_VARIANT_C, "R": RR_VARIANT_R, "G": RR_VARIANT_G}
ORTHS = {"cholqr2": RR_ORTH_CHOLQR2, "rand_cholqr": RR_ORTH_RAND_CHOLQR}


class rr_operator(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("dtype", ctypes.c_int32), ("n", ctypes.c_int64),
        ("dense", ctypes.c_void_p), ("ld", ctypes.c_int64),
        ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("vals", ctypes.c_void_p),
        ("nnz", ctypes.c_int64), ("points", ctypes.c_void_p), ("dim", ctypes.c_int32),
        ("pad_", ctypes.c_int32), ("bandwidth", ctypes.c_double),
    ]


class rr_build_opts(ctypes.Structure):
    _fields_ = [
        ("variant", ctypes.c_int32), ("precision", ctypes.c_int32), ("orth", ctypes.c_int32),
        ("gamma", ctypes.c_int32), ("l_sk", ctypes.c_int32), ("gamma_sk", ctypes.c_int32),
        ("power_iters", ctypes.c_int32), ("max_rhs", ctypes.c_int32), ("profile", ctypes.c_int32),
        ("kernel_impl", ctypes.c_int32), ("iter_impl", ctypes.c_int32), ("q", ctypes.c_int32),
        ("rho", ctypes.c_double),
        ("restart_eta", ctypes.c_double),
        ("keep_sketch", ctypes.c_int32),
        ("ml_l1", ctypes.c_int32), ("ml_gamma", ctypes.c_int32), ("refine", ctypes.c_int32),
    ]


RR_PROF_SKETCH, RR_PROF_MATVEC, RR_PROF_RESIDUAL, RR_PROF_POWER, RR_PROF_COUNT = 0, 1, 2, 3, 8


class rr_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int32 * RR_PROF_COUNT), ("ms", ctypes.c_double * RR_PROF_COUNT)]


class rr_solve_info(ctypes.Structure):
    _fields_ = [
        ("inner_iters", ctypes.c_int32), ("outer_iters", ctypes.c_int32),
        ("matvecs", ctypes.c_int32), ("status", ctypes.c_int32),
        ("rel_residual", ctypes.c_double), ("tau", ctypes.c_double),
        ("normE", ctypes.c_double), ("lam_max", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class rr_request(ctypes.Structure):
    _fields_ = [
        ("op", rr_operator), ("mu", ctypes.c_double), ("k", ctypes.c_int32),
        ("sketch", ctypes.c_int32), ("seed", ctypes.c_uint64), ("opts", rr_build_opts),
        ("b", ctypes.c_void_p), ("x", ctypes.c_void_p), ("ldb", ctypes.c_int64),
        ("ldx", ctypes.c_int64), ("nrhs", ctypes.c_int32), ("maxit", ctypes.c_int32),
        ("rtol", ctypes.c_double),
    ]


class rr_group_rhs(ctypes.Structure):
    _fields_ = [
        ("b", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("x", ctypes.c_void_p),
        ("ldx", ctypes.c_int64), ("nrhs", ctypes.c_int32), ("maxit", ctypes.c_int32),
        ("rtol", ctypes.c_double),
    ]


class rr_rounds_opts(ctypes.Structure):
    _fields_ = [("mp", ctypes.c_int32), ("kmax", ctypes.c_int32), ("max_systems", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("max_rows", ctypes.c_int64)]


class rr_rounds_stats(ctypes.Structure):
    _fields_ = [("replay_s", ctypes.c_double), ("restart_s", ctypes.c_double),
                ("join_s", ctypes.c_double), ("replays", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("rounds_per_replay", ctypes.c_int32), ("pad_", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad_"}


class rr_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("nrhs", ctypes.c_int32), ("ws_bytes", ctypes.c_size_t),
        ("submit_ms", ctypes.c_double), ("start_ms", ctypes.c_double), ("end_ms", ctypes.c_double),
        ("queue_ms", ctypes.c_double), ("build_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
        ("info", rr_solve_info * 8), ("rounds", ctypes.c_int32), ("pad_", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("info", "pad_")}
        d["info"] = [self.info[i].as_dict() for i in range(self.nrhs)]
        return d


class RandRandError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {randrand_status_str(status)} (status {status})")


_LIB = None

# (name, restype, argtypes) of every exported entry point
_SIGNATURES = [
    ("rr_build_opts_default", None, [ctypes.POINTER(rr_build_opts)]),
    ("rr_multilevel_defaults", None, [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(rr_build_opts)]),
    ("randrand_status_str", ctypes.c_char_p, [ctypes.c_int32]),
    ("randrand_workspace_bytes", ctypes.c_int32,
     [ctypes.POINTER(rr_operator), ctypes.c_int32, ctypes.POINTER(rr_build_opts),
      ctypes.POINTER(ctypes.c_size_t)]),
    ("randrand_build", ctypes.c_int32,
     [ctypes.POINTER(rr_operator), ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
      ctypes.c_uint64, ctypes.POINTER(rr_build_opts), ctypes.c_void_p, ctypes.c_size_t,
      ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("randrand_solve", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
      ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
      ctypes.POINTER(rr_solve_info)]),
    ("randrand_solve_host", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
      ctypes.c_int64, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(rr_solve_info)]),
    ("randrand_free", None, [ctypes.c_void_p]),
    ("randrand_set_mu", ctypes.c_int32, [ctypes.c_void_p, ctypes.c_double]),
    ("randrand_export", ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    ("randrand_scalars", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
      ctypes.POINTER(ctypes.c_double)]),
    ("randrand_core_jitter", ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("randrand_group_workspace_bytes", ctypes.c_int32,
     [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    ("randrand_solve_group", ctypes.c_int32,
     [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.POINTER(rr_group_rhs),
      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(rr_solve_info)]),
    ("randrand_apply", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    ("randrand_profile", ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(rr_profile)]),
    ("randrand_kernel_matvec_noalloc", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p]),
    ("randrand_matvec", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    ("randrand_apply_operator", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    ("rr_arena_create", ctypes.c_int32, [ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    ("rr_arena_alloc", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    ("rr_arena_free", ctypes.c_int32, [ctypes.c_void_p, ctypes.c_size_t]),
    ("rr_arena_stats", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    ("rr_arena_destroy", None, [ctypes.c_void_p]),
    ("rr_rounds_workspace_bytes", ctypes.c_int32,
     [ctypes.POINTER(rr_rounds_opts), ctypes.POINTER(ctypes.c_size_t)]),
    ("rr_server_create_rounds", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(rr_rounds_opts),
      ctypes.POINTER(ctypes.c_void_p)]),
    ("rr_server_peak_running", ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    ("randrand_solve_batch_rounds", ctypes.c_int32,
     [ctypes.POINTER(rr_request), ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32,
      ctypes.POINTER(rr_rounds_opts), ctypes.POINTER(rr_result), ctypes.POINTER(rr_rounds_stats)]),
    ("rr_server_rounds_stats", ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(rr_rounds_stats)]),
    ("rr_server_create", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    ("rr_server_submit", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.POINTER(rr_request), ctypes.POINTER(ctypes.c_uint64)]),
    ("rr_server_poll", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(rr_result)]),
    ("rr_server_drain", ctypes.c_int32, [ctypes.c_void_p]),
    ("rr_server_stats", ctypes.c_int32,
     [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
      ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    ("rr_server_destroy", None, [ctypes.c_void_p]),
    ("randrand_solve_batch", ctypes.c_int32,
     [ctypes.POINTER(rr_request), ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32,
      ctypes.POINTER(rr_result)]),
]


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load librandrand.so (built in-tree by build.py); raises if it is missing."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or lib_path()
    if not os.path.exists(p):
        raise RuntimeError(
            f"{p} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(p)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _LIB = lib
    return lib


def _lib() -> ctypes.CDLL:
    return load_library()


# ------------------------------------------------------------ C entry points
def set_multilevel(o: rr_build_opts, sketch: str, n: int, k: int, ml_l1: int = 0,
                   ml_gamma: int = 0) -> None:
    """Reserve the multi-level factors in o when the sketch is "multilevel":
    the given sizes, else rr_multilevel_defaults (argument marshalling)."""
    if sketch != "multilevel":
        return
    _lib().rr_multilevel_defaults(int(n), int(k), ctypes.byref(o))
    if ml_gamma:
        o.ml_gamma = int(ml_gamma)
    if ml_l1:
        o.ml_l1 = int(ml_l1)


def rr_build_opts_default() -> rr_build_opts:
    o = rr_build_opts()
    _lib().rr_build_opts_default(ctypes.byref(o))
    return o


def randrand_status_str(s: int) -> str:
    return _lib().randrand_status_str(int(s)).decode()


def randrand_workspace_bytes(op: rr_operator, k: int, opts: rr_build_opts) -> int:
    out = ctypes.c_size_t(0)
    s = _lib().randrand_workspace_bytes(ctypes.byref(op), int(k), ctypes.byref(opts), ctypes.byref(out))
    if s != RR_OK:
        raise RandRandError(s, "randrand_workspace_bytes")
    return int(out.value)


def randrand_build(op, mu, k, sketch, seed, opts, workspace_ptr, ws_bytes, stream_ptr):
    h = ctypes.c_void_p(None)
    s = _lib().randrand_build(ctypes.byref(op), float(mu), int(k), int(sketch),
                              int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(opts),
                              ctypes.c_void_p(workspace_ptr), int(ws_bytes),
                              ctypes.c_void_p(stream_ptr), ctypes.byref(h))
    if s != RR_OK:
        raise RandRandError(s, "randrand_build")
    return h


def randrand_solve(h, b_ptr, nrhs, ldb, x_ptr, ldx, x_is_guess, rtol, maxit):
    infos = (rr_solve_info * nrhs)()
    s = _lib().randrand_solve(h, ctypes.c_void_p(b_ptr), int(nrhs), int(ldb), ctypes.c_void_p(x_ptr),
                              int(ldx), int(x_is_guess), float(rtol), int(maxit), infos)
    if s not in (RR_OK, RR_ERR_MAXIT, RR_ERR_BREAKDOWN):
        raise RandRandError(s, "randrand_solve")
    return s, [i.as_dict() for i in infos]


def randrand_solve_host(h, b_host_ptr, nrhs, ldb, x_host_ptr, ldx, rtol, maxit):
    infos = (rr_solve_info * nrhs)()
    s = _lib().randrand_solve_host(h, ctypes.c_void_p(b_host_ptr), int(nrhs), int(ldb),
                                   ctypes.c_void_p(x_host_ptr), int(ldx), float(rtol), int(maxit),
                                   infos)
    if s not in (RR_OK, RR_ERR_MAXIT, RR_ERR_BREAKDOWN):
        raise RandRandError(s, "randrand_solve_host")
    return s, [i.as_dict() for i in infos]


def randrand_free(h) -> None:
    _lib().randrand_free(h)


def randrand_export(h, what: int, dst_ptr: int) -> None:
    s = _lib().randrand_export(h, int(what), ctypes.c_void_p(dst_ptr))
    if s != RR_OK:
        raise RandRandError(s, "randrand_export")


def randrand_set_mu(h, mu: float) -> None:
    s = _lib().randrand_set_mu(h, float(mu))
    if s != RR_OK:
        raise RandRandError(s, "randrand_set_mu")


def randrand_scalars(h) -> tuple[float, float, float]:
    t, e, l = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    s = _lib().randrand_scalars(h, ctypes.byref(t), ctypes.byref(e), ctypes.byref(l))
    if s != RR_OK:
        raise RandRandError(s, "randrand_scalars")
    return t.value, e.value, l.value


def randrand_core_jitter(h) -> float:
    a = ctypes.c_double()
    s = _lib().randrand_core_jitter(h, ctypes.byref(a))
    if s != RR_OK:
        raise RandRandError(s, "randrand_core_jitter")
    return a.value


def randrand_apply(h, r_ptr, z_ptr, m, ld) -> None:
    s = _lib().randrand_apply(h, ctypes.c_void_p(r_ptr), ctypes.c_void_p(z_ptr), int(m), int(ld))
    if s != RR_OK:
        raise RandRandError(s, "randrand_apply")


def randrand_profile(h) -> dict:
    p = rr_profile()
    s = _lib().randrand_profile(h, ctypes.byref(p))
    if s != RR_OK:
        raise RandRandError(s, "randrand_profile")
    names = ("sketch", "matvec", "residual", "power")
    return {nm: (int(p.launches[i]), float(p.ms[i])) for i, nm in enumerate(names)}


def randrand_apply_operator(h, v_ptr, w_ptr, m, ld) -> None:
    s = _lib().randrand_apply_operator(h, ctypes.c_void_p(v_ptr), ctypes.c_void_p(w_ptr), int(m), int(ld))
    if s != RR_OK:
        raise RandRandError(s, "randrand_apply_operator")


def randrand_matvec(h, v_ptr, w_ptr, m, ld) -> None:
    s = _lib().randrand_matvec(h, ctypes.c_void_p(v_ptr), ctypes.c_void_p(w_ptr), int(m), int(ld))
    if s != RR_OK:
        raise RandRandError(s, "randrand_matvec")


def randrand_kernel_matvec_noalloc(points_ptr, n, dim, bandwidth, mu, v_ptr, w_ptr, m, ld,
                                   stream_ptr) -> int:
    """Status of the allocation-free kernel product (raises nothing: callers
    check RR_OK / RR_ERR_WORKSPACE themselves)."""
    return int(_lib().randrand_kernel_matvec_noalloc(
        ctypes.c_void_p(points_ptr), int(n), int(dim), float(bandwidth), float(mu),
        ctypes.c_void_p(v_ptr), ctypes.c_void_p(w_ptr), int(m), int(ld), ctypes.c_void_p(stream_ptr)))


# ------------------------------------------------------------- conveniences
class Operator:
    """Device-resident operator description.  Holds references to the torch
    tensors so that the borrowed pointers stay valid."""

    def __init__(self, op: rr_operator, keep: list):
        self.c = op
        self._keep = keep
        self.n = int(op.n)

    @staticmethod
    def dense(A) -> "Operator":
        import torch
        assert A.is_cuda and A.dim() == 2 and A.shape[0] == A.shape[1] and A.is_contiguous()
        dtype = {torch.float64: 0, torch.float32: 1}[A.dtype]
        op = rr_operator(kind=RR_OP_DENSE, dtype=dtype, n=A.shape[0], dense=A.data_ptr(), ld=A.shape[1])
        return Operator(op, [A])

    @staticmethod
    def csr(rowptr, colidx, vals) -> "Operator":
        import torch
        assert rowptr.dtype == torch.int32 and colidx.dtype == torch.int32
        dtype = {torch.float64: 0, torch.float32: 1}[vals.dtype]
        op = rr_operator(kind=RR_OP_CSR, dtype=dtype, n=rowptr.numel() - 1, rowptr=rowptr.data_ptr(),
                         colidx=colidx.data_ptr(), vals=vals.data_ptr(), nnz=colidx.numel())
        return Operator(op, [rowptr, colidx, vals])

    @staticmethod
    def gauss_kernel(points, bandwidth: float = 1.0) -> "Operator":
        import torch
        assert points.is_cuda and points.dtype == torch.float32 and points.is_contiguous()
        op = rr_operator(kind=RR_OP_GAUSS_KERNEL, dtype=1, n=points.shape[0], points=points.data_ptr(),
                         dim=points.shape[1], bandwidth=float(bandwidth))
        return Operator(op, [points])


class Handle:
    """A built RandRAND preconditioner (randrand_build) and its workspace."""

    def __init__(self, op: Operator, mu: float, k: int, sketch: str = "gaussian", seed: int = 0,
                 variant: str = "C", precision: str = "fp64", max_rhs: int = 1,
                 power_iters: int = 20, rho: float = 0.0, restart_eta: float = 1e-2,
                 gamma: int = 8, profile: bool = False, kernel_impl: int = 0, stream=None,
                 orth: str = "cholqr2", l_sk: int = 0, gamma_sk: int = 8, iter_impl: int = 0,
                 q: int = 0, keep_sketch: int = 0, ml_l1: int = 0, ml_gamma: int = 0,
                 refine: int = 0):
        """sketch "multilevel": ml_l1 / ml_gamma give X1's rows and nonzeros per
        column; 0 takes rr_multilevel_defaults."""
        import torch
        self.op = op
        self.n = op.n
        self.k = k
        o = rr_build_opts_default()
        o.variant = VARIANTS[variant]
        o.precision = PRECISIONS[precision]
        o.max_rhs = max_rhs
        o.power_iters = power_iters
        o.rho = rho
        o.restart_eta = restart_eta
        o.gamma = gamma
        o.orth = ORTHS[orth]
        o.l_sk = l_sk
        o.gamma_sk = gamma_sk
        o.profile = 1 if profile else 0
        o.kernel_impl = kernel_impl
        o.iter_impl = iter_impl
        o.q = q
        o.keep_sketch = int(keep_sketch)   # True / 1: Gram separation; 2: joint basis
        o.refine = int(refine)
        set_multilevel(o, sketch, op.n, k, ml_l1, ml_gamma)
        self.opts = o
        self.ws_bytes = randrand_workspace_bytes(op.c, k, o)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = randrand_build(op.c, mu, k, SKETCHES[sketch], seed, o, self.ws.data_ptr(),
                                self.ws_bytes, self.stream.cuda_stream)

    def solve(self, b, rtol: float, maxit: int = 20000, x0=None):
        """b: (n,) or (n, m) float64 CUDA tensor.  Returns (x, status, infos)."""
        import torch
        one = b.dim() == 1
        B = b.reshape(self.n, -1)
        m = B.shape[1]
        Bc = B.t().contiguous()                      # column-major n x m
        Xc = torch.zeros_like(Bc) if x0 is None else x0.reshape(self.n, -1).t().contiguous()
        s, infos = randrand_solve(self.h, Bc.data_ptr(), m, self.n, Xc.data_ptr(), self.n,
                                  0 if x0 is None else 1, rtol, maxit)
        X = Xc.t()
        return (X[:, 0] if one else X), s, infos

    def solve_host(self, b_host, x_host, rtol: float, maxit: int = 20000):
        """b_host, x_host: (m, n) C-contiguous float64 host tensors (= column-major n x m)."""
        m = b_host.shape[0]
        return randrand_solve_host(self.h, b_host.data_ptr(), m, self.n, x_host.data_ptr(), self.n,
                                   rtol, maxit)

    def export(self, what: str):
        import torch
        code = {"omega": 0, "Q": 1, "R": 2, "G": 3}[what]
        shape = (self.n, self.k) if code < 2 else (self.k, self.k)
        out = torch.empty(shape, dtype=torch.float64, device="cuda")
        randrand_export(self.h, code, out.data_ptr())
        self.stream.synchronize()
        return out

    def scalars(self):
        return randrand_scalars(self.h)

    def core_jitter(self) -> float:
        return randrand_core_jitter(self.h)

    def set_mu(self, mu: float):
        """Rebuild for another shift from the kept sketch (keep_sketch 1 or 2)."""
        randrand_set_mu(self.h, mu)

    def profile(self) -> dict:
        return randrand_profile(self.h)

    def apply(self, r):
        import torch
        R = r.reshape(self.n, -1)
        Rc = R.t().contiguous()
        Zc = torch.empty_like(Rc)
        randrand_apply(self.h, Rc.data_ptr(), Zc.data_ptr(), Rc.shape[0], self.n)
        self.stream.synchronize()
        return Zc.t().reshape(r.shape)

    def apply_operator(self, v):
        """(A + mu I) v in the handle's working precision (float32 paths)."""
        import torch
        V = v.reshape(self.n, -1)
        Vc = V.t().contiguous()
        Wc = torch.empty_like(Vc)
        randrand_apply_operator(self.h, Vc.data_ptr(), Wc.data_ptr(), Vc.shape[0], self.n)
        self.stream.synchronize()
        return Wc.t().reshape(v.shape)

    def matvec(self, v):
        import torch
        V = v.reshape(self.n, -1)
        Vc = V.t().contiguous()
        Wc = torch.empty_like(Vc)
        randrand_matvec(self.h, Vc.data_ptr(), Wc.data_ptr(), Vc.shape[0], self.n)
        self.stream.synchronize()
        return Wc.t().reshape(v.shape)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            randrand_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



# ------------------------------------------------- many systems on one GPU
class Arena:
    """Host-side first-fit allocator over byte offsets (rr_arena_*)."""

    def __init__(self, nbytes: int):
        self.a = ctypes.c_void_p(None)
        s = _lib().rr_arena_create(int(nbytes), ctypes.byref(self.a))
        if s != RR_OK:
            raise RandRandError(s, "rr_arena_create")

    def alloc(self, nbytes: int):
        """Offset of a new block, or None when no free block is large enough."""
        off = ctypes.c_size_t(0)
        s = _lib().rr_arena_alloc(self.a, int(nbytes), ctypes.byref(off))
        if s == RR_ERR_WORKSPACE:
            return None
        if s != RR_OK:
            raise RandRandError(s, "rr_arena_alloc")
        return int(off.value)

    def free(self, offset: int):
        s = _lib().rr_arena_free(self.a, int(offset))
        if s != RR_OK:
            raise RandRandError(s, "rr_arena_free")

    def stats(self):
        used, largest = ctypes.c_size_t(0), ctypes.c_size_t(0)
        _lib().rr_arena_stats(self.a, ctypes.byref(used), ctypes.byref(largest))
        return int(used.value), int(largest.value)

    def close(self):
        if self.a.value:
            _lib().rr_arena_destroy(self.a)
            self.a = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Request:
    """One system for Server / solve_batch.  b: (n,) or (n, m) float64 CUDA
    tensor; the solution is written to ``self.x`` (same shape) on completion.
    Keeps every tensor it points to alive."""

    def __init__(self, op: Operator, mu: float, k: int, b, rtol: float, sketch: str = "gaussian",
                 seed: int = 0, maxit: int = 20000, variant: str = "C", precision: str = "mixed",
                 orth: str = "cholqr2", power_iters: int = 20, gamma: int = 8, l_sk: int = 0,
                 gamma_sk: int = 8, kernel_impl: int = 0, iter_impl: int = 0, q: int = 0,
                 ml_l1: int = 0, ml_gamma: int = 0, refine: int = 0):
        import torch
        B = b.reshape(op.n, -1)
        m = B.shape[1]
        self.shape = b.shape
        self.bc = B.t().contiguous()            # column-major n x m
        self.xc = torch.zeros_like(self.bc)
        o = rr_build_opts_default()
        o.variant = VARIANTS[variant]
        o.precision = PRECISIONS[precision]
        o.orth = ORTHS[orth]
        o.max_rhs = m
        o.power_iters = power_iters
        o.gamma = gamma
        o.l_sk = l_sk
        o.gamma_sk = gamma_sk
        o.kernel_impl = kernel_impl
        o.iter_impl = iter_impl
        o.q = q
        o.refine = int(refine)
        set_multilevel(o, sketch, op.n, k, ml_l1, ml_gamma)
        self.op = op
        self.c = rr_request(op=op.c, mu=float(mu), k=int(k), sketch=SKETCHES[sketch],
                            seed=int(seed) & 0xFFFFFFFFFFFFFFFF, opts=o, b=self.bc.data_ptr(),
                            x=self.xc.data_ptr(), ldb=op.n, ldx=op.n, nrhs=m, maxit=int(maxit),
                            rtol=float(rtol))

    @property
    def x(self):
        X = self.xc.t()
        return X.reshape(self.shape)

    def workspace_bytes(self) -> int:
        return randrand_workspace_bytes(self.op.c, self.c.k, self.c.opts)


def rounds_opts(mp: int, kmax: int, max_systems: int, max_rows: int) -> rr_rounds_opts:
    return rr_rounds_opts(mp=int(mp), kmax=int(kmax), max_systems=int(max_systems),
                          max_rows=int(max_rows))


def rounds_workspace_bytes(o: rr_rounds_opts) -> int:
    b = ctypes.c_size_t(0)
    st = _lib().rr_rounds_workspace_bytes(ctypes.byref(o), ctypes.byref(b))
    if st != RR_OK:
        raise RandRandError(st, "rr_rounds_workspace_bytes")
    return int(b.value)


class Server:
    """Serving loop (rr_server_*) over a device arena of ``budget_bytes``;
    with ``rounds`` (an rr_rounds_opts) the qualifying systems iterate in
    shared rounds, whose workspace is added to the arena."""

    def __init__(self, budget_bytes: int, workers: int = 8, rounds: rr_rounds_opts | None = None):
        import torch
        extra = rounds_workspace_bytes(rounds) if rounds is not None else 0
        total = int(budget_bytes) + extra
        self.arena = torch.empty(total, dtype=torch.uint8, device="cuda")
        self.s = ctypes.c_void_p(None)
        self.rounds = rounds
        if rounds is None:
            st = _lib().rr_server_create(ctypes.c_void_p(self.arena.data_ptr()), total,
                                         int(workers), ctypes.byref(self.s))
        else:
            st = _lib().rr_server_create_rounds(ctypes.c_void_p(self.arena.data_ptr()), total,
                                                int(workers), ctypes.byref(rounds), ctypes.byref(self.s))
        if st != RR_OK:
            raise RandRandError(st, "rr_server_create")
        self._keep = {}

    def rounds_stats(self) -> dict:
        r = rr_rounds_stats()
        _lib().rr_server_rounds_stats(self.s, ctypes.byref(r))
        return r.as_dict()

    def peak_running(self) -> int:
        p = ctypes.c_int32(0)
        _lib().rr_server_peak_running(self.s, ctypes.byref(p))
        return int(p.value)

    def submit(self, req: Request) -> int:
        t = ctypes.c_uint64(0)
        st = _lib().rr_server_submit(self.s, ctypes.byref(req.c), ctypes.byref(t))
        if st != RR_OK:
            raise RandRandError(st, "rr_server_submit")
        self._keep[int(t.value)] = req
        return int(t.value)

    def poll(self, ticket: int, wait: bool = False) -> dict:
        r = rr_result()
        st = _lib().rr_server_poll(self.s, int(ticket), 1 if wait else 0, ctypes.byref(r))
        if st != RR_OK:
            raise RandRandError(st, "rr_server_poll")
        if r.status != RR_PENDING:
            self._keep.pop(int(ticket), None)
        return r.as_dict()

    def drain(self):
        _lib().rr_server_drain(self.s)

    def stats(self) -> dict:
        q, r = ctypes.c_int32(0), ctypes.c_int32(0)
        used, peak = ctypes.c_size_t(0), ctypes.c_size_t(0)
        _lib().rr_server_stats(self.s, ctypes.byref(q), ctypes.byref(r), ctypes.byref(used),
                               ctypes.byref(peak))
        return {"queued": q.value, "running": r.value, "bytes_in_use": used.value,
                "peak_bytes": peak.value}

    def close(self):
        if self.s.value:
            _lib().rr_server_destroy(self.s)
            self.s = ctypes.c_void_p(None)
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_group(handles: list, bs: list, rtol, maxit=20000, stream=None):
    """randrand_solve_group: the built handles' systems solved together in
    shared rounds.  bs[i]: (n_i,) or (n_i, m_i) float64 CUDA tensor; rtol and
    maxit scalars or per-system lists.  Returns (status, [x_i], [[info dicts]])."""
    import torch
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.h if isinstance(h, Handle) else h for h in handles])
    rtols = rtol if isinstance(rtol, (list, tuple)) else [rtol] * n
    maxits = maxit if isinstance(maxit, (list, tuple)) else [maxit] * n
    keep, rhs = [], (rr_group_rhs * n)()
    for i, (h, b) in enumerate(zip(handles, bs)):
        nn = b.shape[0]
        B = b.reshape(nn, -1)
        Bc = B.t().contiguous()
        Xc = torch.zeros_like(Bc)
        keep.append((Bc, Xc, b.shape))
        rhs[i] = rr_group_rhs(b=Bc.data_ptr(), ldb=nn, x=Xc.data_ptr(), ldx=nn, nrhs=B.shape[1],
                              maxit=int(maxits[i]), rtol=float(rtols[i]))
    ws_bytes = ctypes.c_size_t(0)
    st = _lib().randrand_group_workspace_bytes(hs, n, ctypes.byref(ws_bytes))
    if st != RR_OK:
        raise RandRandError(st, "randrand_group_workspace_bytes")
    ws = torch.empty(max(int(ws_bytes.value), 256), dtype=torch.uint8, device="cuda")
    strm = stream if stream is not None else torch.cuda.current_stream()
    infos = (rr_solve_info * (8 * n))()
    st = _lib().randrand_solve_group(hs, n, rhs, ctypes.c_void_p(ws.data_ptr()), int(ws_bytes.value),
                                     ctypes.c_void_p(strm.cuda_stream), infos)
    xs = [Xc.t().reshape(shape) for _, Xc, shape in keep]
    out = [[infos[8 * i + c].as_dict() for c in range(rhs[i].nrhs)] for i in range(n)]
    return st, xs, out


def solve_batch(reqs: list, workers: int = 8, arena_bytes: int | None = None,
                rounds: rr_rounds_opts | None = None, stats: dict | None = None):
    """randrand_solve_batch (or, with ``rounds``, randrand_solve_batch_rounds)
    over the requests; returns (status, [result dicts]); ``stats`` (a dict)
    receives the rounds' time split."""
    import torch
    n = len(reqs)
    arr = (rr_request * n)(*[r.c for r in reqs])
    res = (rr_result * n)()
    if arena_bytes is None:
        arena_bytes = sum((r.workspace_bytes() + 255) // 256 * 256 for r in reqs)
    if rounds is not None:
        arena_bytes += rounds_workspace_bytes(rounds)
    arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda")
    if rounds is None:
        st = _lib().randrand_solve_batch(arr, n, ctypes.c_void_p(arena.data_ptr()), int(arena_bytes),
                                         int(workers), res)
    else:
        rs = rr_rounds_stats()
        st = _lib().randrand_solve_batch_rounds(arr, n, ctypes.c_void_p(arena.data_ptr()),
                                                int(arena_bytes), int(workers), ctypes.byref(rounds), res,
                                                ctypes.byref(rs))
        if stats is not None:
            stats.update(rs.as_dict())
    del arena
    return st, [res[i].as_dict() for i in range(n)]


def batch_rounds_opts(reqs: list) -> rr_rounds_opts:
    """Rounds capacity for a batch: every request resident at once."""
    mp = 2
    while mp < max(r.c.nrhs for r in reqs):
        mp *= 2
    rows = sum((r.op.n + 255) // 256 * 256 for r in reqs)
    return rounds_opts(mp, max(r.c.k for r in reqs), min(len(reqs), 152), rows)


load_library()
