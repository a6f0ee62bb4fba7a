#!/usr/bin/env python3
"""Benchmark: RandRAND-PCG solves/s on one GB300 (or N replicas).

Workload (one step = one solve = randrand_build + randrand_solve with every
right-hand side converged): Gaussian-kernel ridge system, n = 20000 points in
d = 8 from a 10-component Gaussian mixture (means ~ N(0, 4I), unit
covariances), K_ij = exp(-|x_i - x_j|^2 / 2), mu = 1e-3, sketch k = 500,
4 Gaussian right-hand sides, rtol 1e-6; bf16 sketch with float32
accumulation, float32 PCG iterations, float64-accurate restart residuals
(iterative refinement).  Inputs are synthetic and seeded (the paper's kernel
ridge datasets are not available offline; the mixture stands in for them).

Prints ONE JSON line (rank 0).  --impl reference times the float64 CPU oracle
instead, on a bounded sample of the same workload.

Other workloads (--workload; each prints its own JSON line):
  sparse_diffusion  512 x 512 variable-coefficient diffusion (CSR float32,
                    n = 262144), mu = 1e-6, k = 256, sparse-sign Omega,
                    Alg. 3 with the basis-less iteration, rtol 1e-6.
  batched           64 independent kernel ridge systems, n ~ U{2000..16000},
                    k = n/40, mu log-uniform in [1e-5, 1e-2], 8 right-hand
                    sides each, one randrand_solve_batch per step.
  serving           Poisson arrivals (200 req/s) of kernel (n log-uniform in
                    [1000, 32000], mu = 1e-3) and CSR diffusion (grid side in
                    128..512, mu = 1e-6) requests, k = n/50, 1 right-hand
                    side, rtol 1e-6, HBM budget 120 GB; p50/p99 latency.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(workload="gaussian_kernel_ridge", n=20000, d=8, components=10, mu=1e-3, k=500,
                nrhs=4, rtol=1e-6, bandwidth=1.0, sketch="gaussian", precision="mixed",
                variant="C", seed=0x52522)
METRIC = "RandRAND-PCG solves/s to rtol 1e-6 vs plain form on 1 GB300; p50/p99 latency"
# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it
# stands (summaries in profiles/: k_kernel_mv_tc_kernel_ridge_n20000.md,
# k_pcg_implicit_win_sparse_diffusion_512.md, the latter per iteration of a
# 256-iteration launch)
TRAFFIC = {"k_kernel_mv_tc": 5.544704e6, "k_pcg_implicit_win": (41.677312e6 + 1.663744e6) / 256}
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison")
    ap.add_argument("--workload", default="kernel_ridge",
                    choices=["kernel_ridge", "sparse_diffusion", "batched", "serving", "shift_path",
                             "indefinite"])
    ap.add_argument("--requests", type=int, default=2000, help="serving: number of requests")
    ap.add_argument("--workers", type=int, default=0, help="batched/serving: 0 = autotune")
    ap.add_argument("--no-rounds", action="store_true",
                    help="serving: every request on its worker's stream (no shared rounds)")
    ap.add_argument("--sketch", default=None,
                    choices=["gaussian", "srht", "multilevel", "sparse_sign"],
                    help="test matrix (default: Gaussian for the kernel ridge workload, "
                         "sparse sign for the sparse diffusion workload)")
    ap.add_argument("--variant", default="C", choices=["C", "R"],
                    help="kernel ridge and sparse diffusion: preconditioner variant")
    ap.add_argument("--joint", action="store_true",
                    help="shift_path: the joint basis of Sec. 5.1 (keep_sketch = 2)")
    ap.add_argument("--refine", action="store_true",
                    help="kernel ridge: refined projector (rr_build_opts.refine)")
    ap.add_argument("--kernel-impl", type=int, default=0,
                    help="kernel ridge: Gaussian-kernel product form (rr_build_opts.kernel_impl)")
    return ap.parse_args()


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(seed):
    from workloads import generators as W
    X = W.mixture_points(WORKLOAD["n"], WORKLOAD["d"], WORKLOAD["components"], seed=seed)
    B = W.gaussian_rhs(WORKLOAD["n"], WORKLOAD["nrhs"], seed)
    return X, B


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (read-only query)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_uuid=None):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.uuid = gpu_uuid

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- CPU oracle
def oracle_solve_timed(X, B, seed, sketch="gaussian", ml_l1=0, ml_gamma=0):
    """The float64 CPU oracle, as it stands, on the whole workload, end to end
    from the points: the dense K materialized once (the oracle's own
    materialize option), the build (the test matrix rounded to bf16 like the
    mixed path's, Householder QR, core matrix, 20 + 20 power iterations) and
    restarted PCG to rtol.  Returns (seconds, X, infos, operator)."""
    from oracle import randrand as O
    t0 = time.perf_counter()
    op = O.GaussKernelOp(X, WORKLOAD["bandwidth"], materialize=True)
    bd = O.build(op, WORKLOAD["mu"], WORKLOAD["k"], sketch, seed, omega_precision="bf16",
                 ml_l1=ml_l1, ml_gamma=ml_gamma)
    Xo, infos = O.solve(bd, np.asarray(B, dtype=np.float64), rtol=WORKLOAD["rtol"])
    return time.perf_counter() - t0, Xo, infos, op


def forward_error(Xg, op, mu, B):
    """|x - x*| / |x*| per column, x* = A_mu^-1 b by the oracle's dense
    Cholesky solve (float64)."""
    from oracle import randrand as O
    Xs = O.exact_solve(op, mu, np.asarray(B, dtype=np.float64))
    return [float(np.linalg.norm(Xg[:, j] - Xs[:, j]) / np.linalg.norm(Xs[:, j]))
            for j in range(Xs.shape[1])], Xs


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


# ------------------------------------------------------------- reference arm
REFERENCE_BUDGET_S = 150.0


def run_reference(args):
    """The oracle timed on the host cores: whole solves of the workload, as
    many of the requested steps as fit in REFERENCE_BUDGET_S (at least one),
    after at most one untimed warm-up solve.  The line reports the steps it
    actually ran and their measured time."""
    rank, world, _ = dist_init(args)
    if rank != 0:
        return
    X, B = make_inputs(WORKLOAD["seed"])
    warm = min(args.warmup, 1)
    for _ in range(warm):
        oracle_solve_timed(X, B, WORKLOAD["seed"])
    times, iters = [], 0
    t_start = time.perf_counter()
    while len(times) < args.steps:
        t, _, infos, _ = oracle_solve_timed(X, B, WORKLOAD["seed"])
        times.append(t)
        iters = max(i.inner_iters for i in infos)
        if time.perf_counter() - t_start + t > REFERENCE_BUDGET_S:
            break
    steps = len(times)
    value = steps / sum(times)
    sample = (f"{steps} whole float64 oracle solve(s) of the workload (n=20000, k=500, 4 right-hand "
              f"sides, rtol 1e-6; dense K materialized from the points, Householder QR, PCG with "
              f"restarts; {iters} iterations), {', '.join(f'{t:.1f}' for t in times)} s each; "
              f"{warm} untimed warm-up solve")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": steps, "steps_requested": args.steps, "warmup": warm,
        "ms_per_step": 1000.0 * sum(times) / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        # the same workload description as the GPU arm's line
        "config": {**{k: WORKLOAD[k] for k in ("workload", "n", "d", "k", "nrhs", "mu", "rtol",
                                               "precision", "variant", "sketch")},
                   "parallelism": f"replicas x{world}", "l2": "host cores (no GPU cache)"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_threads(),
                         "cpu": cpu_model(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    WORKLOAD["sketch"] = args.sketch or "gaussian"
    WORKLOAD["variant"] = args.variant

    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    import paper_2509_19747_gb300 as rr

    seed = WORKLOAD["seed"] + 1000 * rank     # independent systems per rank (replicas)
    X, B = make_inputs(seed)
    n, m, k = WORKLOAD["n"], WORKLOAD["nrhs"], WORKLOAD["k"]
    stream = torch.cuda.Stream()
    Xd = torch.from_numpy(X).cuda()
    Bc = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()        # column-major n x m
    Xc = torch.zeros_like(Bc)
    op = rr.Operator.gauss_kernel(Xd, WORKLOAD["bandwidth"])
    o = rr.rr_build_opts_default()
    o.variant = rr.VARIANTS[WORKLOAD["variant"]]
    o.precision = rr.PRECISIONS[WORKLOAD["precision"]]
    o.max_rhs = m
    o.profile = 0                 # the headline steps run without profiling events
    o.kernel_impl = args.kernel_impl
    o.refine = 1 if args.refine else 0
    rr.set_multilevel(o, WORKLOAD["sketch"], n, k)
    op_prof = rr.rr_build_opts()
    ctypes_copy(op_prof, o)
    op_prof.profile = 1
    ws_bytes = rr.randrand_workspace_bytes(op.c, k, op_prof)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    sk = rr.SKETCHES[WORKLOAD["sketch"]]

    def one_solve(opts, collect=None, rtol=None):
        h = rr.randrand_build(op.c, WORKLOAD["mu"], k, sk, seed, opts, ws.data_ptr(), ws_bytes,
                              stream.cuda_stream)
        Xc.zero_()
        s, infos = rr.randrand_solve(h, Bc.data_ptr(), m, n, Xc.data_ptr(), n, 0,
                                     WORKLOAD["rtol"] if rtol is None else rtol, 20000)
        if s != rr.RR_OK:
            raise RuntimeError(f"solve failed: {rr.randrand_status_str(s)} {infos}")
        if collect is not None:
            collect.append((rr.randrand_profile(h) if opts.profile else None, infos))
        rr.randrand_free(h)
        return infos

    def timed_pass(opts, collect):
        ms = []
        for _ in range(args.steps):
            flush.fill_(1)                           # L2 flush between timed steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_solve(opts, collect)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_solve(o)
        torch.cuda.synchronize()
        smi = ClockSampler(getattr(torch.cuda.get_device_properties(local), "uuid", None) and
                           "GPU-" + str(torch.cuda.get_device_properties(local).uuid))
        barrier(world)
        torch.cuda.synchronize()
        smi.start()
        wall0 = time.perf_counter()
        runs = []
        step_ms = timed_pass(o, runs)
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - wall0
        clocks = smi.stop()
        x_gpu = Xc.t().cpu().numpy().copy()        # the last timed solve's x (n x m)
        # per-kernel split and the roofline: a separate pass of the same steps
        # with CUDA events around every hot launch (randrand_profile)
        prof = []
        prof_ms = timed_pass(op_prof, prof)
        torch.cuda.synchronize()
    total_ms = max_over_ranks(sum(step_ms), world)
    ms_per_step = total_ms / args.steps
    value = world * 1000.0 / ms_per_step

    # per-kernel profile over the profiled pass
    cats = {}
    for p, _ in prof:
        for nm, (cnt, ms) in p.items():
            c = cats.setdefault(nm, [0, 0.0])
            c[0] += cnt
            c[1] += ms
    infos = [i for _, inf in runs for i in inf]
    iters = max(i["inner_iters"] for i in infos)
    rel_res = max(i["rel_residual"] for i in infos)
    gpu_launches = estimate_launches(prof, args.variant)

    # dominant kernel and its roofline
    dom = max(cats.items(), key=lambda kv: kv[1][1])
    roof = roofline(dom[0], dom[1], clocks)
    roof["measured"] = ("CUDA events around each launch in a profiled pass of the same "
                        f"{args.steps} steps ({sum(prof_ms) / args.steps:.2f} ms per step with "
                        "the events), after the headline steps")
    others = {kk: roofline(kk, v, clocks) for kk, v in cats.items() if kk != dom[0] and v[0] > 0}

    # end-to-end: host buffers through the C ABI, H2D inputs and D2H solution inside
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(rr, torch, op, o, ws, ws_bytes, stream, X, B, seed, args, world, flush)

    plain = None if args.no_plain else run_plain(rr, torch, op, m, k, seed, Bc)
    if plain is not None and not plain["converged"]:
        # the float32-only plain form stalls above rtol: compare both at a
        # tolerance it reaches, each a whole build + solve (ours event-timed,
        # median of 3 after one warm-up; the plain form as in run_plain)
        rt = 1e-5
        with torch.cuda.stream(stream):
            one_solve(o, rtol=rt)
            ours = []
            for _ in range(3):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                one_solve(o, rtol=rt)
                e1.record(stream)
                e1.synchronize()
                ours.append(e0.elapsed_time(e1))
        p_rt = run_plain(rr, torch, op, m, k, seed, Bc, rtol=rt)
        ours_ms = float(np.median(ours))
        plain["at_reachable_rtol"] = {
            "rtol": rt, "ours_ms": ours_ms, "plain_ms": 1e3 * p_rt["seconds"],
            "plain_converged": p_rt["converged"], "plain_inner_iters_max": p_rt["inner_iters_max"],
            "speedup": (1e3 * p_rt["seconds"] / ours_ms) if p_rt["converged"] else None}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {**{kk: WORKLOAD[kk] for kk in ("workload", "n", "d", "k", "nrhs", "mu", "rtol",
                                                  "precision", "variant", "sketch")},
                   **({"refine": "eq:accurate_proj"} if args.refine else {}),
                   "parallelism": f"replicas x{world}", "l2": "flushed between steps"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "solve": {"inner_iters_max": iters, "rel_residual_max": rel_res},
        "kernels_ms_per_step": {kk: v[1] / args.steps for kk, v in cats.items()},
        "roofline": roof, "roofline_other": others, "clocks": clocks,
        "gpu_launches": gpu_launches, "e2e": e2e, "plain_form": plain,
        "wall_s": wall,
    }
    if rank == 0 and not args.no_cpu_baseline:
        t, Xo, oinfos, oop = oracle_solve_timed(X, B, seed, WORKLOAD["sketch"], o.ml_l1, o.ml_gamma)
        fe, Xs = forward_error(x_gpu, oop, WORKLOAD["mu"], B)
        fe_o = [float(np.linalg.norm(Xo[:, j] - Xs[:, j]) / np.linalg.norm(Xs[:, j]))
                for j in range(Xs.shape[1])]
        line["solve"]["forward_error_vs_oracle"] = fe
        line["solve"]["forward_error_note"] = (
            "|x - x*| / |x*| per right-hand side of the last timed solve, x* = (K + mu I)^-1 b "
            "by the float64 oracle's dense Cholesky solve; the oracle's own rtol-1e-6 solve is at "
            + ", ".join(f"{e:.2e}" for e in fe_o))
        line["cpu_baseline"] = {
            "value": 1.0 / t, "unit": "solves/s", "cores": cpu_threads(), "cpu": cpu_model(),
            "kind": "oracle",
            "sample": (f"one whole float64 oracle solve of this workload, timed end to end from the "
                       f"points ({t:.1f} s: dense K materialized, build, PCG with restarts, "
                       f"{max(i.inner_iters for i in oinfos)} iterations)")}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_plain(rr, torch, op, m, k, seed, Bc, maxit=4000, rtol=None):
    """The plain form: float32 sketch on the float32 cores, float32 PCG and
    float32 residuals, direct launches on the legacy stream (no graphs), one
    system.  Reported with its own residual; it may stop short of rtol."""
    n = WORKLOAD["n"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = rr.Handle(op, WORKLOAD["mu"], k, WORKLOAD["sketch"], seed=seed, precision="fp32",
                  max_rhs=m, kernel_impl=1, stream=torch.cuda.default_stream())
    Xc = torch.zeros_like(Bc)
    s, infos = rr.randrand_solve(h.h, Bc.data_ptr(), m, n, Xc.data_ptr(), n, 0,
                                 WORKLOAD["rtol"] if rtol is None else rtol, maxit)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h.close()
    conv = s == rr.RR_OK
    return {"value": (1.0 / dt) if conv else None, "unit": "solves/s", "seconds": dt,
            "converged": conv, "status": rr.randrand_status_str(s),
            "inner_iters_max": max(i["inner_iters"] for i in infos),
            "rel_residual_max": max(i["rel_residual"] for i in infos),
            "config": "fp32 sketch on float32 cores, fp32 iterations and residuals, no graphs, "
                      f"maxit {maxit}"}


def estimate_launches(prof, variant="C"):
    # our kernels per solve, counted from the profile's launch counts: each
    # PCG product with the persistent step after it (2; variant R has a
    # persistent launch on each side of the product: 3), each power-iteration
    # product with its two projection launches (3), each restart residual with
    # its split sum and updates (4), and ~150 for the rest of the build
    # (sketch, Cholesky QR panels, core matrix); the one-step launch list of
    # this workload (profiles/launches_kernel_ridge_n20000_k500.md) counts 623
    total = 0
    for p, infos in prof:
        total += (p["matvec"][0] * (3 if variant == "R" else 2) + p["power"][0] * 3 + p["residual"][0] * 4 + 150 +
                  p["sketch"][0])
    return total


def roofline(name, stat, clocks):
    """Roofline of the dominant kernel from its event-timed launches."""
    cnt, ms = stat
    n, d, m = WORKLOAD["n"], WORKLOAD["d"], WORKLOAD["nrhs"]
    avg_s = ms / 1000.0 / max(cnt, 1)
    f = (clocks.get("sm_max_mhz") or 2070.0) * 1e6
    if name in ("matvec", "power"):
        # tensor-core float32 kernel product: the exponent arguments come from
        # the tensor cores, so each of the n^2 entries needs exactly one ex2 on
        # the special-function units (MUFU): peak 152 SMs x 32 ex2/clk x clock
        # (a throughput probe measured 31.6 ex2 per SM per clock on this part)
        ops = float(n) * n
        peak = 152 * 32 * f
        return {"kernel": "k_kernel_mv_tc", "bound": "alu", "achieved": ops / avg_s / 1e9,
                "peak": peak / 1e9, "unit": "G ex2/s (MUFU)", "frac": ops / avg_s / peak,
                "traffic": TRAFFIC["k_kernel_mv_tc"], "launches": cnt, "avg_us": avg_s * 1e6,
                "peak_note": "derived: 152 SMs x 32 ex2 per clock x sampled max SM clock"}
    if name == "residual":
        # double-float restart residual over the symmetric K: n (n + 1) / 2
        # distinct entries, each ~142 float32-pipe ops to evaluate in
        # double-float and 2 x 12 per right-hand side for its row and column
        # products
        ops = float(n) * (n + 1) / 2 * (142 + 24 * m)
        peak = 152 * 128 * f
        return {"kernel": "k_kernel_mv_df2s", "bound": "alu", "achieved": ops / avg_s / 1e9,
                "peak": peak / 1e9, "unit": "G f32-op/s", "frac": ops / avg_s / peak,
                "traffic": None, "launches": cnt, "avg_us": avg_s * 1e6}
    # sketch: 2 n^2 k flops on the tensor cores (bf16, dense)
    flops = 2.0 * n * n * WORKLOAD["k"]
    peak_tf = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0
    return {"kernel": "k_kernel_sketch_sk", "bound": "tensor", "achieved": flops / avg_s / 1e12,
            "peak": peak_tf, "unit": "TFLOP/s", "frac": flops / avg_s / 1e12 / peak_tf,
            "traffic": None, "launches": cnt, "avg_us": avg_s * 1e6}


def run_e2e(rr, torch, op, o, ws, ws_bytes, stream, X, B, seed, args, world, flush):
    n, m, k = WORKLOAD["n"], WORKLOAD["nrhs"], WORKLOAD["k"]
    Xh = torch.from_numpy(X).pin_memory()
    Bh = torch.from_numpy(np.ascontiguousarray(B.T)).pin_memory()
    Xout = torch.zeros_like(Bh).pin_memory()
    Xd = op._keep[0]
    o2 = rr.rr_build_opts()
    ctypes_copy(o2, o)
    o2.profile = 0
    sk = rr.SKETCHES[WORKLOAD["sketch"]]

    def step():
        with torch.cuda.stream(stream):
            Xd.copy_(Xh, non_blocking=True)
            h = rr.randrand_build(op.c, WORKLOAD["mu"], k, sk, seed, o2, ws.data_ptr(), ws_bytes,
                                  stream.cuda_stream)
            s, _ = rr.randrand_solve_host(h, Bh.data_ptr(), m, n, Xout.data_ptr(), n,
                                          WORKLOAD["rtol"], 20000)
            rr.randrand_free(h)
            if s != rr.RR_OK:
                raise RuntimeError("e2e solve failed")

    step()
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    tot = max_over_ranks(sum(ts), world)
    return {"value": world * args.steps / tot, "unit": "solves/s",
            "h2d_bytes_per_step": int(X.nbytes + B.nbytes), "d2h_bytes_per_step": int(B.nbytes)}


def ctypes_copy(dst, src):
    for f, _ in src._fields_:
        setattr(dst, f, getattr(src, f))


# ------------------------------------------------------------ other workloads
SPARSE = dict(workload="sparse_diffusion", side=512, n=262144, mu=1e-6, k=256, l_sk=1024,
              gamma=8, gamma_sk=8, nrhs=1, rtol=1e-6, precision="mixed",
              orth="rand_cholqr (basis-less)", seed=0x52523)
BATCHED = dict(workload="batched_kernel_ridge", systems=64, n_min=2000, n_max=16000,
               k="n/40", mu="10^U(-5,-2)", nrhs=8, rtol=1e-6, precision="mixed", seed=0x52524)
INDEF = dict(workload="kernel_shift_invert", n=20000, d=8, k=500, nrhs=4, mu=-20.0, rtol=1e-6,
             precision="mixed", variant="G", q=1, solver="MINRES")
SHIFTS = dict(workload="kernel_ridge_shift_path", n=20000, d=8, k=500, nrhs=4, rtol=1e-6,
              precision="mixed", mus=[1e-1, 3e-2, 1e-2, 3e-3, 1e-3, 3e-4, 1e-4, 3e-5])
SERVING = dict(workload="serving_mix", rate_per_s=200.0, kernel_share=0.5, kernel_n=[1000, 32000],
               csr_side=[128, 512], k="n/50", nrhs=1, rtol=1e-6, budget_gb=120.0,
               precision="mixed", seed=0x52525)


def _line(args, world, metric, value, unit, ms_per_step, config, **extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config}
    line.update(extra)
    return line


def run_other(args):
    if args.impl == "reference":
        rank, world, _ = dist_init(args)
        if rank == 0:
            print(json.dumps({"impl": "reference", "workload": args.workload,
                              "unavailable": "the oracle arm times the kernel ridge workload only"}))
        return
    {"sparse_diffusion": run_sparse, "batched": run_batched, "serving": run_serving,
     "shift_path": run_shift_path, "indefinite": run_indefinite}[args.workload](args)


def sparse_iteration_bytes(nnz, n, gamma, mp=1):
    """Algorithmic bytes of one basis-less CSR iteration: three products with
    A_mu (float32 values and int32 column indices, int32 row pointers, one
    float32 vector read and one written per column), Omega^T and Omega as
    sparse-sign patterns (gamma entries of a 4-byte index and a 1-byte sign
    per row, each read once), and ~10 float32 vector streams per column."""
    return (3 * (8.0 * nnz + 4.0 * (n + 1) + 2 * 4.0 * n * mp) + 2 * 5.0 * gamma * n
            + 10 * 4.0 * n * mp)


def run_sparse(args):
    import torch
    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    import paper_2509_19747_gb300 as rr
    from workloads import generators as W
    cfg = SPARSE
    seed = cfg["seed"] + 1000 * rank
    C = W.diffusion_csr(side=cfg["side"], seed=cfg["seed"])
    b = W.gaussian_rhs(C.n, 1, seed)
    stream = torch.cuda.Stream()
    rp, ci, va = (torch.from_numpy(a).cuda() for a in (C.rowptr, C.colidx, C.vals))
    op = rr.Operator.csr(rp, ci, va)
    o = rr.rr_build_opts_default()
    o.precision = rr.RR_PREC_MIXED
    o.orth = rr.RR_ORTH_RAND_CHOLQR
    o.l_sk = cfg["l_sk"]
    o.gamma = cfg["gamma"]
    o.gamma_sk = cfg["gamma_sk"]
    o.profile = 0                 # the timed steps run without profiling events
    sketch = args.sketch or "sparse_sign"
    o.variant = rr.VARIANTS[args.variant]
    rr.set_multilevel(o, sketch, C.n, cfg["k"])
    o_prof = rr.rr_build_opts()
    ctypes_copy(o_prof, o)
    o_prof.profile = 1
    ws_bytes = rr.randrand_workspace_bytes(op.c, cfg["k"], o_prof)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    bd = torch.from_numpy(np.ascontiguousarray(b[:, 0])).cuda()
    xd = torch.zeros_like(bd)

    def one(opts, collect=None):
        h = rr.randrand_build(op.c, cfg["mu"], cfg["k"], rr.SKETCHES[sketch], seed, opts,
                              ws.data_ptr(), ws_bytes, stream.cuda_stream)
        st, infos = rr.randrand_solve(h, bd.data_ptr(), 1, C.n, xd.data_ptr(), C.n, 0, cfg["rtol"],
                                      100000)
        if st != rr.RR_OK:
            raise RuntimeError(f"sparse solve failed: {rr.randrand_status_str(st)} {infos}")
        if collect is not None:
            collect.append((rr.randrand_profile(h) if opts.profile else None, infos))
        rr.randrand_free(h)

    def timed_pass(opts, collect):
        out = []
        for _ in range(args.steps):
            flush.fill_(1)                           # L2 flush between timed steps (not timed)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one(opts, collect)
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return out

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one(o)
        torch.cuda.synchronize()
        smi = ClockSampler()
        barrier(world)
        smi.start()
        runs = []
        step_ms = timed_pass(o, runs)
        barrier(world)
        clocks = smi.stop()
        # per-kernel split and the roofline: a separate pass of the same steps
        # with CUDA events around the hot launches (randrand_profile)
        prof = []
        timed_pass(o_prof, prof)
        torch.cuda.synchronize()
    ms = max_over_ranks(sum(step_ms), world) / args.steps
    infos = [i for _, inf in runs for i in inf]

    e2e = None
    if not args.no_e2e:
        # end to end through the C ABI: every step copies the CSR arrays from
        # pinned host memory into the operator's device arrays, builds, and
        # solves with host b and x (randrand_solve_host)
        hrp, hci, hva = (torch.from_numpy(a).pin_memory() for a in (C.rowptr, C.colidx, C.vals))
        bh = torch.from_numpy(np.ascontiguousarray(b[:, 0])).pin_memory()
        xh = torch.zeros_like(bh).pin_memory()

        def e2e_step():
            with torch.cuda.stream(stream):
                rp.copy_(hrp, non_blocking=True)
                ci.copy_(hci, non_blocking=True)
                va.copy_(hva, non_blocking=True)
                h = rr.randrand_build(op.c, cfg["mu"], cfg["k"], rr.SKETCHES[sketch], seed, o,
                                      ws.data_ptr(), ws_bytes, stream.cuda_stream)
                st, _ = rr.randrand_solve_host(h, bh.data_ptr(), 1, C.n, xh.data_ptr(), C.n,
                                               cfg["rtol"], 100000)
                rr.randrand_free(h)
                if st != rr.RR_OK:
                    raise RuntimeError(f"sparse e2e solve failed: {rr.randrand_status_str(st)}")

        e2e_step()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        e2e = {"value": world * args.steps / max_over_ranks(sum(ts), world), "unit": "solves/s",
               "h2d_bytes_per_step": int(C.rowptr.nbytes + C.colidx.nbytes + C.vals.nbytes +
                                         bh.numel() * bh.element_size()),
               "d2h_bytes_per_step": int(xh.numel() * xh.element_size())}
    mv = [p["matvec"] for p, _ in prof]
    cnt, tot = sum(c for c, _ in mv), sum(t for _, t in mv)
    # iterations of the profiled pass, whose event times the roofline divides
    iters_total = sum(i["inner_iters"] for _, inf in prof for i in inf)
    mp = 1    # one right-hand side (stored padded to two columns; the step computes one)
    peaks = _peaks()
    if cnt < iters_total / 2:
        # persistent launches: the event pair spans whole runs of iterations.
        # The window form keeps the matrix and the patterns in shared memory
        # across iterations, so these bytes are what an unfused iteration
        # would move, not its traffic.
        per_s = tot / 1000.0 / max(iters_total, 1)
        bytes_ = sparse_iteration_bytes(len(C.vals), C.n, cfg["gamma"], mp)
        kern, unit_note = "k_pcg_implicit_win (per iteration)", "iterations"
        traffic = TRAFFIC["k_pcg_implicit_win"]
    else:
        per_s = tot / 1000.0 / max(cnt, 1)
        bytes_ = 8.0 * len(C.vals) + 4.0 * (C.n + 1) + 2 * 4.0 * C.n * mp
        kern, unit_note = "k_csr_mv_add", "launches"
        traffic = None
    roof = {"kernel": kern, "bound": "hbm", "achieved": bytes_ / per_s / 1e9,
            "peak": peaks["hbm"], "unit": "GB/s", "frac": bytes_ / per_s / 1e9 / peaks["hbm"],
            "traffic": traffic, "launches": cnt, "avg_us": per_s * 1e6, "per": unit_note,
            "algorithmic_bytes": bytes_,
            "note": "the working set of one iteration stays in L2 between iterations"}
    line = _line(args, world, "RandRAND-PCG solves/s to rtol 1e-6 (sparse diffusion 512^2)",
                 world * 1000.0 / ms, "solves/s", ms,
                 {**{kk: cfg[kk] for kk in ("workload", "side", "n", "k", "l_sk", "mu", "rtol",
                                            "precision", "orth")},
                  "variant": args.variant,
                  "sketch": sketch if sketch != "multilevel"
                  else f"multilevel (l1 = {o.ml_l1}, gamma1 = {o.ml_gamma})",
                  "parallelism": f"replicas x{world}", "l2": "flushed between steps"},
                 latency_ms={"p50": float(np.percentile(step_ms, 50)),
                             "p99": float(np.percentile(step_ms, 99))},
                 solve={"inner_iters_max": max(i["inner_iters"] for i in infos),
                        "rel_residual_max": max(i["rel_residual"] for i in infos),
                        "ms_per_iteration": ms / max(i["inner_iters"] for i in infos)},
                 kernels_ms_per_step={kk: sum(p[kk][1] for p, _ in prof) / args.steps
                                      for kk in prof[0][0]},
                 roofline=roof, clocks=clocks, e2e=e2e)
    if rank == 0 and not args.no_cpu_baseline:
        # bounded sample: the oracle's build of this system (sparse-sign Omega,
        # basis by Householder QR: its Alg. 3 forms Theta as a dense l_sk x n
        # matrix, 2 GB here) and 50 of its PCG iterations, each timed; the
        # iteration time is scaled to the GPU solve's iteration count
        from oracle import randrand as O
        cop = O.CsrOp(C.rowptr, C.colidx, C.vals, C.n)
        t0 = time.perf_counter()
        bd = O.build(cop, cfg["mu"], cfg["k"], "sparse_sign", seed, gamma=cfg["gamma"])
        t_build = time.perf_counter() - t0
        fixed = 50
        t1 = time.perf_counter()
        O.solve(bd, np.asarray(b, dtype=np.float64), rtol=cfg["rtol"], fixed_inner=fixed)
        t_it = (time.perf_counter() - t1) / fixed
        iters = max(i["inner_iters"] for i in infos)
        line["cpu_baseline"] = {
            "value": 1.0 / (t_build + iters * t_it), "unit": "solves/s", "cores": cpu_threads(),
            "cpu": cpu_model(), "kind": "oracle",
            "sample": (f"the float64 oracle's build of this system ({t_build:.1f} s; Householder "
                       f"basis) and {fixed} of its PCG iterations ({t_it * 1e3:.1f} ms each), "
                       f"scaled to the GPU solve's {iters} iterations")}
    if rank == 0:
        print(json.dumps(line), flush=True)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm": d.get("hbm_gbs", 6800.0), "bf16": d.get("bf16_tflops", 1900.0)}
    return {"hbm": 6800.0, "bf16": 1900.0}


def batched_systems(rr, torch, rank, iter_impl=0):
    from workloads import generators as W
    cfg = BATCHED
    rng = np.random.default_rng([cfg["seed"], 7, rank])
    reqs, meta = [], []
    for i in range(cfg["systems"]):
        n = int(rng.integers(cfg["n_min"], cfg["n_max"] + 1))
        mu = float(10.0 ** rng.uniform(-5, -2))
        sd = cfg["seed"] * 1000 + 64 * rank + i
        X = torch.from_numpy(W.mixture_points(n, seed=sd)).cuda()
        B = torch.from_numpy(W.gaussian_rhs(n, cfg["nrhs"], sd)).cuda()
        op = rr.Operator.gauss_kernel(X)
        reqs.append(rr.Request(op, mu, n // 40, B, cfg["rtol"], seed=sd, precision="mixed",
                               iter_impl=iter_impl))
        meta.append((n, mu))
    return reqs, meta


def run_batched(args):
    import torch
    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    import paper_2509_19747_gb300 as rr
    sets = {impl: batched_systems(rr, torch, rank, iter_impl=impl)[0] for impl in (0, 1)}
    arena = sum((q.workspace_bytes() + 255) // 256 * 256 for q in sets[0])
    ropts = rr.batch_rounds_opts(sets[0])
    # schedule: shared rounds (every system's iterations in one grouped launch
    # per round; the library tunes the rounds per graph replay) or one stream
    # per worker with the persistent step or separate kernels, and the worker
    # count: the best of a few on untimed passes, or as given
    cands = [(w, impl) for w in ([args.workers] if args.workers > 0 else [4, 8, 16])
             for impl in ("rounds", 0, 1)]
    tune, rstats = {}, {}
    for w, impl in cands:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if impl == "rounds":
            rs = {}
            st, _ = rr.solve_batch(sets[0], workers=w, arena_bytes=arena, rounds=ropts, stats=rs)
            rstats[w] = rs
        else:
            st, _ = rr.solve_batch(sets[impl], workers=w, arena_bytes=arena)
        torch.cuda.synchronize()
        tune[(w, impl)] = time.perf_counter() - t0
        if st != rr.RR_OK:
            raise RuntimeError(f"batch failed ({impl}): {rr.randrand_status_str(st)}")
    workers, impl = min(tune, key=tune.get)
    reqs = sets[0] if impl == "rounds" else sets[impl]
    kw = dict(rounds=ropts) if impl == "rounds" else {}
    for _ in range(max(args.warmup - 1, 0)):
        rr.solve_batch(reqs, workers=workers, arena_bytes=arena, **kw)
    smi = ClockSampler()
    torch.cuda.synchronize()
    barrier(world)
    smi.start()
    step_ms, lat = [], []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        t0 = time.perf_counter()
        st, res = rr.solve_batch(reqs, workers=workers, arena_bytes=arena, **kw)
        torch.cuda.synchronize()
        e1.record()
        e1.synchronize()
        step_ms.append(max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3))
        if st != rr.RR_OK:
            raise RuntimeError(f"batch failed: {rr.randrand_status_str(st)}")
        lat += [r["end_ms"] - r["submit_ms"] for r in res]
    barrier(world)
    clocks = smi.stop()
    ms = max_over_ranks(sum(step_ms), world) / args.steps
    # one system after another on one stream: the same systems, one worker
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rr.solve_batch(reqs, workers=1, arena_bytes=arena)
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    iters = [i["inner_iters"] for r in res for i in r["info"]]
    line = _line(args, world, "RandRAND-PCG solves/s to rtol 1e-6 (64 batched kernel ridge systems)",
                 world * BATCHED["systems"] * 1000.0 / ms, "solves/s", ms,
                 {**BATCHED, "workers": workers, "schedule": "shared rounds" if impl == "rounds"
                  else f"one stream per worker, iter_impl {impl}", "parallelism": f"replicas x{world}",
                  "l2": "inputs of the batch exceed L2"},
                 latency_ms={"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                 one_after_another={"value": BATCHED["systems"] / seq_s, "unit": "solves/s",
                                    "seconds": seq_s},
                 autotune_s={f"workers={k[0]},schedule={k[1]}": v for k, v in tune.items()},
                 in_rounds=sum(r.get("rounds", 0) for r in res),
                 rounds_split_s={f"workers={w}": v for w, v in rstats.items()},
                 solve={"inner_iters_max": max(iters), "inner_iters_median": float(np.median(iters))},
                 roofline=None, clocks=clocks)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_indefinite(args):
    """Shift-and-invert on the Gaussian kernel system of the main workload: A_mu
    = K - 20 I is indefinite (about a hundred eigenvalues of K lie above 20), solved with
    G-RandRAND MINRES (Sec. 3.3, 6.3; q = 1).  One step = build + solve."""
    import torch
    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    import paper_2509_19747_gb300 as rr
    cfg = INDEF
    seed = WORKLOAD["seed"] + 1000 * rank
    X, B = make_inputs(seed)
    Xd = torch.from_numpy(X).cuda()
    Bd = torch.from_numpy(B).cuda()
    op = rr.Operator.gauss_kernel(Xd, WORKLOAD["bandwidth"])

    def step():
        h = rr.Handle(op, cfg["mu"], cfg["k"], "gaussian", seed=seed, variant=cfg["variant"],
                      q=cfg["q"], precision=cfg["precision"], max_rhs=cfg["nrhs"])
        _, st, infos = h.solve(Bd, rtol=cfg["rtol"])
        h.close()
        if st != rr.RR_OK:
            raise RuntimeError(f"indefinite solve: {rr.randrand_status_str(st)}")
        return infos

    for _ in range(args.warmup):
        step()
    smi = ClockSampler()
    barrier(world)
    smi.start()
    ms = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = step()
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t0) * 1e3)
    barrier(world)
    clocks = smi.stop()
    mean = max_over_ranks(sum(ms), world) / args.steps
    line = _line(args, world, "G-RandRAND MINRES solves/s to rtol 1e-6 (kernel shift-and-invert, mu = -20)",
                 world * 1000.0 / mean, "solves/s", mean,
                 {**cfg, "parallelism": f"replicas x{world}", "l2": "inputs of a solve exceed L2"},
                 solve={"inner_iters_max": max(i["inner_iters"] for i in infos),
                        "outer_iters_max": max(i["outer_iters"] for i in infos),
                        "rel_residual_max": max(i["rel_residual"] for i in infos),
                        "tau": infos[0]["tau"], "norm_I_minus_Pi_A": infos[0]["normE"],
                        "norm_Pit_A": infos[0]["lam_max"]},
                 timing="host wall clock around build + solve with the device synchronised",
                 roofline=None, clocks=clocks)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_shift_path(args):
    """A regularization path (Sec. 5.1): the kernel ridge system of the main
    workload solved for 8 shifts.  One step = the whole path with the sketch
    kept (one build with keep_sketch, then randrand_set_mu + solve per shift);
    the same path with a fresh build per shift is timed beside it."""
    import torch
    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    import paper_2509_19747_gb300 as rr
    cfg = SHIFTS
    seed = WORKLOAD["seed"] + 1000 * rank
    X, B = make_inputs(seed)
    Xd = torch.from_numpy(X).cuda()
    Bd = torch.from_numpy(B).cuda()
    op = rr.Operator.gauss_kernel(Xd, WORKLOAD["bandwidth"])
    mus = cfg["mus"]

    def kept():
        h = rr.Handle(op, mus[0], cfg["k"], "gaussian", seed=seed, precision=cfg["precision"],
                      max_rhs=cfg["nrhs"], keep_sketch=2 if args.joint else 1)
        its = []
        for i, mu in enumerate(mus):
            if i > 0:
                h.set_mu(mu)
            _, st, infos = h.solve(Bd, rtol=cfg["rtol"])
            if st != rr.RR_OK:
                raise RuntimeError(f"shift {mu}: {rr.randrand_status_str(st)}")
            its.append(max(j["inner_iters"] for j in infos))
        h.close()
        return its

    def fresh():
        its = []
        for mu in mus:
            h = rr.Handle(op, mu, cfg["k"], "gaussian", seed=seed, precision=cfg["precision"],
                          max_rhs=cfg["nrhs"])
            _, st, infos = h.solve(Bd, rtol=cfg["rtol"])
            if st != rr.RR_OK:
                raise RuntimeError(f"shift {mu}: {rr.randrand_status_str(st)}")
            its.append(max(j["inner_iters"] for j in infos))
            h.close()
        return its

    def timed(fn, steps):
        ms = []
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its = fn()
            torch.cuda.synchronize()
            ms.append((time.perf_counter() - t0) * 1e3)
        return ms, its

    for _ in range(args.warmup):
        kept()
    fresh()
    smi = ClockSampler()
    barrier(world)
    smi.start()
    ms_kept, its = timed(kept, args.steps)
    barrier(world)
    clocks = smi.stop()
    ms_fresh, its_fresh = timed(fresh, max(1, args.steps // 2))
    ms = max_over_ranks(sum(ms_kept), world) / args.steps
    line = _line(args, world, "RandRAND-PCG shifts solved/s along a regularization path (sketch kept)",
                 world * len(mus) * 1000.0 / ms, "solves/s", ms,
                 {**cfg, "recycling": "joint basis" if args.joint else "Gram separation",
                  "parallelism": f"replicas x{world}", "l2": "inputs of a path exceed L2"},
                 fresh_builds={"value": len(mus) * 1000.0 / (sum(ms_fresh) / len(ms_fresh)),
                               "unit": "solves/s", "ms_per_path": sum(ms_fresh) / len(ms_fresh)},
                 solve={"inner_iters_max_per_shift": its, "fresh_inner_iters_max_per_shift": its_fresh},
                 timing="host wall clock around each path with the device synchronised",
                 roofline=None, clocks=clocks)
    if rank == 0:
        print(json.dumps(line), flush=True)


def serving_requests(rr, torch, count, rank):
    from workloads import generators as W
    cfg = SERVING
    rng = np.random.default_rng([cfg["seed"], 11, rank])
    arrivals = np.cumsum(rng.exponential(1.0 / cfg["rate_per_s"], size=count))
    csr_ops = {}
    reqs = []
    for i in range(count):
        sd = cfg["seed"] * 10000 + i
        if rng.random() < cfg["kernel_share"]:
            n = int(round(np.exp(rng.uniform(np.log(cfg["kernel_n"][0]), np.log(cfg["kernel_n"][1])))))
            X = torch.from_numpy(W.mixture_points(n, seed=sd)).cuda()
            b = torch.from_numpy(W.gaussian_rhs(n, 1, sd)[:, 0].copy()).cuda()
            reqs.append(("kernel", n, rr.Request(rr.Operator.gauss_kernel(X), 1e-3, n // 50, b,
                                                 cfg["rtol"], seed=sd, precision="mixed")))
        else:
            # grid sides on a 64-cell lattice in [128, 512]; one operator per side
            side = int(rng.integers(2, 9)) * 64
            if side not in csr_ops:
                C = W.diffusion_csr(side=side, seed=cfg["seed"] + side)
                csr_ops[side] = (C.n, rr.Operator.csr(*(torch.from_numpy(a).cuda()
                                                        for a in (C.rowptr, C.colidx, C.vals))))
            n, op = csr_ops[side]
            b = torch.from_numpy(W.gaussian_rhs(n, 1, sd)[:, 0].copy()).cuda()
            reqs.append(("csr", n, rr.Request(op, 1e-6, n // 50, b, cfg["rtol"], sketch="sparse_sign",
                                              seed=sd, precision="mixed", orth="rand_cholqr",
                                              maxit=100000)))
    return arrivals, reqs


def run_serving(args):
    import torch
    rank, world, local = dist_init(args)
    torch.cuda.set_device(local)
    import paper_2509_19747_gb300 as rr
    arrivals, reqs = serving_requests(rr, torch, args.requests, rank)
    budget = int(SERVING["budget_gb"] * 1e9)
    workers = args.workers if args.workers > 0 else 16
    # the kernel requests (one right-hand side, k = n / 50 <= 640) iterate in
    # shared rounds; the CSR requests iterate in their own persistent launches
    ropts = rr.rounds_opts(2, 640, 152, 2 << 20) if not args.no_rounds else None
    srv = rr.Server(budget, workers=workers, rounds=ropts)
    # warm-up: a few requests of each kind, untimed
    warm = [q for _, _, q in reqs[: max(args.warmup, 1) * 2]]
    for q in warm:
        srv.submit(q)
    srv.drain()
    smi = ClockSampler()
    barrier(world)
    smi.start()
    t0 = time.perf_counter()
    tickets = []
    for (kind, n, q), ta in zip(reqs, arrivals):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append((kind, n, srv.submit(q)))
    srv.drain()
    makespan = time.perf_counter() - t0
    clocks = smi.stop()
    res = [(kind, n, srv.poll(t)) for kind, n, t in tickets]
    stats = srv.stats()
    srv.close()
    ok = [r for _, _, r in res if r["status"] == rr.RR_OK]
    lat = [r["end_ms"] - r["submit_ms"] for _, _, r in res]
    by_kind = {}
    for kind, n, r in res:
        by_kind.setdefault(kind, []).append(r["end_ms"] - r["submit_ms"])
    value = world * len(ok) / max_over_ranks(makespan, world)
    line = _line(args, world, "RandRAND-PCG solves/s to rtol 1e-6 (serving mix)", value, "solves/s",
                 1000.0 * makespan / len(res),
                 {**SERVING, "requests": len(res), "workers": workers,
                  "schedule": "kernel requests in shared rounds" if ropts is not None
                  else "one stream per worker", "parallelism": f"replicas x{world}"},
                 latency_ms={"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                             **{f"p50_{k}": float(np.percentile(v, 50)) for k, v in by_kind.items()}},
                 completed=len(ok), failed=len(res) - len(ok), makespan_s=makespan,
                 offered_s=float(arrivals[-1]),
                 overloaded=bool(makespan > 1.5 * float(arrivals[-1])),
                 # when the arrivals outrun the server it runs saturated, so the
                 # completion rate is the mix's sustainable request rate
                 capacity_req_per_s=(len(ok) / makespan
                                     if makespan > 1.5 * float(arrivals[-1]) else None),
                 peak_arena_gb=stats["peak_bytes"] / 1e9,
                 in_rounds=sum(r.get("rounds", 0) for _, _, r in res), roofline=None, clocks=clocks)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload != "kernel_ridge":
        run_other(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
