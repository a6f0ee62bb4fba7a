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
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
def oracle_sample(X, B, products_per_solve, reps=1):
    """Float64 CPU oracle, as it stands, on a bounded sample of the workload:
    `reps` full-size products (K + mu I) V with the 4 right-hand sides and one
    Householder QR of an n x k basis; scaled to one solve by the number of
    such products the solve performs.  Returns (solves/s, seconds of sample)."""
    from oracle import randrand as O
    op = O.GaussKernelOp(X, WORKLOAD["bandwidth"])
    V = np.asarray(B, dtype=np.float64)
    t0 = time.perf_counter()
    for _ in range(reps):
        O.shifted(op, WORKLOAD["mu"])(V)
    t_mv = (time.perf_counter() - t0) / reps
    Y = np.random.default_rng(0).standard_normal((WORKLOAD["n"], WORKLOAD["k"]))
    t1 = time.perf_counter()
    O.householder_qr(Y)
    t_qr = time.perf_counter() - t1
    per_solve = products_per_solve * t_mv + 2 * t_qr
    return 1.0 / per_solve, time.perf_counter() - t0, t_mv, t_qr


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count() or 1


def products_per_solve(iters, k, nrhs, power_iters=20, restarts=3):
    # sketch: k columns = k / nrhs products of nrhs columns; power: 2 x 20 single
    # columns (= 40 / nrhs products); iterations: one product each; restarts.
    return k / nrhs + 2 * power_iters / nrhs + iters + restarts


# ------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_init(args)
    if rank != 0:
        return
    X, B = make_inputs(WORKLOAD["seed"])
    # iteration count of the oracle's own solve of this workload (committed
    # fixture written by tests/golden/make_golden.py from the oracle)
    gpath = os.path.join(ROOT, "tests", "golden", "kernel_ridge_oracle_iters.json")
    iters = json.load(open(gpath))["inner_iters_max"] if os.path.exists(gpath) else 250
    pps = products_per_solve(iters, WORKLOAD["k"], WORKLOAD["nrhs"])
    for _ in range(args.warmup):
        oracle_sample(X, B, pps)
    vals, secs = [], 0.0
    for _ in range(args.steps):
        v, s, _, _ = oracle_sample(X, B, pps)
        vals.append(v)
        secs += s
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {k: WORKLOAD[k] for k in ("workload", "n", "d", "k", "nrhs", "mu", "rtol")},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_threads(),
                         "kind": "oracle",
                         "sample": f"per step: one float64 (K+mu I)V product with 4 columns at "
                                   f"n=20000 and one 20000x500 Householder QR, scaled by "
                                   f"{pps:.0f} products per solve (oracle iteration count {iters})"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch

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
    o.profile = 1
    ws_bytes = rr.randrand_workspace_bytes(op.c, k, o)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    sk = rr.SKETCHES[WORKLOAD["sketch"]]

    def one_solve(collect=None):
        h = rr.randrand_build(op.c, WORKLOAD["mu"], k, sk, seed, o, ws.data_ptr(), ws_bytes,
                              stream.cuda_stream)
        Xc.zero_()
        s, infos = rr.randrand_solve(h, Bc.data_ptr(), m, n, Xc.data_ptr(), n, 0,
                                     WORKLOAD["rtol"], 20000)
        if s != rr.RR_OK:
            raise RuntimeError(f"solve failed: {rr.randrand_status_str(s)} {infos}")
        if collect is not None:
            collect.append((rr.randrand_profile(h), infos))
        rr.randrand_free(h)
        return infos

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_solve()
        torch.cuda.synchronize()
        smi = ClockSampler(getattr(torch.cuda.get_device_properties(local), "uuid", None) and
                           "GPU-" + str(torch.cuda.get_device_properties(local).uuid))
        barrier(world)
        torch.cuda.synchronize()
        smi.start()
        wall0 = time.perf_counter()
        step_ms, prof = [], []
        for _ in range(args.steps):
            flush.fill_(1)                           # L2 flush between timed steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_solve(prof)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - wall0
        clocks = smi.stop()
    total_ms = max_over_ranks(sum(step_ms), world)
    ms_per_step = total_ms / args.steps
    value = world * 1000.0 / ms_per_step

    # per-kernel profile over the timed region
    cats = {}
    for p, _ in prof:
        for nm, (cnt, ms) in p.items():
            c = cats.setdefault(nm, [0, 0.0])
            c[0] += cnt
            c[1] += ms
    infos = [i for _, inf in prof for i in inf]
    iters = max(i["inner_iters"] for i in infos)
    rel_res = max(i["rel_residual"] for i in infos)
    gpu_launches = estimate_launches(prof)

    # dominant kernel and its roofline
    dom = max(cats.items(), key=lambda kv: kv[1][1])
    roof = roofline(dom[0], dom[1], clocks)
    others = {kk: roofline(kk, v, clocks) for kk, v in cats.items() if kk != dom[0] and v[0] > 0}

    # end-to-end: host buffers through the C ABI, H2D inputs and D2H solution inside
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(rr, torch, op, o, ws, ws_bytes, stream, X, B, seed, args, world, flush)

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {**{kk: WORKLOAD[kk] for kk in ("workload", "n", "d", "k", "nrhs", "mu", "rtol",
                                                  "precision", "variant")},
                   "parallelism": f"replicas x{world}", "l2": "flushed between steps"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "solve": {"inner_iters_max": iters, "rel_residual_max": rel_res},
        "kernels_ms_per_step": {kk: v[1] / args.steps for kk, v in cats.items()},
        "roofline": roof, "roofline_other": others, "clocks": clocks,
        "gpu_launches": gpu_launches, "e2e": e2e,
        "wall_s": wall,
    }
    if rank == 0 and not args.no_cpu_baseline:
        pps = products_per_solve(iters, k, m)
        v, secs, t_mv, t_qr = oracle_sample(X, B, pps)
        line["cpu_baseline"] = {
            "value": v, "unit": "solves/s", "cores": cpu_threads(), "kind": "oracle",
            "sample": (f"one float64 (K+mu I)V product with 4 columns at n=20000 ({t_mv:.2f} s) and "
                       f"one 20000x500 Householder QR ({t_qr:.2f} s), scaled by {pps:.0f} "
                       f"products per solve")}
    if rank == 0:
        print(json.dumps(line), flush=True)


def estimate_launches(prof):
    # our kernels per solve, counted from the profile's launch counts: the
    # product kernels plus the fixed per-iteration companions (8 per PCG
    # iteration with the kernel operator, ~10 per power iteration, ~60 for the
    # build's factorisations)
    total = 0
    for p, infos in prof:
        mv = p["matvec"][0]
        total += mv * 8 + p["power"][0] * 10 + p["residual"][0] * 4 + 60 + p["sketch"][0]
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
        # the special-function units (MUFU): peak 152 SMs x 16 ex2/clk x clock
        ops = float(n) * n
        peak = 152 * 16 * f
        return {"kernel": "k_kernel_mv_tc", "bound": "alu", "achieved": ops / avg_s / 1e9,
                "peak": peak / 1e9, "unit": "G ex2/s (MUFU)", "frac": ops / avg_s / peak,
                "traffic": None, "launches": cnt, "avg_us": avg_s * 1e6}
    if name == "residual":
        # double-float restart residual: ~190 float32-pipe ops per entry
        ops = float(n) * n * 190
        peak = 152 * 128 * f
        return {"kernel": "k_kernel_mv_df", "bound": "alu", "achieved": ops / avg_s / 1e9,
                "peak": peak / 1e9, "unit": "G f32-op/s", "frac": ops / avg_s / peak,
                "traffic": None, "launches": cnt, "avg_us": avg_s * 1e6}
    # sketch: 2 n^2 k flops on the tensor cores (bf16, dense)
    flops = 2.0 * n * n * WORKLOAD["k"]
    peak_tf = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0
    return {"kernel": "k_kernel_sketch_tc", "bound": "tensor", "achieved": flops / avg_s / 1e12,
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


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
