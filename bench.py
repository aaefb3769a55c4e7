#!/usr/bin/env python
"""Benchmark of the CBC application (arXiv 2601.19650, Sec. III A) on one GB300.

Workload: MPO applied to an MPS and compressed by CBC, L=64 sites, d=2, MPS bond 128,
MPO bond 16, cap 128, complex64 Gaussian entries with unit Frobenius norm per tensor.
A step applies B independent instances (default 128; rank r uses seeds r*B .. r*B+B-1)
through cbc_apply_batched, which runs them as one lockstep group of 128; every
application is a full forward sweep with compressions and backward sweep with
CholeskyQR2, on inputs resident in HBM.  Several GPUs run independent replicas (no
collective on the data path); the step time is the maximum over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
    python bench.py --impl reference ...   # the FP64 CPU oracle, timed on the host
    python bench.py --sweep                # error vs runtime, the paper's benchmark (Sec. IV A)

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CBC applications/sec & TFLOP/s, mixed vs FP64 plain on 1 GB300 at rel err ≤1e-6"
WORKLOADS = {
    # the headline: MPO on MPS (config 2); a step is B instances in one lockstep group
    "mpo_mps": dict(workload="MPO on MPS, L=64, d=2, chi=128, D=16, max_bond=128, complex64 "
                             "Gaussian entries (unit Frobenius norm per tensor)",
                    L=64, d=2, chi=128, D=16, max_bond=128, input_dtype="complex64"),
    # TTNO on TTNS (config 3)
    "tree": dict(workload="TTNO on TTNS, perfect binary tree with 64 physical leaves (d=2) and "
                          "63 virtual nodes, state bond 64, operator bond 8, max_bond 64, "
                          "float32 Gaussian entries", L=6, d=2, chi=64, D=8, max_bond=64,
                 input_dtype="float32"),
    # the serving set (config 4): heterogeneous chains, instance j with seed j
    "serving": dict(workload="independent MPO.MPS instances, L ~ U{16..64}, chi in "
                             "{32,64,128,256}, D in {4,8,16,32}, d=2, max_bond = chi, float32",
                    input_dtype="float32"),
    # the paper's own random benchmark (Sec. IV A), MPS part: the error-vs-runtime sweep
    "paper": dict(workload="MPO on MPS, L=50, d=3, D_S=D_O=40, complex128 entries with real "
                           "and imaginary parts iid U[-0.5, 1], max_bond swept 2..40 step 2",
                  L=50, d=3, chi=40, D=40, input_dtype="complex128"),
    # the large tensor train (config 5)
    "large": dict(workload="MPO on MPS, L=100, d=4, chi=1024, D=32, max_bond=1024, complex64 "
                           "Gaussian entries", L=100, d=4, chi=1024, D=32, max_bond=1024,
                  input_dtype="complex64"),
}
DEFAULT_B = {"mpo_mps": 128, "tree": 8, "serving": 256, "large": 1, "paper": 1}
# instances per lockstep group (cbc_options.max_group) when --group is not given: the whole
# headline step in one group (larger groups fill more SMs in the per-matrix kernels)
DEFAULT_GROUP = {"mpo_mps": 128}
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64, nominal: the fallback when the DGEMM probe fails
# DRAM bytes per launch of a class's dominant kernel, read from an ncu capture of this
# workload; each entry names the summary under profiles/ it comes from.  A class whose
# kernel changed after its capture has no entry (traffic null).
PROFILED_TRAFFIC = {}
KERNEL_OF_CLASS = {"tridiag": "tridiag_cluster_kernel", "eig": "bisect32/invit/rank/backtransform",
                   "gemm_tc": "gemm_tc_kernel (+ operand slicing)", "cholqr": "chol_kernel + trsm",
                   "gemm_f64": "gemm_f64_kernel"}


def instance_seeds(rank: int, B: int):
    """Seeds of the B instances a rank applies: disjoint across ranks."""
    return [rank * B + j for j in range(B)]


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (the job's step time); x itself on one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, B: int, steps: int, t_max_ms: float) -> float:
    """Applications per second of the whole job: every rank's instances over the
    slowest rank's time."""
    return world * B * steps / (t_max_ms / 1e3)


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# --------------------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------------------
def make_workload(seed: int, sites: int = 0, workload: str = "mpo_mps"):
    """One instance of a tensor-train or tree workload (`sites` shortens a chain)."""
    from synth import make_problem
    cfg = {"mpo_mps": 2, "tree": 3, "large": 5, "paper": "P"}[workload]
    over = {"L": sites} if (sites > 0 and workload != "tree") else {}
    return make_problem(cfg, seed=seed, **over)


def make_workloads(workload: str, rank: int, B: int, sites: int = 0):
    """The B instances a rank applies per step."""
    if workload == "serving":
        from synth.networks import make_batch
        return make_batch(n=B, seed0=rank * B)
    return [make_workload(sd, sites, workload) for sd in instance_seeds(rank, B)]


def oracle_time(prob, reps: int = 1):
    """The FP64 oracle as it stands, timed on the host cores."""
    from oracle import cbc as ocbc
    t0 = time.perf_counter()
    res = None
    for _ in range(reps):
        res = ocbc.cbc(prob.state.parent, prob.state.tensors, prob.op.tensors, prob.max_bond,
                       prob.tol)
    return (time.perf_counter() - t0) / reps, res


def measure_fp64_peak(device, n: int = 8192, reps: int = 3):
    """FP64 throughput of a cuBLAS DGEMM (torch.matmul, n^3, 2 n^3 flops) on this GPU:
    the best of `reps` back-to-back runs after one warm-up, timed with CUDA events.  The
    FP64 rooflines of the report use it as their peak (no FP64 figure is driver-written)."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device=device)
    b = torch.randn(n, n, dtype=torch.float64, device=device)
    c = a @ b
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b, c
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best / 1e3) / 1e12, {"gemm": f"cuBLAS DGEMM via torch.matmul, {n}^3",
                                               "best_ms": best, "reps": reps}


def blas_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def run_sweep(args, local):
    """Error against runtime of one application of the paper's benchmark MPS/MPO (Sec. IV A)
    for max_bond = 2, 4, ..., 40, in both precisions, for CBC and for the comparison methods
    of Sec. III C built here (Zip-Up with the same cap, SRC with sketch width s = max_bond and
    seeded Gaussian random matrices, the direct method at max_bond 4, 20 and 40 in the mixed
    path, one timed run).  The error is ||O psi - psi'|| /
    ||O psi|| from ||O psi||^2 (one exact FP64 sandwich contraction, the oracle's
    chain_applied_norm2), ||psi'||^2 and the overlap <psi'|O psi> (chain_applied_overlap);
    its floor is ~1e-8 (FP64 cancellation in the sum of the three)."""
    import numpy as np
    import torch

    from oracle import metrics
    from paper_2601_19650_gb300 import _cbc, build as _build
    from synth import make_problem, sketch_matrices

    _build.build()
    torch.cuda.set_device(local)
    p = make_problem("P", seed=0)
    st, op = p.state, p.op
    t0 = time.perf_counter()
    n2 = metrics.chain_applied_norm2(st.tensors, op.tensors)
    t_norm = time.perf_counter() - t0
    hs = _cbc.create_from_host(st.parent, st.phys, st.bond, st.tensors, "state")
    ho = _cbc.create_from_host(op.parent, op.phys, op.bond, op.tensors, "op")
    shape = _cbc.output_shape_fn(st.parent, st.phys)
    methods = [m for m in args.sweep_methods.split(",") if m]

    def apply(method, opt, mb, om):
        if method == "cbc":
            return _cbc.cbc_apply(hs, ho, mb, 0.0, opt)
        if method == "zipup":
            return _cbc.zipup_apply(hs, ho, mb, 0.0, opt)
        if method == "direct":
            return _cbc.direct_apply(hs, ho, mb, 0.0, opt)
        return _cbc.src_apply(hs, ho, mb, om, opt)

    rows = []
    for mb in range(2, 41, 2):
        row = {"max_bond": mb}
        om = sketch_matrices(st.phys, mb, seed=0, cplx=True)
        for method in methods:
            # the direct method contracts to bond D_S D_O = 1600 first (~6 GB, seconds per
            # application): a few bonds only
            if method == "direct" and mb not in (4, 20, 40):
                continue
            precs = (("mixed", _cbc.CBC_PREC_MIXED), ("fp64", _cbc.CBC_PREC_FP64))
            if method == "direct":
                precs = precs[:1]
            for name, prec in precs:
                key = name if method == "cbc" else f"{method}_{name}"
                opt = _cbc.make_options(prec)
                try:
                    _cbc.ttn_destroy(apply(method, opt, mb, om))  # warm-up
                    times = []
                    out = None
                    for _ in range(1 if method == "direct" else 3):
                        torch.cuda.synchronize()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record()
                        if out is not None:
                            _cbc.ttn_destroy(out)
                        out = apply(method, opt, mb, om)
                        e1.record()
                        e1.synchronize()
                        times.append(e0.elapsed_time(e1))
                except _cbc.CBCError as exc:
                    row[key] = {"error": str(exc)[:160]}
                    continue
                tens, bonds, log_norm = _cbc.fetch_network(out, shape, True)
                _cbc.ttn_destroy(out)
                # ||O psi - psi'||^2 = ||O psi||^2 + ||psi'||^2 - 2 Re <psi'|O psi>, relative
                # to ||O psi||^2 (the overlap by an FP64 sandwich: no assumption that psi'
                # is an exact projection)
                # ||psi'|| by the oracle's QR sweep (the mixed path's isometries are exact
                # only to its precision, so the root tensor's norm alone is not ||psi'||)
                sc2 = float(np.exp(2.0 * log_norm))
                out2 = sc2 * metrics.tree_norm(st.parent, tens) ** 2
                ov = float(np.exp(log_norm)) * metrics.chain_applied_overlap(
                    st.tensors, op.tensors, tens).real
                err = float(np.sqrt(max(0.0, 1.0 + out2 / n2 - 2.0 * ov / n2)))
                row[key] = {"ms": statistics.median(times), "rel_err": err,
                            "max_out_bond": int(max(bonds))}
        rows.append(row)
    _cbc.ttn_destroy(hs)
    _cbc.ttno_destroy(ho)
    line = {"metric": "relative error ||O psi - psi'|| / ||O psi|| against runtime, paper "
                      "benchmark (Sec. IV A): CBC and the Sec. III C comparators",
            "unit": "ms per application",
            "n_gpus": 1, "data": "synthetic", "dtype": "bf16-slices+f64 | f64",
            "config": dict(WORKLOADS["paper"], seed=0, methods=methods,
                           direct_bonds=[4, 20, 40],
                           src_sketch="s = max_bond, Gaussian (x+iy)/sqrt(2), seed 0"),
            "norm_note": f"||O psi||^2 by an exact FP64 sandwich contraction on the host "
                         f"({t_norm:.1f} s), <psi'|O psi> likewise per result; errors below "
                         f"~1e-8 sit at FP64 cancellation",
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    prob = make_workloads(args.workload, 0, 1)[0]
    for _ in range(args.warmup):
        oracle_time(prob)
    t = 0.0
    for _ in range(args.steps):
        dt, _ = oracle_time(prob)
        t += dt
    value = args.steps / t
    line = {"metric": METRIC, "value": value, "unit": "applications/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": dict(WORKLOADS[args.workload], precision="fp64 (numpy, host)",
                           l2="n/a (host)"),
            "cpu_baseline": {"value": value, "unit": "applications/s", "cores": blas_threads(),
                             "kind": "oracle",
                             "sample": "one full application of the workload per step (seed 0)"},
            "e2e": {"value": value, "unit": "applications/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--concurrency", type=int, default=0,
                    help="independent applications per step (seeds rank*B .. rank*B+B-1), "
                         "run by cbc_apply_batched: same-shape instances go in lockstep "
                         "groups (--group; one launch per step per group); default per "
                         "workload: mpo_mps 128, tree 8, serving 256, large 1")
    ap.add_argument("--workload", default="mpo_mps", choices=sorted(WORKLOADS),
                    help="mpo_mps (the headline), tree, serving, large")
    ap.add_argument("--sites", type=int, default=0,
                    help="shorter chains for profiling captures (default: the workload's 64)")
    ap.add_argument("--no-fp64-arm", action="store_true",
                    help="skip timing the same step in plain FP64 (the ratio's denominator)")
    ap.add_argument("--sweep", action="store_true",
                    help="error-vs-runtime sweep of the paper's benchmark (max_bond 2..40) "
                         "instead of the throughput step; prints one line of rows")
    ap.add_argument("--sweep-methods", default="cbc,zipup,src,direct",
                    help="methods of --sweep (comma separated: cbc, zipup, src, direct)")
    ap.add_argument("--tol", type=float, default=0.0,
                    help="truncation tolerance of every compression besides max_bond (Sec. V; "
                         "the large workload's second run uses 1e-8)")
    ap.add_argument("--group", type=int, default=0,
                    help="most instances per lockstep group (0: the workload's default, "
                         "128 for mpo_mps, else the library's 32)")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the FP64 arm (after one warm-up step)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank, world, local = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.sweep:
        return run_sweep(args, local) if rank == 0 else 0

    import numpy as np
    import torch

    from paper_2601_19650_gb300 import _cbc, build as _build

    _build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    B = args.concurrency if args.concurrency > 0 else DEFAULT_B[args.workload]
    if args.group <= 0:
        args.group = DEFAULT_GROUP.get(args.workload, 0)
    streams = [torch.cuda.Stream() for _ in range(B)]
    stream = streams[0]
    sptr = stream.cuda_stream

    # precision of the headline number: mixed when built, else fp64
    prec_name = args.precision
    probs = make_workloads(args.workload, rank, B, args.sites)
    for p in probs:
        p.tol = args.tol
    prob = probs[0]
    st, op = prob.state, prob.op
    hs_list, ho_list = [], []
    for p, sm in zip(probs, streams):
        dev_st = [torch.from_numpy(t).to(f"cuda:{local}") for t in p.state.tensors]
        dev_op = [torch.from_numpy(t).to(f"cuda:{local}") for t in p.op.tensors]
        torch.cuda.synchronize()
        hs_list.append(_cbc.create_from_device(p.state.parent, p.state.phys, p.state.bond, dev_st,
                                               "state", sm.cuda_stream))
        ho_list.append(_cbc.create_from_device(p.op.parent, p.op.phys, p.op.bond, dev_op, "op",
                                               sm.cuda_stream))
        torch.cuda.synchronize()
    hs, ho = hs_list[0], ho_list[0]

    def apply_once(prec):
        opt = _cbc.make_options(prec, max_group=args.group)
        if B == 1:
            return [_cbc.cbc_apply(hs, ho, prob.max_bond, prob.tol, opt)]
        return _cbc.cbc_apply_batched(hs_list, ho_list, [p.max_bond for p in probs], [p.tol for p in probs],
                                      opt)

    def destroy(outs):
        for o in outs:
            _cbc.ttn_destroy(o)

    if prec_name == "auto":
        prec_name = "mixed"
    prec = _cbc.CBC_PREC_MIXED if prec_name == "mixed" else _cbc.CBC_PREC_FP64

    # FP64 peak for the FP64 rooflines: a cuBLAS DGEMM on this GPU (untimed region)
    try:
        fp64_peak, fp64_peak_info = measure_fp64_peak(f"cuda:{local}")
        fp64_note = "of measured cuBLAS DGEMM"
    except Exception as exc:  # e.g. out of memory: the nominal figure, said so
        fp64_peak, fp64_peak_info = FP64_NOMINAL_TFLOPS, {"error": str(exc)[:120]}
        fp64_note = "of nominal (152 SMs x 2 DFMA/clk x ~2.06 GHz)"

    # L2 flush buffer (larger than the 129 MB L2), written between timed steps
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")

    for _ in range(args.warmup):
        destroy(apply_once(prec))
    torch.cuda.synchronize()

    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except (ValueError, IndexError):
            gpu_index = local
    clocks = ClockSampler(gpu_index)

    def timed_arm(prec_arm, steps, single=False):
        """`steps` timed steps (L2 flushed before each, untimed); each step is the B
        instances through cbc_apply_batched, or instance 0 alone through cbc_apply.
        Returns the summed CUDA-event time and the last step's outputs."""
        t_ms, last_outs = 0.0, None
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            for sm in streams[1:]:
                sm.wait_event(e0)
            # an NVTX range per timed step: profilers can select exactly one step's launches
            torch.cuda.nvtx.range_push("timed_step")
            if single:
                outs = [_cbc.cbc_apply(hs, ho, prob.max_bond, prob.tol, _cbc.make_options(prec_arm))]
            else:
                outs = apply_once(prec_arm)
            torch.cuda.nvtx.range_pop()
            for sm in streams[1:]:
                ev = torch.cuda.Event()
                ev.record(sm)
                stream.wait_event(ev)
            e1.record(stream)
            e1.synchronize()
            t_ms += e0.elapsed_time(e1)
            if last_outs is not None:
                destroy(last_outs)
            last_outs = outs
        return t_ms, last_outs

    _cbc.cbc_stats_reset()
    _cbc.cbc_stats_enable(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    total_ms, last = timed_arm(prec, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clock_info = clocks.stop()
    stats = _cbc.cbc_stats_read()
    _cbc.cbc_stats_enable(False)

    t_max = max_over_ranks(total_ms, dist, f"cuda:{local}")
    value = whole_job_value(world, B, args.steps, t_max)
    ms_per_step = t_max / args.steps

    # per-kernel-class roofline of the dominant class
    issued = stats.pop("tc_issued", {"flops": 0.0})["flops"]  # tensor-pipe flops, no time
    classes = {k: v for k, v in stats.items() if v["ms"] > 0}
    dom = max(classes, key=lambda k: classes[k]["ms"]) if classes else None
    flops_per_app = sum(v["flops"] for v in stats.values()) / args.steps
    bf16_peak, bf16_note = 1700.0, "of fallback"
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        bf16_peak = float(mp.get("bf16_tflops_sustained") or mp.get("bf16_tflops"))
        bf16_note = "of measured sustained bf16"
    except (OSError, ValueError, TypeError):
        pass
    roofline_tc = None
    if "gemm_tc" in classes:
        d = classes["gemm_tc"]
        sec = d["ms"] / 1e3
        roofline_tc = {"bound": "tensor", "kernel_class": "gemm_tc",
                       "achieved": issued / sec / 1e12, "peak": bf16_peak, "unit": "TFLOP/s",
                       "frac": issued / sec / 1e12 / bf16_peak,
                       "algorithmic_tflops": d["flops"] / sec / 1e12,
                       "note": "bf16 slice products issued on the tensor pipe (padded, "
                               f"real-embedded shapes) over the class's event time, {bf16_note}"}
    roofline = None
    if dom is not None:
        d = classes[dom]
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12
        if dom == "gemm_tc":
            peak, bound = bf16_peak, "tensor"
            achieved = issued / (d["ms"] / 1e3) / 1e12
            note = f"bf16 slice products issued on the tensor pipe, {bf16_note}"
        else:
            peak, bound = fp64_peak, "alu"
            note = (f"FP64-equivalent flops over the class's event time, {fp64_note} "
                    f"({fp64_peak:.3f} TFLOP/s)")
        # the captured traffic belongs to the default step (32 instances, 64 sites)
        default_step = args.workload == "mpo_mps" and B == 32 and args.sites == 0
        prof = PROFILED_TRAFFIC.get(dom, {}) if default_step else {}
        roofline = {"bound": bound, "kernel_class": dom, "kernel": KERNEL_OF_CLASS.get(dom, dom),
                    "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
                    "traffic": prof.get("bytes_per_launch"),
                    "traffic_source": prof.get("source") if prof.get("bytes_per_launch") else None,
                    "note": note,
                    "launch_groups": d["groups"], "ms_total": d["ms"],
                    "share_of_step": d["ms"] / total_ms}

    line = {"metric": METRIC, "value": value, "unit": "applications/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec_name == "fp64" else "bf16-slices+f64",
            "data": "synthetic",
            "config": dict(WORKLOADS[args.workload], precision=prec_name, tol=args.tol, concurrent_applications=B,
                           batching=(f"cbc_apply_batched: lockstep groups of <= "
                                     f"{args.group or 32} same-shape instances")
                           if B > 1 else "single cbc_apply",
                           parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                           l2="flushed between steps (256 MB write, untimed)"),
            "tflops": flops_per_app / B * value / 1e12,
            "algorithmic_gflop_per_app": flops_per_app / B / 1e9,
            "kernel_classes": {k: {"ms_per_step": v["ms"] / args.steps,
                                   "launches_per_step": v["launches"] / args.steps}
                               for k, v in stats.items() if v["launches"]},
            "roofline": roofline,
            "roofline_tensor": roofline_tc,
            "gpu_launches": int(sum(v["launches"] for v in stats.values())),
            "clocks": clock_info,
            "fp64_peak": dict(fp64_peak_info, tflops=fp64_peak, note=fp64_note)}

    if args.sites > 0:  # a shortened chain: not the headline workload
        line["config"]["L"] = args.sites
        line["config"]["workload"] = line["config"]["workload"].replace("L=64", f"L={args.sites}")
    # parity of this run's output with the oracle, and the oracle's own time
    ref = None
    shape0 = _cbc.output_shape_fn(st.parent, st.phys)
    cplx0 = bool(np.iscomplexobj(st.tensors[0]))

    def err_vs_oracle(out):
        from oracle import metrics
        tens, bonds, log_norm = _cbc.fetch_network(out, shape0, cplx0)
        return metrics.rel_err(st.parent, tens, ref.tensors, log_norm, 0.0)

    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "large":
        line["cpu_baseline"] = None
        line["cpu_baseline_note"] = "not timed: the FP64 oracle needs hours per application here"
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        # instance 0 against the oracle; the oracle timed on instances 0, 1, ... until about
        # 20 s of host time (a bounded sample of the step's instances)
        t_or, ref = oracle_time(prob)
        line["rel_err_vs_oracle"] = err_vs_oracle(last[0])
        n_or, t_sum = 1, t_or
        while t_sum < 20.0 and n_or < len(probs):
            t_sum += oracle_time(probs[n_or])[0]
            n_or += 1
        line["cpu_baseline"] = {"value": n_or / t_sum, "unit": "applications/s",
                                "cores": blas_threads(), "kind": "oracle",
                                "sample": f"full applications of instances 0..{n_or - 1} of the "
                                          f"step (seeds {rank * B}..{rank * B + n_or - 1})"}
    if last is not None:
        destroy(last)

    # the denominator of the headline ratio: the same B instances in plain FP64 through
    # cbc_apply_batched, and instance 0 alone through cbc_apply ("plain FP64 GPU CBC"),
    # timed like the headline step
    if (prec == _cbc.CBC_PREC_MIXED and not args.no_fp64_arm
            and args.workload in ("mpo_mps", "tree")):
        f64 = _cbc.CBC_PREC_FP64
        destroy(timed_arm(f64, 1)[1])
        t64, out64 = timed_arm(f64, args.fp64_steps)
        t64 = max_over_ranks(t64, dist, f"cuda:{local}")
        n1 = max(3, args.fp64_steps)
        destroy(timed_arm(f64, 1, single=True)[1])
        t1, out1 = timed_arm(f64, n1, single=True)
        t1 = max_over_ranks(t1, dist, f"cuda:{local}")
        fp64_value = whole_job_value(world, B, args.fp64_steps, t64)
        fp64_single = world * n1 / (t1 / 1e3)
        line["fp64"] = {"value": fp64_value, "unit": "applications/s",
                        "ms_per_step": t64 / args.fp64_steps, "steps": args.fp64_steps,
                        "warmup": 1, "batching": line["config"]["batching"],
                        "single_application_value": fp64_single,
                        "single_application_ms": t1 / n1}
        line["mixed_over_fp64"] = value / fp64_value
        line["mixed_over_fp64_single"] = value / fp64_single
        if ref is not None:
            line["fp64"]["rel_err_vs_oracle"] = err_vs_oracle(out64[0])
            line["fp64"]["single_rel_err_vs_oracle"] = err_vs_oracle(out1[0])
        destroy(out64)
        destroy(out1)

    # end to end through the C ABI with host buffers: H2D of the inputs, the application,
    # D2H of every output tensor, each step
    if not args.no_e2e:
        pins = [([torch.from_numpy(t).pin_memory().numpy() for t in p.state.tensors],
                 [torch.from_numpy(t).pin_memory().numpy() for t in p.op.tensors]) for p in probs]
        h2d = sum(sum(t.nbytes for t in a) + sum(t.nbytes for t in b) for a, b in pins)
        shapes = [_cbc.output_shape_fn(p.state.parent, p.state.phys) for p in probs]
        cplxs = [bool(np.iscomplexobj(p.state.tensors[0])) for p in probs]
        d2h = 0
        e2e_t = 0.0
        n_e2e = max(2, args.steps)
        for k in range(n_e2e):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ha = [_cbc.create_from_host(p.state.parent, p.state.phys, p.state.bond, pa, "state",
                                        sm.cuda_stream) for p, (pa, _), sm in zip(probs, pins, streams)]
            hb = [_cbc.create_from_host(p.op.parent, p.op.phys, p.op.bond, pb, "op", sm.cuda_stream)
                  for p, (_, pb), sm in zip(probs, pins, streams)]
            opt = _cbc.make_options(prec, max_group=args.group)
            if B == 1:
                outs = [_cbc.cbc_apply(ha[0], hb[0], prob.max_bond, prob.tol, opt)]
            else:
                outs = _cbc.cbc_apply_batched(ha, hb, [p.max_bond for p in probs], [p.tol for p in probs], opt)
            d2h = 0
            for o, shp, cx in zip(outs, shapes, cplxs):
                tens, bonds, _ = _cbc.fetch_network(o, shp, cx)
                d2h += sum(t.nbytes for t in tens)
            e2e_t += time.perf_counter() - t0
            destroy(outs + ha)
            for h in hb:
                _cbc.ttno_destroy(h)
        line["e2e"] = {"value": world * B * n_e2e / e2e_t, "unit": "applications/s",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    for h in hs_list:
        _cbc.ttn_destroy(h)
    for h in ho_list:
        _cbc.ttno_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
