#!/usr/bin/env python3
"""Benchmark of the GB300 PC-stable skeleton search (reversed-order schedule).

One step = the whole hot path on one synthetic input resident in HBM:
pc_corr (standardise + correlation GEMM) followed by pc_skeleton (every stage
of the skeleton search with PC-stable deletion).  Default workload: the p=1000
Erdos-Renyi SEM (expected degree 10, n=20000, FP32 data, alpha=0.01, all
stages, conventional order), with the proposal network trained on 200 seeded
p=200 SEMs of the same recipe; --workload p95_dense runs the dense p=95 SEM in
the reversed order (Algorithm 2).

Prints ONE JSON line.  ``value`` is canonical CI tests per second of step time,
counted in the lexicographic order (the tests the sequential algorithm of the
oracle executes, so the CPU baseline and every GPU configuration are counted
alike; the learned order reaches the same skeleton with fewer tests); the L2 is
flushed (a 512 MB write) before every timed step.  --impl reference times the FP64 CPU oracle
on the same workload (the reference arm).
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import signal
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CI tests/s and skeleton time at 1 GB300: learned+mixed vs plain GPU, identical skeleton"
UNIT = "CI tests/s"
FP64_PEAK_TFLOPS = 1.25     # nominal GB300 FP64 (CUDA cores)
SM_COUNT, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.070
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_GHZ / 1000.0   # 80.5


def dominant_class(tim):
    """The kernel class with the most device time among those with algorithmic work.
    The stage bookkeeping (head, commit, degrees, tail: counts, scans, sepset records)
    and the proposal scoring have none of their own; their time stays in class_ms and
    the largest class of all is named beside the roofline.  corr_gemm is a part of
    corr and is reported on its own line (roofline_gemm)."""
    from paper_2109_04626_gb300 import fastpc as fp
    return max((c for c in fp.TIMING_CLASSES if c not in ("bookkeeping", "scoring", "corr_gemm")),
               key=lambda c: tim[c][0])


# the kernels behind each timing class that the roofline names
CLASS_KERNELS = {
    "ci_direct": "ci_pairwarp_kernel (l = 1, 2, degree > 32: a warp per ordered pair) + ci_node_kernel "
                 "(degree <= 128: corr block in shared memory) + ci_lane_kernel (other stages l <= 12) + "
                 "ci_direct_kernel (one warp per test) + ci_redecide_kernel (FP64 pass)",
    "ci_complement": "ci_complement_kernel (FP64, from neighbourhood precision blocks)",
    "prec": "prec_update_kernel (neighbourhood precision blocks, FP64)",
    "stage_a": "stage_a sweep inverse (FP64)",
    "corr": "pc_corr: column statistics, standardisation, correlation GEMM",
    "stage_loop": "stage_loop_kernel (one cooperative kernel over the complement-only stages: head, FP32-first "
                  "complement tests, commit, degrees, tail, FP64 precision downdates, grid barriers between)",
}


def measured_peaks():
    """(bf16 TFLOP/s burst, HBM GB/s, source): the machine's measured peaks when the
    file is present, else the fallback figures."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, 6800.0, "of fallback"


# DRAM bytes (read + write) per launch of a class's kernels, from one ncu
# capture of the current kernels (the profile summary of that workload and
# kernel gives the command and the per-launch figures); absent: not captured
# since the kernels last changed (the roofline's traffic is then null)
DRAM_BYTES_PER_LAUNCH = {("p1000_er", "ci_direct"): 1.677e7}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="p1000_er",
                    choices=["p20_fp64", "p95_dense", "p500_powerlaw", "p1000_er", "many64", "paper_sweep", "power"],
                    help="many64: 64 independent SEMs (p in [50,400], edge prob in [0.05,0.3], "
                         "n in [2000,20000]), conventional order; paper_sweep: the paper's "
                         "simulation (p = 15..100, both orders, CI tests per graph)")
    ap.add_argument("--sweep-mc", type=int, default=100, help="paper_sweep: graphs per size")
    ap.add_argument("--power-datasets", type=int, default=500, help="power: datasets of the 10-node graph")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--train-seeds", type=int, default=None,
                    help="training SEMs of the proposal network (default: 200 for p1000_er, "
                         "whose network is trained on p=200 SEMs; 24 otherwise)")
    ap.add_argument("--learned-max-level", type=int, default=None,
                    help="largest stage the proposal network scores (library default if unset)")
    ap.add_argument("--corr-only", action="store_true",
                    help="time only pc_corr (standardise + tensor-core correlation GEMM) on the workload")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shape of the test kernels (no pc_autotune)")
    ap.add_argument("--opt", action="append", default=[], metavar="KEY=VALUE",
                    help="a handle option (pc_set_opt) for the timed handle, e.g. pair_warp=0 or node_dmax=0; "
                         "repeatable")
    ap.add_argument("--graph", type=int, default=1,
                    help="1: stage loop as one CUDA graph (default); 0: host-driven launches "
                         "(for ncu launch lists, which do not enter conditional graph bodies)")
    return ap.parse_args()


def workload(name):
    from paper_2109_04626_gb300 import sem
    cfg = {w["name"]: c for c, w in sem.WORKLOADS.items()}[name]
    w = dict(sem.WORKLOADS[cfg])
    s = sem.make(cfg)
    # the p=500 and p=1000 sparse workloads run the conventional order (Algorithm 1):
    # their stage l=p-2 leaves moral graphs of mean degree ~46-49 whose exhaustive
    # reversed enumeration is beyond 1e12 tests
    w["order"] = 1 if cfg in (1, 2) else 0
    w["cfg"] = cfg
    return s, w


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region.

    Samples are taken every PERIOD_MS; each carries nvidia-smi's own timestamp, and
    the summary keeps those taken between entering and leaving the ``with`` block (the
    timed region), so that a region of a few tens of milliseconds still holds samples.
    Entering waits (bounded) for the first sample, so the sampler is running when the
    region starts.  Where no timestamp parses, every sample is kept."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20
    START_WAIT_S = 2.0

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t_begin = self.t_end = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.monotonic() + self.START_WAIT_S
            while not self.lines and self.proc.poll() is None and time.monotonic() < deadline:
                time.sleep(0.005)
        except (OSError, FileNotFoundError):
            self.proc = None
        self.t_begin = time.time()
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        self.t_end = time.time()
        if self.proc:
            time.sleep(2 * self.PERIOD_MS / 1000.0)      # the sample that covers the end
            try:
                self.proc.send_signal(signal.SIGINT)     # its loop's own exit: output flushed
                self.proc.wait(timeout=5)
            except (subprocess.TimeoutExpired, OSError):
                self.proc.kill()
            self.t.join(timeout=5)

    @staticmethod
    def _stamp(s):
        try:
            return datetime.datetime.strptime(s.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self):
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((self._stamp(f[0]), float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        stamped = [r for r in rows if r[0] is not None]
        window = "timed region"
        inside = [r for r in stamped if self.t_begin is not None and self.t_end is not None
                  and self.t_begin <= r[0] <= self.t_end]
        if inside:
            rows = inside
        elif rows:
            window = "whole sampler run (no sample stamped inside the region)"
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = {nm for r in rows for nm, v in zip(names, r[3]) if v.lower() == "active"}
        sm = [r[1] for r in rows]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": rows[-1][2] if rows else None,
                "reasons": sorted(reasons), "samples": len(sm), "period_ms": self.PERIOD_MS, "window": window}


def dist_setup(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def oracle_run(X, w):
    """One full oracle pass (Pearson + skeleton), returns (seconds, result)."""
    import oracle
    t0 = time.perf_counter()
    C = oracle.pearson(X)
    R = oracle.skeleton(C, X.shape[0], w["alpha"], w["max_level"], reversed_order=bool(w["order"]))
    return time.perf_counter() - t0, R


def cpu_baseline(X, w, budget_s=20.0):
    """The oracle as it stands on the host cores, on a bounded sample: whole runs
    of the workload repeated until ~budget_s (at least one run)."""
    import oracle
    runs, tot_t, tot_tests, R = 0, 0.0, 0, None
    while runs == 0 or (tot_t < budget_s and runs < 20 and tot_t / runs * (runs + 1) < budget_s * 1.5):
        dt, R = oracle_run(X, w)
        runs += 1
        tot_t += dt
        tot_tests += R["tests_total"]
        if dt > budget_s:
            break
    return {"value": tot_tests / tot_t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{runs} full run(s) of the workload (Pearson + skeleton), {tot_t:.1f} s"}, R


def run_reference(args):
    rank, world, local = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), 0
    if rank != 0:
        return 0
    if args.workload in ("paper_sweep", "power"):
        # these metrics are counts and fractions, which the oracle recomputes inside them
        print(json.dumps({"impl": "reference", "unavailable": f"{args.workload} reports counts and fractions; "
                          "the oracle recomputes them inside the workload itself"}), flush=True)
        return 0
    if args.workload == "many64":
        # a bounded sample: the 8 smallest of the 64 instances per step
        from paper_2109_04626_gb300 import sem
        inst = sorted(sem.make_many(MANY["count"]), key=lambda s_: s_.X.shape[1])[:8]
        w = {"name": "many64", "p": sum(s_.X.shape[1] for s_ in inst), "n": max(s_.X.shape[0] for s_ in inst),
             "alpha": MANY["alpha"], "max_level": -1, "order": 0}
        sample = "the 8 smallest of the 64 instances (Pearson + skeleton) per step"
        Xs = [s_.X for s_ in inst]
    else:
        s, w = workload(args.workload)
        Xs = [s.X]
        sample = "full run(s) of the workload"

    def one():
        dt, nt = 0.0, 0
        for X in Xs:
            d_, R = oracle_run(X, w)
            dt += d_
            nt += R["tests_total"]
        return dt, nt
    for _ in range(max(0, args.warmup)):
        one()
    times, tests = [], 0
    for _ in range(args.steps):
        dt, nt = one()
        times.append(dt)
        tests += nt
    tot = sum(times)
    import oracle
    val = tests / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w["name"], "p": w["p"], "n": w["n"], "alpha": w["alpha"],
                       "max_level": w["max_level"], "order": "reversed" if w["order"] else "conventional",
                       "l2": "inputs on the host; oracle runs on CPU cores"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{args.steps} step(s): {sample}"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_corr_only(args, fp, X, w, stream, flush):
    """pc_corr alone: FP64 column statistics, standardised planes and the BF16x3
    tensor-core correlation GEMM (the FP64 matrix is left lazy in the conventional order)."""
    import torch
    n, p = X.shape
    pc = fp.PC(n, p, w["alpha"], w["max_level"], order=0, precision=2)
    fp.pc_set_stream(pc.h, stream)
    Xd = torch.from_numpy(X).cuda()
    for _ in range(args.warmup):
        pc.corr(Xd)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pc.corr(Xd)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    flops = 2.0 * n * p * (p + 1) / 2           # useful flops of the symmetric product
    t = float(np.mean(ms)) * 1e-3
    print(json.dumps({"metric": "correlation (pc_corr) time", "value": float(np.mean(ms)), "unit": "ms",
                      "higher_is_better": False, "config": {"workload": w["name"], "p": p, "n": n},
                      "tensor_core_gemm": bool(fp.pc_get_opt(pc.h, "tensor_core_gemm")),
                      "useful_tflops": flops / t / 1e12}), flush=True)
    pc.close()
    return 0


def run_ours(args):
    import torch
    from paper_2109_04626_gb300 import fastpc as fp
    rank, world, local = dist_setup(args)
    fp.load()
    s, w = workload(args.workload)
    X = s.X
    n, p = X.shape
    dev = torch.device("cuda", torch.cuda.current_device())
    Xd = torch.from_numpy(X).to(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    if args.corr_only:
        return run_corr_only(args, fp, X, w, stream, flush)

    def make(precision, complement, graph=1):
        pc = fp.PC(n, p, w["alpha"], w["max_level"], order=w["order"], precision=precision,
                   complement=complement, graph=graph)
        fp.pc_set_stream(pc.h, stream)
        return pc

    mixed_prec = 0 if w["cfg"] == 1 else 2
    pc = make(mixed_prec, 1, graph=args.graph)
    for kv in args.opt:
        key, val = kv.split("=", 1)
        fp.pc_set_opt(pc.h, key.strip(), float(val))
    adj_d = torch.empty((p, p), dtype=torch.uint8, device=dev)

    def step(pcx):
        pcx.corr(Xd)
        _, st = pcx.skeleton(adj_d)
        return st

    def timed_steps(pcx, k):
        out, st = [], None
        for _ in range(k):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = step(pcx)
            b.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return float(np.mean(out)), st

    # proposal network: trained on plain-run outcomes of other seeds of the same recipe
    # (untimed); the timed configuration then enumerates in its order
    learned = None
    train_seeds = args.train_seeds if args.train_seeds is not None else (200 if w["cfg"] == 4 else 24)
    if not args.no_learned:
        from paper_2109_04626_gb300 import proposal, sem as _sem
        t0 = time.perf_counter()
        base = 1000 * w["cfg"] + 100
        # training SEMs: the workload's recipe at its own size, except p=1000 ER,
        # whose network is trained on p=200 SEMs of the same expected degree
        tp_, tn_ = (200, 5000) if w["cfg"] == 4 else (p, n)

        def make_X(sd):
            rng = np.random.Generator(np.random.PCG64(base + sd))
            if w["prob"] is None:
                dag, W_, order_ = _sem.powerlaw_dag(tp_, rng)
            else:
                prob = 10.0 / (tp_ - 1) if w["cfg"] == 4 else w["prob"]
                dag, W_, order_ = _sem.er_dag(tp_, prob, rng)
            Xs = _sem.sample(W_, order_, tn_, rng)
            return Xs.astype(np.float32) if w["dtype"] == "float32" else Xs

        # at most 100k rows of each training run (seeded draw): 200 p=200 runs give
        # about 1.6M rows each, far more than the 16->128->128->1 network needs
        feats, labels = proposal.collect(make_X, range(train_seeds), w["alpha"], w["order"],
                                         w["max_level"], mixed_prec, max_rows_per_seed=100_000)
        loss = proposal.train(pc.h, feats, labels, epochs=6, batch=8192, lr=2e-3, seed=1)
        if args.learned_max_level is not None:
            fp.pc_set_opt(pc.h, "learned_max_level", args.learned_max_level)
        learned = {"train_rows": int(labels.shape[0]), "train_seeds": train_seeds,
                   "train_sems": f"p={tp_}, n={tn_}",
                   "final_loss": loss, "train_s": time.perf_counter() - t0,
                   "max_level": int(fp.pc_get_opt(pc.h, "learned_max_level"))}
        fp.pc_set_opt(pc.h, "learned", 1)

    for _ in range(args.warmup):
        st = step(pc)
    torch.cuda.synchronize()
    # launch shape of the test kernels for this problem (untimed; results do not depend
    # on it), chosen for the configuration that is timed; the lexicographic order below
    # runs with the same shape, so the two orders differ in the enumeration order only
    tune = fp.pc_autotune(pc.h, 2) if not args.no_autotune else None

    # lexicographic order: its canonical count is the oracle's, the unit of the metric
    fp.pc_set_opt(pc.h, "learned", 0)
    for _ in range(args.warmup):
        step(pc)
    lex_ms, lex_st = timed_steps(pc, max(3, min(args.steps, 5)))
    adj_lex = adj_d.cpu().numpy()
    tests_unit = lex_st["tests_canonical"]
    if learned is not None:
        fp.pc_set_opt(pc.h, "learned", 1)

    for _ in range(args.warmup):
        st = step(pc)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    barrier(world)
    torch.cuda.synchronize()
    l0 = fp.pc_kernel_launches()
    with ClockSampler(local if world > 1 else torch.cuda.current_device()) as clk:
        # the NVTX range lets a profiler select exactly the timed steps
        torch.cuda.nvtx.range_push("bench_timed")
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            stats.append(step(pc))
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    launches = fp.pc_kernel_launches() - l0
    barrier(world)
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = float(np.mean(ms))
    t_max = max_over_ranks(sum(ms) / 1000.0, world)
    total_tests = sum_over_ranks(float(tests_unit * args.steps), world)
    value = total_tests / t_max
    adj_ours = adj_d.cpu().numpy()
    if learned is not None:
        learned.update({"tests_canonical": stats[-1]["tests_canonical"],
                        "tests_executed": stats[-1]["tests_executed"], "ms_per_step": ms_step,
                        "identical_skeleton": bool(np.array_equal(adj_ours, adj_lex))})

    # per-kernel-class device time of one more step (CUDA events on the launching stream)
    fp.pc_set_opt(pc.h, "timing", 1)
    fp.pc_timing(pc.h, reset=True)
    flush.zero_()
    st_t = step(pc)
    tim = fp.pc_timing(pc.h, reset=True)
    fp.pc_set_opt(pc.h, "timing", 0)
    cls = fp.TIMING_CLASSES
    dom = dominant_class(tim)
    di = cls.index(dom)
    dom_ms = tim[dom][0]
    flops_cls = list(st_t["flops_class"]) + [0.0]
    if dom == "stage_loop":
        # the loop runs the precision updates and complement tests of most stages:
        # the step's flops of both classes (the few outside it included)
        dom_flops = flops_cls[2] + flops_cls[4]
    else:
        dom_flops = flops_cls[di] if di > 0 else 2.0 * n * p * (p + 1)
    fp64_classes = {"stage_a", "prec", "ci_complement", "stage_loop"}
    if dom in fp64_classes or (dom == "ci_direct" and mixed_prec == 0):
        peak = FP64_PEAK_TFLOPS
    else:
        peak = FP32_PEAK_TFLOPS
    achieved = dom_flops / (dom_ms * 1e-3) / 1e12 if dom_ms > 0 else 0.0
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": DRAM_BYTES_PER_LAUNCH.get((w["name"], dom)),
                "kernel": dom, "kernels": CLASS_KERNELS.get(dom, dom),
                "work": "algorithmic flops F(l) = l^3/3 + 2l^2 + 6l + 10 per executed test (direct), "
                        "k^3/3 + 2k^2 + 6k + 20 (complement)" if dom in ("ci_direct", "ci_complement") else
                        ("precision-block flops (|R|^3/3 + 2|T||R|(|R|+|T|) per downdate, m^3 per build) + "
                         "complement-test flops of the step" if dom == "stage_loop" else
                         "algorithmic flops counted by the kernels"),
                "kernel_ms_per_step": dom_ms, "launch_groups": tim[dom][1],
                "peak_source": "nominal FP64 1.25 TFLOP/s" if peak == FP64_PEAK_TFLOPS else
                "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                "class_ms": {c: tim[c][0] for c in cls},
                "largest_class": max(cls, key=lambda c: tim[c][0])}

    # the correlation step against the tensor roofline: useful flops n p (p+1) of the
    # symmetric product (the BF16x3 split issues three products per useful one); the
    # GEMM kernels alone (class corr_gemm) and the whole pc_corr (statistics,
    # standardisation, GEMM, reduce)
    roofline_gemm = roofline_corr = None
    bf16, hbm, src = measured_peaks()
    gemm_flops = n * p * (p + 1)
    if tim["corr_gemm"][0] > 0:
        ach = gemm_flops / (tim["corr_gemm"][0] * 1e-3) / 1e12
        roofline_gemm = {"bound": "tensor", "kernel": "corr_bf16x3_kernel (tcgen05, TMA) + corr_tc_reduce_kernel"
                         if mixed_prec == 2 else "Gram kernel (CUDA cores)",
                         "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
                         "issued_tflops": 3 * ach if mixed_prec == 2 else ach,
                         "useful_flops_per_launch": gemm_flops, "ms_per_step": tim["corr_gemm"][0],
                         "launch_groups": tim["corr_gemm"][1],
                         "peak_source": f"bf16 dense burst, {src}"}
    if tim["corr"][0] > 0:
        ach = gemm_flops / (tim["corr"][0] * 1e-3) / 1e12
        roofline_corr = {"bound": "tensor", "kernel": "pc_corr (column statistics, standardisation, "
                         "BF16x3 tcgen05 GEMM, Kahan FP32 split-K reduce)" if mixed_prec == 2 else "pc_corr",
                         "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
                         "issued_tflops": 3 * ach if mixed_prec == 2 else ach, "ms_per_step": tim["corr"][0],
                         "peak_source": f"bf16 dense burst, {src}"}

    # Phase II of Algorithm 1 (pc_orient) on this skeleton: outside the metric's step,
    # timed on its own (host wall time; pc_orient synchronises once per rule round)
    codes = np.empty((p, p), dtype=np.int8)
    fp.pc_orient(pc.h, p, codes)
    o_t = []
    for _ in range(5):
        t0 = time.perf_counter()
        _, o_rounds = fp.pc_orient(pc.h, p, codes)
        o_t.append(time.perf_counter() - t0)
    orient = {"ms": 1e3 * float(np.median(o_t)), "rule_rounds": o_rounds,
              "directed": int((codes == 2).sum()), "undirected": int((codes == 1).sum() // 2),
              "bidirected": int((codes == 4).sum() // 2)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        ref, _ = oracle.orient(adj_ours, fp.pc_sepsets(pc.h, p))
        orient["matches_oracle_phase2"] = bool(np.array_equal(codes, ref))

    # plain GPU form: FP32 SIMT GEMM, FP32 tests one warp per test (no rank-major
    # small-stage kernel, no complement path), one host-driven launch sequence per
    # stage (no graph), lexicographic order
    plain = None
    if not args.no_plain:
        pcp = make(1 if w["cfg"] != 1 else 0, 0, graph=0)
        fp.pc_set_opt(pcp.h, "small_stage_kernel", 0)
        step(pcp)
        pms, stp = timed_steps(pcp, max(3, min(args.steps, 5)))
        plain = {"ms_per_step": pms, "value": stp["tests_canonical"] / (pms / 1000.0),
                 "skeleton_ms": stp["t_skeleton_ms"],
                 "identical_skeleton": bool(np.array_equal(adj_d.cpu().numpy(), adj_ours))}
        pcp.close()

    # end to end through the C-ABI with host buffers (H2D of X, D2H of the adjacency)
    adj_h = np.empty((p, p), dtype=np.uint8)
    Xh = np.ascontiguousarray(X)
    fp.pc_set_stream(pc.h, None)
    pc.corr(Xh)
    pc.skeleton(adj_h)
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(max(3, min(args.steps, 5))):
        t0 = time.perf_counter()
        pc.corr(Xh)
        pc.skeleton(adj_h)
        e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": tests_unit / float(np.mean(e2e_t)), "unit": UNIT,
           "h2d_bytes_per_step": int(Xh.nbytes), "d2h_bytes_per_step": int(adj_h.nbytes)}

    cpu = None
    matches = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, R = cpu_baseline(X, w)
        matches = bool(np.array_equal(R["adj"], adj_ours)) and R["tests_total"] == tests_unit

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if mixed_prec == 0 else "f32+f64",
                "data": "synthetic",
                "config": {"workload": w["name"], "p": p, "n": n, "alpha": w["alpha"],
                           "max_level": w["max_level"],
                           "order": "reversed" if w["order"] else "conventional",
                           "precision": {0: "fp64", 1: "fp32", 2: "bf16x3-gemm+fp32-tests"}[mixed_prec],
                           "tensor_core_gemm": bool(fp.pc_get_opt(pc.h, "tensor_core_gemm")),
                           "learned_order": learned is not None,
                           "parallelism": f"replicas x{world}",
                           "l2": "flushed before every step (512 MB write)",
                           "options": list(args.opt)},
                "tests_canonical_per_step": tests_unit,
                "tests_executed_per_step": stats[-1]["tests_executed"],
                "skeleton_ms": float(np.mean([x["t_skeleton_ms"] for x in stats])),
                "levels_run": stats[-1]["levels_run"],
                "redecided": stats[-1]["tests_redecided"],
                "complement_tests": stats[-1]["complement_tests"],
                "roofline": roofline,
                "roofline_gemm": roofline_gemm,
                "roofline_corr": roofline_corr,
                "autotune": tune,
                "cpu_baseline": cpu,
                "skeleton_matches_oracle": matches,
                "lexicographic": {"ms_per_step": lex_ms, "tests_canonical": lex_st["tests_canonical"],
                                  "tests_executed": lex_st["tests_executed"]},
                "learned": learned,
                "plain_gpu": plain,
                "orient": orient,
                "e2e": e2e,
                "gpu_launches": int(launches),
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    pc.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


MANY = {"name": "many64", "count": 64, "alpha": 0.01, "max_level": -1, "order": 0, "streams": 16}


def run_many(args):
    """64 independent problems in one batched handle (pc_create_batch: block-diagonal
    layout, every stage one launch sequence over all instances' tests), mixed
    precision, the proposal order behind the autotuned scoring gate -- the timed
    configuration; beside it the same problems as 64 handles searched concurrently
    on 16 streams (pc_skeleton_many)."""
    import torch
    from paper_2109_04626_gb300 import fastpc as fp, proposal, sem
    rank, world, local = dist_setup(args)
    fp.load()
    inst = sem.make_many(MANY["count"])
    ns = [s_.X.shape[0] for s_ in inst]
    ps = [s_.X.shape[1] for s_ in inst]
    dev = torch.device("cuda", torch.cuda.current_device())
    Xd = [torch.from_numpy(s_.X).to(dev) for s_ in inst]
    main_s = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn, k):
        ms, out = [], None
        for _ in range(k):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main_s)
            out = fn()
            b.record(main_s)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return ms, out

    # the batched handle: every instance's correlation block (concurrently), then one search
    pb = fp.PCBatch(ns, ps, MANY["alpha"], MANY["max_level"], precision=2)
    for kv in args.opt:
        key, val = kv.split("=", 1)
        fp.pc_set_opt(pb.h, key.strip(), float(val))
    fp.pc_set_stream(pb.h, main_s)
    adj_b = torch.empty((pb.p, pb.p), dtype=torch.uint8, device=dev)

    def step_b(Xs=Xd, adj=adj_b):
        pb.corr_blocks(Xs)                  # the instances' correlation steps on the handle's side streams
        _, st = pb.skeleton(adj)
        return st

    # lexicographic order first: its canonical count is the oracle's, the unit of the metric
    st_lex = step_b()
    tests_unit = st_lex["tests_canonical"]
    adjs_lex = pb.split(adj_b.cpu().numpy())
    learned = None
    if not args.no_learned:
        t0 = time.perf_counter()
        train = sem.make_many(24, base_seed=9000)          # other seeds of the same recipe
        feats, labels = proposal.collect(lambda i: train[i].X, range(len(train)), MANY["alpha"], 0,
                                         MANY["max_level"], 2, max_rows_per_seed=50_000)
        loss = proposal.train(pb.h, feats, labels, epochs=4, batch=8192, lr=2e-3, seed=2)
        fp.pc_set_opt(pb.h, "learned", 1)
        learned = {"train_rows": int(labels.shape[0]), "train_sems": "24 instances of the recipe (other seeds)",
                   "final_loss": loss, "train_s": time.perf_counter() - t0}
    for _ in range(args.warmup):
        step_b()
    torch.cuda.synchronize()
    tune = fp.pc_autotune(pb.h, 2) if not args.no_autotune else None
    for _ in range(args.warmup):
        step_b()
    torch.cuda.synchronize()
    barrier(world)
    l0 = fp.pc_kernel_launches()
    with ClockSampler(local if world > 1 else torch.cuda.current_device()) as clk:
        torch.cuda.nvtx.range_push("bench_timed")
        ms, st_b = timed(step_b, args.steps)
        torch.cuda.nvtx.range_pop()
    launches = fp.pc_kernel_launches() - l0
    barrier(world)
    t_max = max_over_ranks(sum(ms) / 1000.0, world)
    value = sum_over_ranks(float(tests_unit * args.steps), world) / t_max
    blocks = pb.split(adj_b.cpu().numpy())
    identical = all(np.array_equal(blocks[i], adjs_lex[i]) for i in range(len(inst)))
    if learned is not None:
        learned.update({"tests_canonical": st_b["tests_canonical"], "tests_executed": st_b["tests_executed"],
                        "max_level": int(fp.pc_get_opt(pb.h, "learned_max_level")),
                        "identical_skeletons": identical})

    # per-kernel-class device time of the batched search (roofline of its dominant class)
    fp.pc_set_opt(pb.h, "timing", 1)
    fp.pc_timing(pb.h, reset=True)
    st_t = step_b()
    tim = fp.pc_timing(pb.h, reset=True)
    fp.pc_set_opt(pb.h, "timing", 0)
    cls = fp.TIMING_CLASSES
    dom = dominant_class(tim)
    di = cls.index(dom)
    flops_cls = list(st_t["flops_class"]) + [0.0]
    dom_flops = flops_cls[di] if di > 0 else sum(2.0 * n_ * p_ * (p_ + 1) for n_, p_ in zip(ns, ps))
    peak = FP64_PEAK_TFLOPS if dom in ("stage_a", "prec", "ci_complement") else FP32_PEAK_TFLOPS
    achieved = dom_flops / (tim[dom][0] * 1e-3) / 1e12 if tim[dom][0] > 0 else 0.0
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": dom, "kernels": CLASS_KERNELS.get(dom, dom),
                "measured_on": "batched handle, timing step",
                "peak_source": "nominal FP64 1.25 TFLOP/s" if peak == FP64_PEAK_TFLOPS else
                "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz", "class_ms": {c: tim[c][0] for c in cls},
                "launch_groups": tim[dom][1], "largest_class": max(cls, key=lambda c: tim[c][0])}

    # end to end with host buffers: every instance's X from pinned host memory, the
    # block-diagonal skeleton back to the host
    Xh = [torch.from_numpy(s_.X).pin_memory() for s_ in inst]
    adj_h = np.empty((pb.p, pb.p), dtype=np.uint8)
    e2e_ms, _ = timed(lambda: step_b(Xh, adj_h), max(2, min(args.steps, 3)))
    e2e = {"value": tests_unit / (np.mean(e2e_ms) / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(sum(s_.X.nbytes for s_ in inst)), "d2h_bytes_per_step": int(adj_h.nbytes)}
    pb.close()

    # the same problems as 64 handles on 16 streams, searched concurrently
    streams = [torch.cuda.Stream() for _ in range(MANY["streams"])]
    pcs = []
    for i in range(len(inst)):
        pc = fp.PC(ns[i], ps[i], MANY["alpha"], MANY["max_level"], order=0, precision=2)
        fp.pc_set_stream(pc.h, streams[i % len(streams)])
        pcs.append(pc)
    hs = [pc.h for pc in pcs]

    def step_s():
        ev = torch.cuda.Event()
        ev.record(main_s)
        for st in streams:
            st.wait_event(ev)
        for i, pc in enumerate(pcs):
            pc.corr(Xd[i])
        _, stats, status = fp.pc_skeleton_many(hs, ps, adj_out=False)
        if any(status):
            raise RuntimeError(f"pc_skeleton_many: statuses {status}")
        for st in streams:
            e2 = torch.cuda.Event()
            e2.record(st)
            main_s.wait_event(e2)
        return stats
    step_s()
    ms_s, stats_s = timed(step_s, max(2, min(args.steps, 5)))
    streams_obj = {"ms_per_step": float(np.mean(ms_s)), "value": tests_unit / (np.mean(ms_s) / 1e3),
                   "streams": MANY["streams"], "tests_executed": int(sum(x["tests_executed"] for x in stats_s))}
    for pc in pcs:
        pc.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        t_tot, n_tests, k = 0.0, 0, 0
        for s_ in inst:
            dt, R = oracle_run(s_.X, {"alpha": MANY["alpha"], "max_level": -1, "order": 0})
            t_tot += dt
            n_tests += R["tests_total"]
            k += 1
            if t_tot > 20.0:
                break
        cpu = {"value": n_tests / t_tot, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"the first {k} of the 64 instances (Pearson + skeleton), {t_tot:.1f} s"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": float(np.mean(ms)), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": "many64", "instances": len(inst), "p_total": int(sum(ps)),
                           "alpha": MANY["alpha"], "order": "conventional",
                           "precision": "bf16x3-gemm+fp32-tests",
                           "form": "one batched handle (block-diagonal, one launch sequence per stage)",
                           "learned_order": learned is not None, "options": list(args.opt),
                           "parallelism": f"replicas x{world}", "l2": "flushed before every step (512 MB write)"},
                "tests_canonical_per_step": tests_unit,
                "tests_executed_per_step": st_b["tests_executed"],
                "skeleton_ms": float(st_b["t_skeleton_ms"]),
                "roofline": roofline, "autotune": tune, "learned": learned,
                "lexicographic": {"tests_canonical": st_lex["tests_canonical"],
                                  "tests_executed": st_lex["tests_executed"]},
                "streams_16": streams_obj, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


SWEEP = {"sizes": list(range(15, 101, 5)), "n": 5000, "alpha": 1e-3, "oracle_instances": 5}
# Sec. 6.2: CI tests for the 95-node graphs (PC, PC-reverse, PC-reverse-parallel)
PAPER_TESTS_P95 = {"pc": 90394, "pc_reverse": 8678, "pc_reverse_parallel": 4563}


def dag_scores(codes, dag):
    """Skeleton TPR / FPR against the true DAG's skeleton, and the structural Hamming
    distance of the oriented graph to the DAG (Sec. 6.3: one count per pair whose state
    -- no edge, a -> b, b -> a -- differs; an undirected or bidirected edge differs from
    any directed one)."""
    p = dag.shape[0]
    iu = np.triu_indices(p, 1)
    est = codes[iu]
    t_ab, t_ba = dag[iu] == 1, dag.T[iu] == 1
    true_edge = t_ab | t_ba
    found = est != 0
    tpr = float((found & true_edge).sum() / max(1, true_edge.sum()))
    fpr = float((found & ~true_edge).sum() / max(1, (~true_edge).sum()))
    same = (~found & ~true_edge) | ((est == 2) & t_ab) | ((est == 3) & t_ba)
    return tpr, fpr, int((~same).sum())


def run_sweep(args):
    """The paper's simulation (Sec. 6.1-6.3): for p = 15, 20, ..., 100, args.sweep_mc
    graphs each (mean degree 5, two hubs of 10 neighbours, weights +-U[0.2,0.8],
    alpha = 1e-3): CI tests per graph, skeleton time, and the accuracy of the oriented
    graph (skeleton TPR / FPR, SHD to the DAG) of the conventional (Algorithm 1) and
    reversed (Algorithm 2) orders on the GPU.  The oracle, timed as the CPU baseline,
    recounts the first graphs of every size."""
    import torch
    from paper_2109_04626_gb300 import fastpc as fp, sem
    rank, world, local = dist_setup(args)
    fp.load()
    check = rank == 0 and world == 1 and not args.no_cpu_baseline
    if check:
        import oracle
    n, alpha = SWEEP["n"], SWEEP["alpha"]
    rows = []
    cpu_t, cpu_tests = 0.0, 0
    with ClockSampler(local if world > 1 else torch.cuda.current_device()) as clk:
        for p in SWEEP["sizes"]:
            pcs = {o: fp.PC(n, p, alpha, -1, order=o) for o in (0, 1)}
            acc = {o: np.zeros(6) for o in (0, 1)}   # tests, executed, skeleton ms, TPR, FPR, SHD
            equal = True
            codes = np.empty((p, p), dtype=np.int8)
            for m in range(args.sweep_mc):
                s = sem.make_sweep(p, m, n=n)
                Xd = torch.from_numpy(s.X).cuda()
                counts = {}
                for o, pc in pcs.items():
                    pc.corr(Xd)
                    pc.skeleton()                        # the first search of a handle builds its graph
                    _, st = pc.skeleton()
                    fp.pc_orient(pc.h, p, codes)
                    counts[o] = st["tests_canonical"]
                    acc[o] += (st["tests_canonical"], st["tests_executed"], st["t_skeleton_ms"],
                               *dag_scores(codes, s.dag))
                if check and m < SWEEP["oracle_instances"]:
                    t0 = time.perf_counter()
                    C = oracle.pearson(s.X.astype(np.float64))
                    for o in (0, 1):
                        R = oracle.skeleton(C, n, alpha, -1, reversed_order=bool(o))
                        equal &= R["tests_total"] == counts[o]
                        cpu_tests += R["tests_total"]
                    cpu_t += time.perf_counter() - t0
            for pc in pcs.values():
                pc.close()
            mc = float(args.sweep_mc)
            res = {}
            for o, name in ((0, "conventional"), (1, "reversed")):
                a_ = acc[o] / mc
                res[name] = {"tests": a_[0], "executed": a_[1], "skeleton_ms": a_[2], "tpr": a_[3], "fpr": a_[4],
                             "shd": a_[5]}
            conv, rev = res["conventional"], res["reversed"]
            rows.append({"p": p, "conventional": conv, "reversed": rev,
                         "tests_ratio": conv["tests"] / rev["tests"] if rev["tests"] else None,
                         "time_ratio": conv["skeleton_ms"] / rev["skeleton_ms"] if rev["skeleton_ms"] else None,
                         "oracle_counts_equal": bool(equal) if check else None})
    if rank == 0:
        r95 = next(r for r in rows if r["p"] == 95)
        cpu = None
        if check and cpu_t > 0:
            cpu = {"value": cpu_tests / cpu_t, "unit": "CI tests/s", "cores": oracle.num_threads(), "kind": "oracle",
                   "sample": f"Pearson + skeleton, both orders, first {SWEEP['oracle_instances']} graphs per size "
                             f"({cpu_t:.1f} s)"}
        line = {"metric": "CI tests per graph: conventional / reversed order (the paper's simulation, Sec. 6.2)",
                "value": r95["tests_ratio"], "unit": "ratio", "higher_is_better": True, "n_gpus": world,
                "data": "synthetic",
                "config": {"workload": "paper_sweep", "sizes": SWEEP["sizes"], "graphs_per_size": args.sweep_mc,
                           "n": n, "alpha": alpha, "generator": "mean degree 5, two hubs of 10, +-U[0.2,0.8]"},
                "sweep": rows, "paper_p95_tests": PAPER_TESTS_P95, "cpu_baseline": cpu, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    return 0


POWER = {"n": 100000, "alpha": 1e-3, "oracle_datasets": 5,
         "tests": [("X5-X6 | {0}", 5, 6, [0]), ("X5-X6 | {0,1,2,3,4,7,8}", 5, 6, [0, 1, 2, 3, 4, 7, 8]),
                   ("X8-X9 | {0}", 8, 9, [0]), ("X8-X9 | {0,...,7}", 8, 9, list(range(8)))]}


def run_power(args):
    """The power experiment (Sec. 6.4) on the substitute 10-node graph: datasets of
    N = 100000 samples, alpha = 1e-3.  Per dataset the GPU computes the four partial
    correlations of the text (pc_ci_batch) and both orders' skeletons; reported: the
    Fisher statistic |F_Z(r)| = |atanh r| of each test against its threshold
    Phi^{-1}(1 - alpha/2) / sqrt(N - |S| - 3), the stage at which X5 - X6 is removed
    and how often X8 - X9 is kept.  The oracle recomputes the first datasets."""
    import torch
    from paper_2109_04626_gb300 import fastpc as fp, sem
    rank, world, local = dist_setup(args)
    fp.load()
    check = rank == 0 and world == 1 and not args.no_cpu_baseline
    if check:
        import oracle
    n, alpha, D = POWER["n"], POWER["alpha"], args.power_datasets
    q = fp.pc_fisher_threshold(alpha)
    stat = {name: [] for name, *_ in POWER["tests"]}
    stage56 = {0: {}, 1: {}}
    kept89 = {0: 0, 1: 0}
    dr, cpu_t, cpu_tests = 0.0, 0.0, 0
    pcs = {o: fp.PC(n, 10, alpha, -1, order=o) for o in (0, 1)}
    with ClockSampler(local if world > 1 else torch.cuda.current_device()) as clk:
        for m in range(D):
            s = sem.make_power(m, n=n)
            Xd = torch.from_numpy(s.X).cuda()
            for o, pc in pcs.items():
                pc.corr(Xd)
                if o == 0:
                    for name, a, b, S in POWER["tests"]:
                        ij = torch.tensor([[a, b]], dtype=torch.int32, device="cuda")
                        Sd = torch.tensor([S], dtype=torch.int32, device="cuda")
                        r, _, _ = fp.pc_ci_batch(pc.h, ij, Sd, len(S))
                        rv = float(r.item())
                        stat[name].append(abs(float(np.arctanh(rv))))
                        if check and m < POWER["oracle_datasets"]:
                            C = oracle.pearson(s.X.astype(np.float64))
                            dr = max(dr, abs(rv - oracle.partial_corr(C, a, b, S)[0]))
                adj, st = pc.skeleton()
                seps = pc.sepsets()
                lv = seps[(5, 6)][0] if (5, 6) in seps else -1
                stage56[o][lv] = stage56[o].get(lv, 0) + 1
                kept89[o] += int(adj[8, 9])
            if check and m < POWER["oracle_datasets"]:
                t0 = time.perf_counter()
                C = oracle.pearson(s.X.astype(np.float64))
                for o in (0, 1):
                    cpu_tests += oracle.skeleton(C, n, alpha, -1, reversed_order=bool(o))["tests_total"]
                cpu_t += time.perf_counter() - t0
    for pc in pcs.values():
        pc.close()
    if rank == 0:
        tests = []
        for name, a, b, S in POWER["tests"]:
            v = np.array(stat[name])
            thr = q / np.sqrt(n - len(S) - 3)
            tests.append({"test": name, "threshold": thr, "mean": float(v.mean()), "min": float(v.min()),
                          "max": float(v.max()), "below_threshold": float((v <= thr).mean())})
        removed = {o: sum(c for lv, c in stage56[o].items() if lv >= 0) / D for o in (0, 1)}
        value = min(removed[0], removed[1], kept89[0] / D, kept89[1] / D)
        cpu = None
        if check and cpu_t > 0:
            cpu = {"value": cpu_tests / cpu_t, "unit": "CI tests/s", "cores": oracle.num_threads(), "kind": "oracle",
                   "sample": f"Pearson + skeleton, both orders, first {POWER['oracle_datasets']} datasets "
                             f"({cpu_t:.1f} s)"}
        line = {"metric": "fraction of datasets with X5 - X6 removed and X8 - X9 kept, both orders "
                          "(the power experiment, Sec. 6.4, substitute graph)",
                "value": value, "unit": "fraction", "higher_is_better": True, "n_gpus": world, "data": "synthetic",
                "config": {"workload": "power", "datasets": D, "n": n, "alpha": alpha,
                           "graph": "substitute: X0 -> X5, X6; X0 -> X1 -> X2 -> X3 -> X4 -> X7 -> X8 -> X9; X0 -> X8"},
                "tests": tests,
                "x5_x6_removed_at_stage": {"conventional": {str(k): v for k, v in sorted(stage56[0].items())},
                                           "reversed": {str(k): v for k, v in sorted(stage56[1].items())}},
                "x8_x9_kept": {"conventional": kept89[0] / D, "reversed": kept89[1] / D},
                "max_abs_r_vs_oracle": dr if check else None, "cpu_baseline": cpu, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "many64":
        return run_many(args)
    if args.workload == "paper_sweep":
        return run_sweep(args)
    if args.workload == "power":
        return run_power(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
