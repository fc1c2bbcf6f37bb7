#!/usr/bin/env python
"""OFM iterations/s of the GB300 path on a seeded degree-corrected SBM (2,000,000 nodes, k = 128).

One step = one ofsc_iterate call of 30 updates of Algorithm 2 from the same X0, with the graph and
X0 resident in HBM. By default the gathered block D^-1/2 V is stored in BF16 with the FP32 master
copy and FP32 accumulation (the configured mixed-precision form); the plain FP32 path is timed on
the same steps and reported as `plain_fp32`. `value` is updates per second over all ranks. `e2e`
times the same steps through the public API from pinned host buffers (X0 copied in, X copied out
every step; the copies of neighbouring steps overlap the current step's iterations on a copy
stream, and the serial form is reported beside it). The dominant kernel's roofline comes from CUDA-event phase timings taken inside the
timed steps. `--impl reference` times the FP64 CPU oracle on the same workload instead.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference] [--gather bf16|fp32]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METHODS = {"ofm_f1": 0, "tri_f1": 1, "ofm_f2": 2, "tri_f2": 3}
METHOD_LABEL = {"ofm_f1": "OFM-f1", "tri_f1": "TriOFM-f1", "ofm_f2": "OFM-f2", "tri_f2": "TriOFM-f2"}
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal
FP32_LANES_PER_SM = 128
NUM_SMS = 152
SM_MAX_MHZ = 2070.0


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": d["hbm_gbs"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


DIR_PRODUCT_SOURCES = ("spmm_dir.cu", "spmm_dir.cuh", "spmm_dir_body.inc")  # the direction product, its body and header


def source_digest(names=None) -> str:
    """Digest of the CUDA sources (all of them, or the named files of csrc/)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2305_10356_gb300", "csrc")
    for name in sorted(names if names is not None else os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    if names is None:
        with open(os.path.join(ROOT, "include", "ofsc.h"), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, device_id: str):
        self.device_id = device_id
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.device_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="dcsbm_n2m_k128")
    ap.add_argument("--method", default="ofm_f1", choices=list(METHODS))
    ap.add_argument("--gather", default="bf16", choices=["fp32", "bf16"],
                    help="storage of the gathered block D^-1/2 V (bf16: FP32 master copy, FP32 accumulation)")
    ap.add_argument("--no-fp32-compare", action="store_true",
                    help="skip timing the plain FP32 path next to the BF16-gather one")
    ap.add_argument("--no-time-to-tol", action="store_true",
                    help="skip the time to a 1e-4 rad subspace angle against the FP32 reference")
    ap.add_argument("--iters", type=int, default=30, help="updates of Algorithm 2 per step")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the 1,000-node all-methods leg and the batched-vs-loop leg")
    ap.add_argument("--spmm-engine", default="auto", choices=["auto", "simt", "tma"])
    ap.add_argument("--nodes", type=int, default=None, help="shrink the workload (testing only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--unrolled", type=int, default=0,
                    help="time d f1(X_T)/d(X_0, w) through this many unrolled OFM-f1 updates instead")
    ap.add_argument("--ckpt", type=int, default=5, help="checkpoint interval of --unrolled")
    return ap.parse_args()


def dist_setup(backend: str):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
    return world, rank, local


def max_over_ranks(x: float, world: int) -> float:
    """The largest of every rank's x (the job's time is its slowest rank's); x itself for one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


L2_BYTES = 129 * 2**20  # GB300's L2 (126.5 MiB reported), rounded up


def l2_flushed(args) -> bool:
    """Whether the steps flush the L2: unless every N x kp block and the CSR (stored entries about
    N times the mean degree) are each more than twice the L2."""
    from paper_2305_10356_gb300 import synth
    spec = synth.WORKLOADS[args.workload]
    n = args.nodes or spec["n"]
    kp = ((spec["n_blocks"] + 7) // 8) * 8
    csr = 8 * (n + 1) + 4 * n * spec["mean_degree"]
    return min(4 * n * kp, csr) <= 2 * L2_BYTES


def workload_config(args) -> dict:
    from paper_2305_10356_gb300 import synth
    spec = synth.WORKLOADS[args.workload]
    n = args.nodes or spec["n"]
    kind = "degree-corrected SBM" if spec.get("gamma") else "SBM"
    l2 = (f"L2 flushed at the start of every step by a {2 * L2_BYTES >> 20} MB write inside the timed region "
          "(the inputs are smaller than the L2)" if l2_flushed(args) else
          "inputs larger than L2 (X, state and CSR are each > 129 MB)")
    return {"workload": f"{args.workload}: {kind}, N={n}, k={spec['n_blocks']}, mean degree "
                        f"{spec['mean_degree']:g}, power-law {spec.get('gamma')}, within:between "
                        f"{spec['ratio']:g}:1 ({spec['ratio_kind']}), int32 CSR, seeded synthetic",
            "n": n, "k": spec["n_blocks"], "method": METHOD_LABEL[args.method],
            "gather": args.gather, "updates_per_step": args.iters, "l2": l2}


SAMPLE_FRACTION = 5  # the CPU oracle runs on a graph of N / 5 nodes drawn with the same recipe


def cpu_oracle_step(og, method, x0):
    """One oracle update (maxit=1); returns seconds."""
    from oracle import ofsc_oracle as o
    t0 = time.perf_counter()
    o.iterate(og, method, x0, 0.0, 1)
    return time.perf_counter() - t0


def oracle_sample(args):
    """The bounded CPU sample: the same workload recipe at N / SAMPLE_FRACTION nodes."""
    from oracle import ofsc_oracle as o
    from paper_2305_10356_gb300 import synth
    n_full = args.nodes or synth.WORKLOADS[args.workload]["n"]
    n_s = max(1000, n_full // SAMPLE_FRACTION)
    e, x0 = synth.workload(args.workload, n=n_s)
    return o.build_graph(e.n, e.src, e.dst, e.w), x0, n_s, n_full


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


ONE_THREAD_FRACTION = SAMPLE_FRACTION  # the single-thread sample: the same N / 5 graph as the all-core one


def oracle_one_thread_seconds(args) -> float | None:
    """Seconds of one oracle update on one thread (BLAS limited to one thread in a child
    process), on N / ONE_THREAD_FRACTION nodes of the same recipe, scaled to the full N."""
    from paper_2305_10356_gb300 import synth
    n_full = args.nodes or synth.WORKLOADS[args.workload]["n"]
    n_s = max(1000, n_full // ONE_THREAD_FRACTION)
    code = ("import sys, time; sys.path.insert(0, %r)\n"
            "from oracle import ofsc_oracle as o\nfrom paper_2305_10356_gb300 import synth\n"
            "e, x0 = synth.workload(%r, n=%d)\ng = o.build_graph(e.n, e.src, e.dst, e.w)\n"
            "t0 = time.perf_counter(); o.iterate(g, %d, x0, 0.0, 1); print(time.perf_counter() - t0)\n"
            % (ROOT, args.workload, n_s, METHODS[args.method]))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300, env=env)
        return float(r.stdout.strip().splitlines()[-1]) * n_full / n_s
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return None


SAMPLE_TEXT = ("one update of Algorithm 2 (maxit=1) by the FP64 numpy/scipy oracle on a graph of "
               "N/5 nodes drawn with the same recipe, scaled to the full N (the oracle's cost is "
               "linear in N and nnz); BLAS on all cores, sparse product single-threaded")


def run_reference(args):
    world, rank, _ = dist_setup("gloo")
    if rank != 0:
        return 0
    og, x0, n_s, n_full = oracle_sample(args)
    method = METHODS[args.method]
    for _ in range(args.warmup):
        cpu_oracle_step(og, method, x0)
    times = [cpu_oracle_step(og, method, x0) for _ in range(args.steps)]
    total = sum(times) * n_full / n_s  # the full workload's time, scaled from the sample
    value = args.steps / total
    cores = os.cpu_count()
    cfg = workload_config(args)
    # ms_per_step is the measured time of a step (one update on the N/5 sample), so that steps x
    # ms_per_step is the run's real duration; value is the full workload's rate scaled from it
    line = {"metric": "OFM iterations/s", "value": value, "unit": "iterations/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sum(times) / args.steps,
            "sample_nodes": n_s, "full_nodes": n_full,
            "ms_per_full_update_scaled": 1000.0 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "iterations/s", "cores": cores, "kind": "oracle",
                             "sample": SAMPLE_TEXT},
            "e2e": {"value": value, "unit": "iterations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def spmm_bytes(n: int, kp: int, nnz: int, gather_bytes: int, weighted: bool, h: float) -> dict:
    """Algorithmic HBM bytes of one direction product W = A V (the cost model of the one-product
    design): CSR (int64 row pointers, int32 columns, FP32 weights), the gathered rows of
    D^-1/2 V that miss L2 (nnz k b_g (1 - h)), the epilogue read of V and D^-1/2, the write of W."""
    csr = 8 * (n + 1) + 4 * nnz + (4 * nnz if weighted else 0)
    gather_all = nnz * kp * gather_bytes
    return {"csr": csr, "gather": int(gather_all * (1.0 - h)), "gather_all": gather_all,
            "epilogue": 4 * n * kp + 4 * n, "write": 4 * n * kp,
            "total": int(csr + gather_all * (1.0 - h) + 4 * n * kp + 4 * n + 4 * n * kp)}


def measured_traffic(workload: str, gather: str, any_build: bool = False) -> dict | None:
    """ncu DRAM counters at this workload (profiles/traffic.json): of the direction product (keyed
    to the digest of its own sources) or, for gather "update", of all kernels of one update (keyed
    to the digest of every source); None when those sources changed since (any_build: the entry
    whatever build it was taken on)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        tj = json.load(fh)
    entry = tj.get("entries", {}).get(f"{workload}/{gather}")
    digest = source_digest() if gather == "update" else source_digest(DIR_PRODUCT_SOURCES)
    if not entry or (entry.get("source_digest") != digest and not any_build):
        return None
    return entry


TTT_TOL = 1e-4          # rad
TTT_REF_UPDATES = 400   # the FP32 reference run (its relative gradient reaches the FP32 floor)


TTT_REFINE_TOL = 1e-2   # the refined BF16 form switches to FP32 gathers below this relative gradient
TTT_SEEDS = 3           # starting blocks: updates-to-tolerance of Algorithm 2 vary widely with tiny
                        # perturbations (chaotic CG), so forms are compared by their median


def time_to_tol(g, method, n, k, stream, seed0: int) -> dict:
    """Updates and seconds until X is within TTT_TOL rad of an FP32 reference subspace (400 plain FP32
    updates from the same start), for the BF16-gather form, the BF16 form with the FP32 refinement
    sweep (FP32 gathers once the relative direction norm read at a host check is <= TTT_REFINE_TOL),
    the plain FP32 path, and the BF16 and FP32 forms with the optional CG restart. Per start: the
    smallest multiple of 10 updates (fresh calls from X0) that gets there, then that call timed with
    CUDA events (fixed per-call costs included). Reported per start and as medians over TTT_SEEDS
    seeded starts X0 ~ N(0, 1/N)."""
    import statistics

    import torch
    from paper_2305_10356_gb300 import ofsc, synth

    def sin_angle(A, B):
        qa, _ = torch.linalg.qr(A.double())
        qb, _ = torch.linalg.qr(B.double())
        sv = torch.linalg.svdvals(qa.T @ qb)
        return float(torch.sqrt(torch.clamp(1.0 - sv.min() ** 2, min=0.0)))

    forms = (("bf16_gather", dict(gather=ofsc.GATHER_BF16)),
             ("bf16_refined", dict(gather=ofsc.GATHER_BF16, refine_tol=TTT_REFINE_TOL)),
             ("fp32", dict(gather=ofsc.GATHER_FP32)),
             ("bf16_gather_restart", dict(gather=ofsc.GATHER_BF16, cg_restart=True)),
             ("fp32_restart", dict(gather=ofsc.GATHER_FP32, cg_restart=True)))
    out = {"tol_rad": TTT_TOL, "reference": f"plain FP32, {TTT_REF_UPDATES} updates from the same X0",
           "starts": TTT_SEEDS, "refine_tol": TTT_REFINE_TOL, "runs": {name: [] for name, _ in forms}}
    for si in range(TTT_SEEDS):
        X0 = torch.from_numpy(synth.initial_block(n, k, seed0 + si)).cuda()
        X = X0.clone()
        ofsc.ofsc_iterate(g, method, X, 0.0, TTT_REF_UPDATES, gather=ofsc.GATHER_FP32)
        ref = X.clone()
        for name, kw in forms:
            m, ang, r = 0, 1.0, None
            while ang > TTT_TOL and m < TTT_REF_UPDATES:
                m += 10
                X.copy_(X0)
                r = ofsc.ofsc_iterate(g, method, X, 0.0, m, **kw)
                ang = sin_angle(X, ref)
            X.copy_(X0)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            ofsc.ofsc_iterate(g, method, X, 0.0, m, **kw)
            t1.record(stream)
            torch.cuda.synchronize()
            out["runs"][name].append({"updates": m, "seconds": t0.elapsed_time(t1) / 1000.0, "sin_angle": ang,
                                      "rel_dir_norm": r.rel_dir_norm if r else None,
                                      "fp32_from_update": r.refined_at if (r and r.refined_at >= 0) else None})
        del ref, X, X0
    for name, _ in forms:
        runs = out["runs"][name]
        out[name] = {"median_updates": statistics.median(x["updates"] for x in runs),
                     "median_seconds": statistics.median(x["seconds"] for x in runs)}
    return out


C1_TOL, C1_MAXIT = 1e-6, 2000


def c1_leg(stream) -> dict:
    """The 1,000-node, 11-block SBM (the oracle-sized case): every method to tol 1e-6 (2,000 updates
    at most) from the seeded X0, in FP32 and with BF16 gathers; updates and device seconds per run
    (one warm-up run each, then the run timed with CUDA events)."""
    import torch
    from paper_2305_10356_gb300 import ofsc, synth
    e, x0 = synth.workload("sbm_n1000_k11")
    g = ofsc.ofsc_graph_build(e.n, torch.from_numpy(e.src).cuda(), torch.from_numpy(e.dst).cuda())
    X0 = torch.from_numpy(x0).cuda()
    X = torch.empty_like(X0)
    out = {"workload": "sbm_n1000_k11: SBM N=1000, k=11, mean degree 20, 10:1 edge probabilities",
           "tol": C1_TOL, "maxit": C1_MAXIT}
    for label, method in METHODS.items():
        row = {}
        for prec, gather in (("fp32", ofsc.GATHER_FP32), ("bf16", ofsc.GATHER_BF16)):
            X.copy_(X0)
            ofsc.ofsc_iterate(g, method, X, C1_TOL, C1_MAXIT, gather=gather)
            X.copy_(X0)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            r = ofsc.ofsc_iterate(g, method, X, C1_TOL, C1_MAXIT, gather=gather)
            t1.record(stream)
            torch.cuda.synchronize()
            secs = t0.elapsed_time(t1) / 1000.0
            row[prec] = {"updates": r.iterations, "converged": r.status == ofsc.OK, "rel_dir_norm": r.rel_dir_norm,
                         "seconds": secs, "updates_per_s": r.iterations / secs if secs > 0 else None}
        out[METHOD_LABEL[label]] = row
    g.free()
    return out


def batched_leg(stream, tol: float = 1e-4, iters: int = 300, steps: int = 2) -> dict:
    """The 32-graph batch (sbm_batch32, N from 3.5K to 99K, k from 8 to 64), every graph to
    tol (relative direction norm, at most `iters` updates): one ofsc_iterate_batched call (one
    launch per graph and kernel on the graphs' streams, replayed), the same call with grouped
    launches (one launch per kernel over the blocks of the graphs of each of 4 lanes), and a loop
    of one ofsc_iterate call per graph (all three run the same updates of every graph, bit for
    bit), timed with CUDA events over `steps` steps after one warm-up."""
    import torch
    from paper_2305_10356_gb300 import ofsc, synth
    probs = synth.batch("sbm_batch32", 1.0)
    graphs, X0s = [], []
    for e, x0 in probs:
        graphs.append(ofsc.ofsc_graph_build(e.n, torch.from_numpy(e.src).cuda(), torch.from_numpy(e.dst).cuda()))
        X0s.append(torch.from_numpy(x0).cuda())
    Xs = [torch.empty_like(x) for x in X0s]

    def batched(group=0):
        for X, X0 in zip(Xs, X0s):
            X.copy_(X0)
        return sum(r.iterations for r in ofsc.ofsc_iterate_batched(graphs, 0, Xs, tol, iters, group_launches=group))

    def loop():
        n = 0
        for g, X, X0 in zip(graphs, Xs, X0s):
            X.copy_(X0)
            n += ofsc.ofsc_iterate(g, 0, X, tol, iters).iterations
        return n

    out = {"workload": f"sbm_batch32: {len(probs)} SBMs, sum N = {sum(x.shape[0] for x in X0s)}, OFM-f1, "
                       f"every graph to tol {tol:g} (at most {iters} updates), FP32"}
    for name, fn in (("batched", batched), ("batched_grouped_launches", lambda: batched(4)), ("loop", loop)):
        fn()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        ups = sum(fn() for _ in range(steps))
        t1.record(stream)
        torch.cuda.synchronize()
        secs = t0.elapsed_time(t1) / 1000.0
        out[name] = {"updates_per_s": ups / secs, "ms_per_step": 1000.0 * secs / steps,
                     "updates_per_step": ups // steps}
    for g in graphs:
        g.free()
    return out


def run_stream(args):
    """Streaming form: the snapshots of a synth.STREAMS workload, each built on the device and
    iterated args.iters updates from the previous snapshot's X; one step = the whole stream, graph
    builds included. `value` = updates per second over the stream."""
    import torch

    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    from paper_2305_10356_gb300 import build, ofsc, synth
    build.build()
    snaps, x0 = synth.stream(args.workload, n=args.nodes)
    method = METHODS[args.method]
    gather = ofsc.GATHER_BF16 if args.gather == "bf16" else ofsc.GATHER_FP32
    dev = [(torch.from_numpy(e.src).cuda(), torch.from_numpy(e.dst).cuda()) for e in snaps]
    X0 = torch.from_numpy(x0).cuda()
    X = torch.empty_like(X0)
    stream = torch.cuda.current_stream()

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")  # the state is below 2x L2

    def step():
        flush.zero_()
        X.copy_(X0)
        n_up = 0
        for (src, dst), e in zip(dev, snaps):
            g = ofsc.ofsc_graph_build(e.n, src, dst)
            r = ofsc.ofsc_iterate(g, method, X, 0.0, args.iters, gather=gather)
            n_up += r.iterations
            g.free()
        return n_up

    for _ in range(args.warmup):
        step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    updates = 0
    for _ in range(args.steps):
        updates += step()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    ms = max_over_ranks(ms, world)
    spec = synth.STREAMS[args.workload]
    if rank == 0:
        line = {"metric": "OFM iterations/s", "value": updates * world / (ms / 1000.0), "unit": "iterations/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "storage": "f32" if args.gather == "fp32" else "bf16 gather copy, f32 master", "data": "synthetic",
                "config": {"workload": f"{args.workload}: SBM, N={args.nodes or spec['n']}, k={spec['n_blocks']}, "
                                       f"mean degree {spec['mean_degree']:g} at 100%, {spec['parts']} cumulative "
                                       f"edge-sampled snapshots, warm start, graph builds timed",
                           "updates_per_snapshot": args.iters, "method": METHOD_LABEL[args.method],
                           "l2": f"L2 flushed at the start of every step by a {2 * L2_BYTES >> 20} MB write "
                                 "inside the timed region"},
                "impl": "gpu", "parallelism": "replicas only" if world > 1 else "single GPU"}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """A batch of independent graphs (synth.BATCHES): one step = ofsc_iterate_batched over all of
    them, `iters` updates each from their X0. `value` = updates summed over the graphs per second.
    The same steps are also timed with direct launches (no CUDA graph replay) and as a loop of
    one ofsc_iterate call per graph."""
    import torch

    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    from paper_2305_10356_gb300 import build, ofsc, synth
    build.build()
    spec = synth.BATCHES[args.workload]
    scale = 1.0 if args.nodes is None else args.nodes / 51_000.0
    probs = synth.batch(args.workload, scale)
    method = METHODS[args.method]
    gather = ofsc.GATHER_BF16 if args.gather == "bf16" else ofsc.GATHER_FP32
    graphs, X0s = [], []
    for e, x0 in probs:
        src, dst = torch.from_numpy(e.src).cuda(), torch.from_numpy(e.dst).cuda()
        graphs.append(ofsc.ofsc_graph_build(e.n, src, dst))
        X0s.append(torch.from_numpy(x0).cuda())
    nnz = sum(int(g.info().nnz) for g in graphs)
    # the row-partition granularity of each graph's direction product, by timing (outside the
    # timed steps)
    shapes = [ofsc.ofsc_autotune(g, x.shape[1], gather) for g, x in zip(graphs, X0s)]
    tuned = [w // NUM_SMS for w, _, _ in shapes]
    tuned_slots = [u for _, u, _ in shapes]
    Xs = [torch.empty_like(x) for x in X0s]
    stream = torch.cuda.current_stream()

    def step_batched(direct=False, group=0):
        for X, X0 in zip(Xs, X0s):
            X.copy_(X0)
        rs = ofsc.ofsc_iterate_batched(graphs, method, Xs, 0.0, args.iters, gather=gather, direct_launch=direct,
                                       group_launches=group)
        return sum(r.iterations for r in rs), sum(r.kernel_launches for r in rs) + len(Xs)

    def step_loop():
        n_up = 0
        for g, X, X0 in zip(graphs, Xs, X0s):
            X.copy_(X0)
            n_up += ofsc.ofsc_iterate(g, method, X, 0.0, args.iters, gather=gather).iterations
        return n_up, 0

    def timed(fn, with_clocks=False):
        for _ in range(args.warmup):
            fn()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler = None
        if with_clocks:
            dev_id = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local if world > 1 else 0]
            try:
                dev_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid).replace("GPU-", "")
            except Exception:
                pass
            sampler = ClockSampler(dev_id)
            sampler.start()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        ups = launches = 0
        for _ in range(args.steps):
            u, l = fn()
            ups += u
            launches += l
        t1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        ms = t0.elapsed_time(t1)
        ms = max_over_ranks(ms, world)
        return ups * world / (ms / 1000.0), ms / args.steps, launches, clocks

    value, ms, launches, clocks = timed(step_batched, with_clocks=True)
    grouped, ms_grouped, launches_grouped, _ = timed(lambda: step_batched(group=4))
    direct, ms_direct, _, _ = timed(lambda: step_batched(True))
    loop, ms_loop, _, _ = timed(step_loop)

    # end to end: pinned host X0 -> device, one batched call, device -> pinned host X
    Xh0 = [x.cpu().pin_memory() for x in X0s]
    Xh = [torch.empty_like(x).pin_memory() for x in Xh0]

    def step_e2e():
        for X, h in zip(Xs, Xh0):
            X.copy_(h, non_blocking=True)
        rs = ofsc.ofsc_iterate_batched(graphs, method, Xs, 0.0, args.iters, gather=gather)
        for X, h in zip(Xs, Xh):
            h.copy_(X, non_blocking=True)
        return sum(r.iterations for r in rs), 0

    e2e_v, _, _, _ = timed(step_e2e)
    nbytes = sum(int(x.numel()) * 4 for x in X0s)
    if rank == 0:
        line = {"metric": "OFM iterations/s", "value": value, "unit": "iterations/s (summed over graphs)",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "storage": "f32" if args.gather == "fp32" else "bf16 gather copy, f32 master", "data": "synthetic",
                "config": {"workload": f"{args.workload}: {spec['count']} SBMs, N ~ U[{spec['n'][0]}, {spec['n'][1]}] "
                                       f"(x{scale:g}), k ~ U[{spec['k'][0]}, {spec['k'][1]}], mean degree ~ "
                                       f"U[{spec['mean_degree'][0]:g}, {spec['mean_degree'][1]:g}], within:between "
                                       f"{spec['ratio']:g}:1 (edge counts); sum N = {sum(x.shape[0] for x in X0s)}, "
                                       f"sum nnz = {nnz}",
                           "updates_per_graph_per_step": args.iters, "method": METHOD_LABEL[args.method],
                           "gather": args.gather, "l2": "state of all graphs about 1 GB, larger than L2",
                           "autotuned_warps_per_sm": {str(w): tuned.count(w) for w in sorted(set(tuned))},
                           "autotuned_slots_per_lane": {str(u): tuned_slots.count(u) for u in sorted(set(tuned_slots))}},
                "impl": "gpu", "e2e": {"value": e2e_v, "unit": "iterations/s (summed over graphs)",
                                       "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
                "clocks": clocks, "gpu_launches": launches,
                "batched_grouped_launches": {"value": grouped, "ms_per_step": ms_grouped, "lanes": 4,
                                             "gpu_launches": launches_grouped},
                "batched_direct_launch": {"value": direct, "ms_per_step": ms_direct},
                "per_graph_loop": {"value": loop, "ms_per_step": ms_loop},
                "parallelism": "replicas only" if world > 1 else "single GPU"}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_unrolled(args):
    """One step = one ofsc_unrolled_grad call: T updates of OFM-f1 from X_0, checkpointed, and the
    reverse sweep giving d f1(X_T) / d X_0 and, for a weighted graph, d f1(X_T) / d w.
    `value` = gradients per second; the FP64 oracle's reverse sweep is timed as the CPU baseline."""
    import torch

    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    from paper_2305_10356_gb300 import build, ofsc, synth
    build.build()
    e, x0 = synth.workload(args.workload, n=args.nodes)
    src, dst = torch.from_numpy(e.src).cuda(), torch.from_numpy(e.dst).cuda()
    w = None if e.w is None else torch.from_numpy(e.w).cuda()
    g = ofsc.ofsc_graph_build(e.n, src, dst, w)
    X0 = torch.from_numpy(x0).cuda()
    grad = torch.empty_like(X0)
    gw = torch.empty(e.src.size, dtype=torch.float32, device="cuda") if w is not None else None
    stream = torch.cuda.current_stream()
    T = args.unrolled
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda") if l2_flushed(args) else None

    def step():
        if flush is not None:
            flush.zero_()
        return ofsc.ofsc_unrolled_grad(g, X0, T, grad, ckpt=args.ckpt, src=src if w is not None else None,
                                       dst=dst if w is not None else None, grad_w=gw)

    for _ in range(args.warmup):
        step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    ms = max_over_ranks(ms, world)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import numpy as np
        from oracle import ofsc_oracle as o
        og = o.build_graph(e.n, e.src, e.dst, None if e.w is None else e.w.astype(np.float64), exact=e.w is not None)
        edges = None if e.w is None else (e.src, e.dst, e.w.astype(np.float64))
        c0 = time.perf_counter()
        o.unrolled_grad(og, x0.astype(np.float64), T, edges=edges)
        secs = time.perf_counter() - c0
        cpu = {"value": 1.0 / secs, "unit": "gradients/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "one full FP64 unrolled gradient (numpy/scipy oracle, whole trajectory kept, no checkpoints)"}
    if rank == 0:
        spec = synth.WORKLOADS[args.workload]
        line = {"metric": "unrolled gradients/s", "value": args.steps * world / (ms / 1000.0), "unit": "gradients/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"{args.workload}: N={e.n}, k={spec['n_blocks']}, "
                                       f"{'weighted' if e.w is not None else 'binary'}; d f1(X_T)/dX_0"
                                       f"{' and d/dw' if e.w is not None else ''} through T={T} OFM-f1 updates, "
                                       f"checkpoint every {args.ckpt}",
                           "T": T, "ckpt": args.ckpt, "l2": workload_config(args)["l2"]},
                "impl": "gpu", "cpu_baseline": cpu,
                "parallelism": "replicas only" if world > 1 else "single GPU"}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    from paper_2305_10356_gb300 import build, ofsc, synth
    build.build()
    e, x0 = synth.workload(args.workload, n=args.nodes)
    method = METHODS[args.method]
    gather = ofsc.GATHER_BF16 if args.gather == "bf16" else ofsc.GATHER_FP32
    src, dst = torch.from_numpy(e.src).cuda(), torch.from_numpy(e.dst).cuda()
    g = ofsc.ofsc_graph_build(e.n, src, dst)
    info = g.info()
    del src, dst
    X0 = torch.from_numpy(x0).cuda()
    X = torch.empty_like(X0)
    stream = torch.cuda.current_stream()
    eng = {"auto": ofsc.SPMM_AUTO, "simt": ofsc.SPMM_SIMT, "tma": ofsc.SPMM_TMA}[args.spmm_engine]
    # Between steps no input may be served from L2: either every N x kp block and the CSR are
    # larger than the L2, or the L2 is flushed (a write of twice its size) at the start of every
    # step, inside the timed region.
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda") if l2_flushed(args) else None

    def step(prof=None):
        if flush is not None:
            flush.zero_()
        X.copy_(X0)
        return ofsc.ofsc_iterate(g, method, X, 0.0, args.iters, gather=gather, profile=prof, spmm_engine=eng)

    for _ in range(args.warmup):
        step()
    dev_id = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local if world > 1 else 0]
    try:
        dev_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid).replace("GPU-", "")
    except Exception:
        pass
    sampler = ClockSampler(dev_id)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    launches = 0
    for _ in range(args.steps):
        r = step()  # the library's default path: repeating updates replayed from a CUDA graph
        launches += r.kernel_launches  # the library's kernels (not the X0 copy or the L2 flush)
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    elapsed_ms = max_over_ranks(elapsed_ms, world)
    updates = args.iters * args.steps * world
    value = updates / (elapsed_ms / 1000.0)

    # per-phase device times from separate, untimed steps with CUDA events around every launch
    # (direct launches; the events and launches cost host time, so these steps are not `value`)
    prof = ofsc.Profile()
    prof_steps = min(args.steps, 3)
    torch.cuda.synchronize()
    pp_start = torch.cuda.Event(enable_timing=True)
    pp_end = torch.cuda.Event(enable_timing=True)
    pp_start.record(stream)
    for _ in range(prof_steps):
        step(prof)
    pp_end.record(stream)
    torch.cuda.synchronize()
    profiled_ms_per_step = pp_start.elapsed_time(pp_end) / prof_steps

    # the plain FP32 path on the same steps, for the mixed-vs-plain comparison of the metric
    plain = None
    if gather == ofsc.GATHER_BF16 and not args.no_fp32_compare:
        def step32():
            if flush is not None:
                flush.zero_()
            X.copy_(X0)
            return ofsc.ofsc_iterate(g, method, X, 0.0, args.iters, gather=ofsc.GATHER_FP32, spmm_engine=eng)
        step32()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        p_start = torch.cuda.Event(enable_timing=True)
        p_end = torch.cuda.Event(enable_timing=True)
        p_start.record(stream)
        for _ in range(args.steps):
            step32()
        p_end.record(stream)
        torch.cuda.synchronize()
        p_ms = p_start.elapsed_time(p_end)
        p_ms = max_over_ranks(p_ms, world)
        plain = {"value": updates / (p_ms / 1000.0), "unit": "iterations/s", "ms_per_step": p_ms / args.steps,
                 "gather": "fp32"}

    # end to end through the public API from pinned host buffers: every step uploads its X0 and
    # downloads its X. Serial: upload, iterate, download. Pipelined (reported as `value`): two
    # device buffers, the next step's upload and the previous step's download run on a copy
    # stream while the current step iterates. Wall clock from a synchronised start to the last
    # download, copy stream included.
    Xh0 = torch.from_numpy(x0).pin_memory()
    Xh = [torch.empty_like(Xh0).pin_memory() for _ in range(2)]
    Xd = [torch.empty_like(X0) for _ in range(2)]
    copy = torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]

    def e2e_run(pipelined: bool) -> float:
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        w0 = time.perf_counter()
        if pipelined:
            with torch.cuda.stream(copy):
                Xd[0].copy_(Xh0, non_blocking=True)
                ev_in[0].record(copy)
        for i in range(args.steps):
            cur = i % 2
            if pipelined:
                stream.wait_event(ev_in[cur])
                if i + 1 < args.steps:
                    nxt = (i + 1) % 2
                    with torch.cuda.stream(copy):  # after the download of step i - 1 (same stream)
                        Xd[nxt].copy_(Xh0, non_blocking=True)
                        ev_in[nxt].record(copy)
            else:
                Xd[cur].copy_(Xh0, non_blocking=True)
            if flush is not None:
                flush.zero_()
            ofsc.ofsc_iterate(g, method, Xd[cur], 0.0, args.iters, gather=gather, spmm_engine=eng)
            if pipelined:
                ev_done[cur].record(stream)
                with torch.cuda.stream(copy):
                    copy.wait_event(ev_done[cur])
                    Xh[cur].copy_(Xd[cur], non_blocking=True)
            else:
                Xh[cur].copy_(Xd[cur], non_blocking=True)
        torch.cuda.synchronize()
        secs = time.perf_counter() - w0
        secs = max_over_ranks(secs, world)
        return secs

    e2e_serial_s = e2e_run(False)
    e2e_s = e2e_run(True)
    e2e = {"value": updates / e2e_s, "unit": "iterations/s",
           "h2d_bytes_per_step": int(x0.nbytes), "d2h_bytes_per_step": int(x0.nbytes),
           "form": "pipelined: upload of step i+1 and download of step i-1 overlap step i",
           "serial_value": updates / e2e_serial_s}

    # time to tolerance: the subspace angle to an FP32 reference run of 400 updates
    ttt = None
    if rank == 0 and not args.no_time_to_tol:
        ttt = time_to_tol(g, method, e.n, e.n_blocks, stream, 2305 * 1000 + 50)

    # dominant kernel (the direction product, phase "spmm") and its roofline
    pd = prof.as_dict()
    dom = max(pd, key=lambda p: pd[p]["ms"])
    kp = ((e.n_blocks + 7) // 8) * 8
    gb = 2 if args.gather == "bf16" else 4
    peaks = load_peaks()
    per_launch_ms = pd["spmm"]["ms"] / max(1, pd["spmm"]["launches"])
    wk = args.workload if args.nodes is None else f"{args.workload}@{args.nodes}"
    tr = measured_traffic(wk, args.gather)
    tr_any = tr or measured_traffic(wk, args.gather, any_build=True)
    # L2 hit rate of the gathers: from the measured DRAM reads of the kernel (the rows that did not
    # come from DRAM came from L2). A capture of an earlier build still gives the cost model's h
    # (the hit rate belongs to the graph and the access order); its counters are then not reported
    # as this build's traffic. With no capture at all h = 0 (every gathered row from HBM).
    h = 0.0
    h_source = "none: every gathered row counted as HBM bytes"
    if tr_any is not None:
        base = spmm_bytes(e.n, kp, int(info.nnz), gb, bool(info.weighted), 0.0)
        miss = tr_any["dram_read_bytes"] - base["csr"] - base["epilogue"]
        h = min(1.0, max(0.0, 1.0 - miss / base["gather_all"]))
        h_source = ("ncu DRAM reads of this build" if tr is not None else
                    f"ncu DRAM reads of an earlier build (sources {tr_any['source_digest']}, now "
                    f"{source_digest(DIR_PRODUCT_SOURCES)})")
    alg = spmm_bytes(e.n, kp, int(info.nnz), gb, bool(info.weighted), h)
    achieved = alg["total"] / (per_launch_ms / 1000.0) / 1e9
    roof = {"bound": "hbm", "kernel": "k_spmm_dir (direction product W = A V)", "achieved": achieved,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
            "traffic": (tr["dram_read_bytes"] + tr["dram_write_bytes"]) if tr else None,
            "peak_source": f"{peaks['source']} (copy bandwidth)",
            "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
            "algorithmic_bytes": alg["total"], "gather_l2_hit": round(h, 4), "gather_l2_hit_source": h_source,
            "ms_per_launch": per_launch_ms, "dominant_phase": dom}

    # the whole update: the compulsory-bytes model (and the DRAM bytes of all its kernels from one
    # ncu capture, profiles/traffic.json) over the device time per update. `frac` divides by the
    # full time per update, exact refreshes included (they are part of every call); `frac_steady`
    # by the time of the updates without a refresh.
    # time per update from the timed steps (graph replay, no host gaps); the exact refreshes'
    # share of it from the profiled steps
    all_ms = elapsed_ms / (args.iters * args.steps)
    upd_ms = all_ms - pd["refresh"]["ms"] / (args.iters * prof_steps)
    tu = measured_traffic(f"{args.workload}/{args.gather}" if args.nodes is None else "", "update")
    nkp = e.n * kp
    useful = (alg["total"]                      # the direction product (gathers net of L2 hits)
              + 32 * nkp                        # direction pass: read X, AX, V, AV, G_p; write X, AX, G
              + 12 * nkp + gb * nkp             # V pass: read G, V; write V, D^-1/2 V
              + 8 * nkp)                        # Grams: read V, X
    useful_gbs = useful / (all_ms / 1000.0) / 1e9
    # All the compulsory bytes of one call: its updates, the exact refreshes at its start and end
    # (D^-1/2 X; A X with FP32 gathers; X^T X and X^T AX), the direction pass of update maxit,
    # the evaluation pass of the report, and the copies of X in and out of the padded layout.
    # The FP32 product's gathers hit L2 at the rate of that kernel's capture, else at this one's.
    tr32 = measured_traffic(wk, "fp32", any_build=True)
    h32 = h
    if tr32 is not None:
        b32 = spmm_bytes(e.n, kp, int(info.nnz), 4, bool(info.weighted), 0.0)
        h32 = min(1.0, max(0.0, 1.0 - (tr32["dram_read_bytes"] - b32["csr"] - b32["epilogue"]) / b32["gather_all"]))
    refresh = 8 * nkp + spmm_bytes(e.n, kp, int(info.nnz), 4, bool(info.weighted), h32)["total"] + 8 * nkp
    nk = e.n * e.n_blocks
    call = (args.iters * useful + 2 * refresh + 32 * nkp + 8 * nkp
            + (4 * nk + 4 * nkp) + (4 * nkp + 4 * nk))
    call_frac = call / (all_ms * args.iters / 1000.0) / 1e9 / peaks["hbm_gbs"]
    iteration = {"ms_per_update": all_ms, "ms_per_update_steady": upd_ms, "useful_bytes": useful,
                 "useful_gbs": useful_gbs, "frac": useful_gbs / peaks["hbm_gbs"],
                 "frac_steady": useful / (upd_ms / 1000.0) / 1e9 / peaks["hbm_gbs"],
                 "useful_bytes_per_call": call, "refresh_gather_l2_hit": round(h32, 4), "frac_call": call_frac,
                 "target_frac": 0.70, "gap_to_target": 0.70 - useful_gbs / peaks["hbm_gbs"],
                 "dram_bytes": (tu["dram_read_bytes"] + tu["dram_write_bytes"]) if tu else None}
    if tu:
        gbs = iteration["dram_bytes"] / (upd_ms / 1000.0) / 1e9
        iteration.update({"dram_gbs_steady": gbs, "dram_frac_steady": gbs / peaks["hbm_gbs"]})

    legs = None
    if rank == 0 and not args.no_legs and args.nodes is None:
        legs = {"c1_all_methods": c1_leg(stream), "batched_vs_loop": batched_leg(stream)}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        og, xs, n_s, n_full = oracle_sample(args)
        secs = cpu_oracle_step(og, method, xs) * n_full / n_s
        s1 = oracle_one_thread_seconds(args)
        cpu = {"value": 1.0 / secs, "unit": "iterations/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": SAMPLE_TEXT, "cpu_model": cpu_model(),
               "value_1thread": (1.0 / s1) if s1 else None,
               "sample_1thread": f"one update on N/{ONE_THREAD_FRACTION} nodes, BLAS on one thread, scaled to N"}
    if rank == 0:
        line = {"metric": "OFM iterations/s", "value": value, "unit": "iterations/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "storage": "f32" if args.gather == "fp32" else "bf16 gather copy, f32 master",
                "data": "synthetic", "config": workload_config(args), "impl": "gpu",
                "roofline": roof, "iteration_hbm": iteration, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches, "plain_fp32": plain, "time_to_tol": ttt, "legs": legs,
                "phases_ms_per_step": {p: pd[p]["ms"] / prof_steps for p in pd},
                "profiled_ms_per_step": profiled_ms_per_step,
                "parallelism": "replicas only" if world > 1 else "single GPU"}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    from paper_2305_10356_gb300 import synth
    if args.workload in synth.STREAMS:
        return run_stream(args)
    if args.workload in synth.BATCHES:
        return run_batch(args)
    if args.unrolled > 0:
        return run_unrolled(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
