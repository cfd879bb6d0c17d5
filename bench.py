#!/usr/bin/env python3
"""Throughput benchmark of the GB300 hash SpGEMM (C = A*A on synthetic R-MAT).

One step = one whole product through the C ABI: plan (row flop pass and
binning), symbolic phase (counts, row_ptr scan, nnz(C) to the host), the
allocation of C, and the numeric phase (accumulation and, in sorted mode,
the per-row sort).  Inputs are resident in HBM when a step starts.  Inputs
(about 23 MB) are smaller than L2, so a 256 MiB buffer is written between
steps to flush L2; each step is timed alone with CUDA events on the
launching stream, the flush outside the events.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on
the same workload instead (rank 0 only; other ranks exit at once).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                        [--unsorted] [--impl reference]
Workloads: the named single products of inputs.WORKLOADS (default
rmat16_ef16_f64; also er4096_k8_f64, rmat18_frontier1024_f32,
tc_rmat16_lu_f64), batch_er2000 (batched products), serve_mix (serving
loop), sweep_rmat (density and size sweeps), ablate_probe (linear vs
chunked hash probing) and numeric_repeat (repeated numeric phases of one
structure, plain and as a CUDA graph).
For N > 1 launch under torch.distributed.run: each rank runs an
independent replica on its own GPU (weak scaling); timing takes the maximum
over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpGEMM GFLOP/s (2*flop per second)"
# FP64 peak derived from unit counts and clocks: 152 SMs x 2 FP64 FMA per
# clock per SM x 2070 MHz x 2 FLOP per FMA (= the nominal 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2.070e9 * 2 / 1e12
HBM_FALLBACK_GBS = 6800.0
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="rmat16_ef16_f64")
    p.add_argument("--unsorted", action="store_true", help="time unsorted output as the headline")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--row-blocks", type=int, default=0,
                   help="row blocks of the end-to-end product (0: the library's default)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-variant", action="store_true", help="skip timing the other sort mode")
    return p.parse_args()


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def workload_accounting(A, B, nnz_c: int, vsize: int) -> dict:
    """Algorithmic bytes of the whole path: A once, every touched row of B once,
    C written once (row_ptr + col_idx + values)."""
    flop = int(np.diff(B.row_ptr.astype(np.int64))[A.col_idx].sum())
    touched = np.unique(A.col_idx)
    b_rows = np.diff(B.row_ptr.astype(np.int64))[touched]
    bytes_a = (A.nrows + 1) * 4 + A.nnz * (4 + vsize)
    bytes_b = int(len(touched) * 8 + b_rows.sum() * (4 + vsize))
    bytes_c = (A.nrows + 1) * 4 + nnz_c * (4 + vsize)
    return dict(flop=flop, bytes_alg=bytes_a + bytes_b + bytes_c, bytes_a=bytes_a, bytes_b=bytes_b, bytes_c=bytes_c)


class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.out.close()

    def summary(self) -> dict | None:
        if self.proc is None or not self.path:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def source_digest() -> str:
    """Digest of the kernel sources with comments and blank space removed, so
    that edits to comments do not mark committed counters as stale."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1804_01698_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            code = f.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        code = " ".join(code.split())
        h.update(name.encode() + code.encode())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    e = rec.get(workload, {}).get(kernel)
    if not e or e.get("source_digest") != source_digest():
        return None
    return e.get("dram_bytes_per_launch")


def kernel_units(name: str, stats: dict) -> tuple[int, str]:
    """Useful multiply-adds (products) one launch of `name` performs, from the
    plan's per-bin flop totals."""
    kind, _, size = name.rpartition("_")
    named = {"num_bitmap_l": ("num", 9), "num_global": ("num", 10), "num_bitmap_s": ("num", 11),
             "num_bitmap_m": ("num", 12), "sym_bitmap_heavy": ("sym", 10), "sym_bitmap_mid": ("sym", 11),
             "sym_global": ("sym", 12)}
    if name in named:
        phase, b = named[name]
        return stats[f"{phase}_bin_flop"][b], "numeric" if phase == "num" else "symbolic"
    if size.isdigit():
        table = int(size)
        if kind.startswith("num_"):
            for b, t in enumerate(stats["num_bin_table"]):
                if t == table:
                    return stats["num_bin_flop"][b], "numeric"
        if kind.startswith("sym_"):
            for b, t in enumerate(stats["sym_bin_table"]):
                if t == table:
                    return stats["sym_bin_flop"][b], "symbolic"
    return 0, "other"


def planning_bytes(name: str, A, B, stats: dict) -> tuple[int, str]:
    """Algorithmic bytes of one launch of a planning scope: what it must read
    and write at least once.  row_flop (the flop pass): A's row pointers and
    columns, the pair of B row pointers each stored a_ik selects, and the
    per-row flop, count and bin; compact_a: the per-row counts, the compacted
    row pointers, and per kept entry its column read and its column and
    source written."""
    m, nnz_a = A.nrows, A.nnz
    if name.startswith("row_flop"):
        b = (m + 1) * 4 + nnz_a * 4 + nnz_a * 8 + m * (8 + 4 + 1)
        return b, f"{b} B: A's structure, 8 B of B's row pointers per stored a_ik, 13 B per row"
    if name.startswith("compact_a"):
        kept = int(stats.get("nnz_a_walked", nnz_a))
        b = m * 4 + (m + 1) * 4 + kept * 12
        return b, f"{b} B: per-row counts and row pointers, 12 B per kept a_ik"
    return 0, "no algorithmic byte count for this step"


# ---------------------------------------------------------------------------- reference arm

def workload_config(name: str, A, B, flop: int, nnz_c: int, sorted_output: bool, replicas: int) -> dict:
    """The `config` of a single-product bench line, the same for both arms."""
    from paper_1804_01698_gb300 import inputs
    return {"workload": name, "desc": inputs.WORKLOADS[name]["desc"], "m": A.nrows, "n": A.ncols, "k": B.ncols,
            "nnz_a": A.nnz, "nnz_b": B.nnz, "flop": flop, "nnz_c": int(nnz_c), "sorted": bool(sorted_output),
            "l2": "flushed between steps (256 MiB write, outside the events)", "replicas": replicas}


def run_reference(args) -> int:
    import oracle
    from paper_1804_01698_gb300 import inputs

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload not in inputs.WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single-product workloads; "
                          f"{args.workload} is compared against one GPU call per product instead"}), flush=True)
        return 0
    A, B, sorted_default = inputs.workload(args.workload)
    sorted_output = sorted_default and not args.unsorted
    cores = len(os.sched_getaffinity(0))
    flop = int(oracle.row_flop(A, B).sum())
    nnz_c = 0
    for _ in range(args.warmup):
        nnz_c = oracle.spgemm(A, B, nthreads=cores)[0].nnz
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        nnz_c = oracle.spgemm(A, B, nthreads=cores)[0].nnz
        times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    value = 2 * flop / mean / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if A.vals.dtype == np.float64 else "f32",
        "data": "synthetic",
        "config": workload_config(args.workload, A, B, flop, nnz_c, sorted_output, args.gpus),
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": "the whole product per step (dense-SPA Gustavson, rows split by RowsToThreads)"},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------- batched products

def waves_by_flop(flops, limit=2**31 - 1):
    """Consecutive groups of products whose summed flop (a bound on nnz of C)
    stays within int32 indexing."""
    waves, cur, tot = [], [], 0
    for i, f in enumerate(flops):
        if cur and tot + f > limit:
            waves.append(cur)
            cur, tot = [], 0
        cur.append(i)
        tot += f
    if cur:
        waves.append(cur)
    return waves


def run_batch(args) -> int:
    """2000 independent Erdos-Renyi products A_i*A_i (n_i log-uniform in
    [256, 65536], k_i nonzeros per row uniform in {2..32}, FP64), timed as one
    CUDA graph launch of the whole batch (the headline), as packed batches
    launched wave by wave (waves of products whose summed flop fits int32
    indexing) and as one call per product.  Inputs are resident on the
    device."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1804_01698_gb300 import binding as sg
    from paper_1804_01698_gb300 import inputs

    count = int(args.workload.split("er")[-1]) if args.workload.startswith("batch_er") else 2000
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.time()
    mats = inputs.er_batch(count, seed=inputs.SEED_BASE + 3)
    gen_s = time.time() - t0
    flops = [m.nrows * (m.nnz // max(m.nrows, 1)) ** 2 for m in mats]   # exactly k^2 per row
    dm = [sg.to_device(m, dev) for m in mats]
    stream = torch.cuda.current_stream(dev)
    waves = waves_by_flop(flops)

    def plain_pass():
        launches = 0
        for d in dm:
            p = sg.Plan(d, d, True, stream=stream)
            p.symbolic()
            p.numeric()
            launches += p.stats()["kernel_launches"]
            p.destroy()
        return launches

    def batch_pass(candidate=None):
        kw, tuning = _split(candidate) if candidate else ({}, None)
        launches = 0
        for w in waves:
            b = sg.Batch([dm[i] for i in w], [dm[i] for i in w], True, stream=stream, tuning=tuning, **kw)
            b.symbolic()
            b.numeric()
            launches += b.plan_stats()["kernel_launches"] + 2     # + pack, unpack
            b.destroy()
        return launches

    def timed(fn, k, w):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        ts, launches = [], 0
        for _ in range(k):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launches = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return sum(ts) / len(ts), launches

    # autotuning (bin threshold, lanes per a_ik) on a sample: every 10th product
    from paper_1804_01698_gb300.tune import _split, autotune_batch
    sample = [dm[i] for i in range(0, count, 10)]
    t0 = time.time()
    tuning, tune_table = autotune_batch(sample, sample, True, steps=2, stream=stream)
    tune_s = time.time() - t0
    # the whole batch as one CUDA graph: planned and captured once (setup),
    # then one graph launch per pass that recomputes every product
    kw_g, tuning_g = _split(tuning) if tuning else ({}, None)
    t0 = time.time()
    graph = sg.BatchGraph(dm, dm, True, stream=stream, tuning=tuning_g, **kw_g)
    graph_setup_s = time.time() - t0
    ginfo = graph.info()

    def graph_pass():
        graph.launch()
        return 1

    with ClockSampler(0) as clocks:
        t_graph, _ = timed(graph_pass, args.steps, max(1, args.warmup))
        graph.wait()
        graph.destroy()
        t_batch, l_batch = timed(lambda: batch_pass(tuning), args.steps, max(1, args.warmup))
        t_default, _ = timed(batch_pass, args.steps, max(1, args.warmup))
        t_plain, l_plain = timed(plain_pass, args.steps, max(1, args.warmup))
    flop = sum(flops)
    line = {
        "metric": "batched SpGEMM solves/s (products per second)", "value": count / t_graph, "unit": "solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": max(1, args.warmup), "ms_per_step": t_graph * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{count} Erdos-Renyi products A_i*A_i, n_i log-uniform in [256,65536], "
                               "k_i uniform in {2..32} per row, FP64, sorted output, autotuned plan, "
                               "one CUDA graph launch per pass",
                   "products": count, "flop": flop, "nnz_a": sum(m.nnz for m in mats), "waves": len(waves),
                   "generation_s": gen_s, "l2": "inputs larger than L2"},
        "graph": {"solves_per_s": count / t_graph, "gflops": 2 * flop / t_graph / 1e9, "s_per_pass": t_graph,
                  "host_launches_per_pass": 1, "kernel_nodes": ginfo["kernel_nodes"], "waves": ginfo["waves"],
                  "device_bytes": ginfo["bytes"], "setup_s": graph_setup_s, "tuning": tuning},
        "batched": {"solves_per_s": count / t_batch, "gflops": 2 * flop / t_batch / 1e9, "s_per_pass": t_batch,
                    "kernel_launches": l_batch, "tuning": tuning},
        "batched_default_tuning": {"solves_per_s": count / t_default, "s_per_pass": t_default},
        "autotune": {"sample": f"every 10th product ({len(sample)} products, one packed batch)",
                     "seconds": tune_s, "candidates_ms": [[t, ms] for t, ms in tune_table]},
        "one_call_per_product": {"solves_per_s": count / t_plain, "gflops": 2 * flop / t_plain / 1e9,
                                 "s_per_pass": t_plain, "kernel_launches": l_plain},
        "speedup": t_plain / t_graph,
        "gpu_launches": ginfo["kernel_nodes"] * args.steps,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args) -> int:
    """The serving loop: a stream of products mixing Erdos-Renyi A*A (sizes
    as the batched workload) and AMG-style A*P (7-point Poisson on a g^3
    grid, g uniform in {8..48}, times 2x2x2 aggregation), FP64, sorted
    output, operands resident on the device.  The headline is the served
    rate at saturation (every request present at time 0); a sweep of
    Poisson arrival rates gives solves/s and p50/p99 latency of the
    continuous-batching server and of one call per product on the same
    arrivals.  Admission: 40 GB cap on the symbolic-pass memory estimate."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1804_01698_gb300 import binding as sg
    from paper_1804_01698_gb300 import inputs
    from paper_1804_01698_gb300.serve import GpuBackend, Request, Server, serve_one_by_one

    tail = args.workload[len("serve_mix"):]
    count = int(tail) if tail else 600
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.time()
    mix = inputs.serving_mix(count, seed=inputs.SEED_BASE + 5)
    gen_s = time.time() - t0
    reqs, flop = [], 0
    for i, (A, B) in enumerate(mix):
        dA = sg.to_device(A, dev)
        dB = dA if B is A else sg.to_device(B, dev)
        f = int(np.diff(B.row_ptr)[A.col_idx].sum())
        flop += f
        reqs.append(Request(i, dA, dB, 0.0, f))
    torch.cuda.synchronize()
    cap = 40 << 30

    def with_arrivals(times):
        return [Request(r.rid, r.A, r.B, float(t), r.flop) for r, t in zip(reqs, times)]

    def served(rs):
        be = GpuBackend(sorted_output=True, nstreams=4, device=dev)
        st = Server(be, mem_cap=cap, max_batch=64, max_inflight=3).run(rs)
        torch.cuda.synchronize()
        return st, be.kernel_launches

    def alone(rs):
        be = GpuBackend(sorted_output=True, nstreams=1, device=dev)
        st = serve_one_by_one(be, rs)
        torch.cuda.synchronize()
        return st, be.kernel_launches

    with ClockSampler(0) as clocks:
        for _ in range(max(1, args.warmup)):
            served(reqs)
            alone(reqs[: max(1, count // 4)])
        sat, launches = [], 0
        for _ in range(args.steps):
            st, launches = served(reqs)
            sat.append(st)
        base, base_launches = alone(reqs)
        sweep = []
        cap_alone = base.solves_per_s()
        for mult in (0.5, 0.9, 1.5, 3.0):
            rate = mult * cap_alone
            rs = with_arrivals(inputs.poisson_arrivals(count, rate, inputs.SEED_BASE + 6))
            a, _ = served(rs)
            b, _ = alone(rs)
            sweep.append({"rate_per_s": rate, "served": a.summary(), "one_call_per_product": b.summary()})
    wall = statistics.median(s.wall for s in sat)
    best = min(sat, key=lambda s: s.wall)
    line = {
        "metric": "served SpGEMM solves/s (products per second)", "value": count / wall, "unit": "solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": max(1, args.warmup), "ms_per_step": wall * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"serving mix of {count} products: 1/2 Erdos-Renyi A*A (n log-uniform in "
                               "[256,65536], 2..32 nonzeros per row), 1/2 AMG A*P (7-point Poisson on g^3, "
                               "g uniform in {8..48}, 2x2x2 aggregation); FP64, sorted output",
                   "requests": count, "flop": flop, "mem_cap_bytes": cap, "max_batch": 64, "max_inflight": 3,
                   "generation_s": gen_s, "l2": "operands of the whole stream (GBs) larger than L2"},
        "saturation": {"served": best.summary(), "one_call_per_product": base.summary(),
                       "speedup": base.wall / wall},
        "sweep": sweep,
        "e2e": None,
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_sweep(args) -> int:
    """Scaling with density and with size, as Sec. 5.4.1 and 5.4.2 measure
    them: C = A*A for R-MAT matrices of G500 skew (.57,.19,.19,.05) and of
    uniform (ER, .25 each) parameters, (a) at scale 16 with edge factor 2 to
    64 and (b) at edge factor 16 with scale 8 to 17; FP64, sorted and
    unsorted output.  Each point is timed like the headline step (plan,
    symbolic, allocation of C, numeric; L2 flushed between steps)."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1804_01698_gb300 import binding as sg
    from paper_1804_01698_gb300 import inputs

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    kinds = {"g500": (0.57, 0.19, 0.19, 0.05), "er": (0.25, 0.25, 0.25, 0.25)}
    points = [("density", kind, 16, ef) for kind in kinds for ef in (2, 4, 8, 16, 32, 64)]
    points += [("size", kind, sc, 16) for kind in kinds for sc in (8, 10, 12, 14, 16, 17)]
    steps = max(1, min(args.steps, 5))
    rows, launches = [], 0
    with ClockSampler(0) as clocks:
        for sweep, kind, scale, ef in points:
            A = inputs.rmat(scale, ef, abcd=kinds[kind], seed=inputs.SEED_BASE + 7 + scale * 100 + ef)
            dA = sg.to_device(A, dev)
            row = {"sweep": sweep, "kind": kind, "scale": scale, "edge_factor": ef, "nnz_a": A.nnz}
            for sorted_flag in (True, False):
                ts = []
                for it in range(steps + 1):
                    flush.fill_(it & 0xFF)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    plan = sg.Plan(dA, dA, sorted_flag, stream=stream)
                    nnz = plan.symbolic()
                    C = plan.numeric()
                    e1.record(stream)
                    e1.synchronize()
                    st = plan.stats()
                    if st["status"] != 0:
                        raise RuntimeError(f"device error status {st['status']}")
                    if it > 0:                       # the first run is the warm-up
                        ts.append(e0.elapsed_time(e1))
                        launches += st["kernel_launches"]
                    plan.destroy()
                    del C
                flop = st["total_flop"]
                ms = statistics.median(ts)
                row["flop"], row["nnz_c"] = flop, nnz
                row["sorted_gflops" if sorted_flag else "unsorted_gflops"] = 2 * flop / (ms * 1e-3) / 1e9
                row["sorted_ms" if sorted_flag else "unsorted_ms"] = ms
            row["compression_ratio"] = row["flop"] / row["nnz_c"] if row["nnz_c"] else None
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
            del dA
    g16 = next(r for r in rows if r["sweep"] == "density" and r["kind"] == "g500" and r["edge_factor"] == 16)
    line = {
        "metric": "SpGEMM GFLOP/s (2*flop per second)", "value": g16["sorted_gflops"], "unit": "GFLOP/s",
        "n_gpus": 1, "steps": steps, "warmup": 1, "ms_per_step": g16["sorted_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "R-MAT A*A sweeps: scale 16 with edge factor 2..64, and edge factor 16 with scale "
                               "8..17; G500 and ER parameters; FP64; sorted and unsorted",
                   "headline_point": "G500 scale 16 EF 16, sorted", "l2": "256 MiB flush between steps",
                   "timing": "median over steps per point"},
        "sweep": rows,
        "e2e": None,
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def collision_factor(A, B, row_nnz, rows, chunk: bool, high: bool = False) -> float:
    """Probes per insertion (the collision factor c of Eq. 2) of the numeric
    hash tables, simulated sequentially on the given rows: each row's table
    has the size its bin gives it (warp tables of S = 64..1024 slots hold
    up to S/2 keys, block tables of 2048..16384 slots up to 3S/4), keys
    arrive in product order, slot = (col * 2654435761) mod S (or, `high`,
    its top log2(S) bits of 32).  Linear probing reads one slot per probe;
    chunked probing reads 4 (one probe)."""
    caps = [(s, s // 2) for s in (64, 128, 256, 512, 1024)] + [(s, 3 * s // 4) for s in (2048, 4096, 8192, 16384)]
    probes = inserts = 0
    for i in rows:
        nnz = int(row_nnz[i])
        size = next((s for s, c in caps if nnz <= c), None)
        if size is None or nnz == 0:
            continue
        mask = size - 1
        tab = [-1] * size
        for j in range(A.row_ptr[i], A.row_ptr[i + 1]):
            k = A.col_idx[j]
            for q in range(B.row_ptr[k], B.row_ptr[k + 1]):
                col = int(B.col_idx[q])
                x = (col * 2654435761) & 0xFFFFFFFF
                h = (x >> (32 - size.bit_length() + 1)) if high else (x & mask)
                inserts += 1
                if chunk:
                    h &= ~3
                    while True:
                        probes += 1
                        chunk4 = tab[h:h + 4]
                        if col in chunk4:
                            break
                        if -1 in chunk4:
                            tab[h + chunk4.index(-1)] = col
                            break
                        h = (h + 4) & mask
                else:
                    while True:
                        probes += 1
                        if tab[h] == col:
                            break
                        if tab[h] == -1:
                            tab[h] = col
                            break
                        h = (h + 1) & mask
    return probes / inserts if inserts else float("nan")


def run_ablate_probe(args) -> int:
    """Ablation of the hash probing of Sec. 4.2.1 (one slot per probe) against
    the chunked probing of HashVector, Sec. 4.2.2 (4 slots per 16-byte load,
    SPGEMM_PROBE_CHUNK4): whole products (concurrent bins, L2 flushed) and
    the hash-table kernels alone (bins serialised, an event pair per
    kernel), plus the collision factor c of Eq. 2 of each scheme: counted on
    the device (SPGEMM_COUNT_PROBES, every hash insert of both phases) and
    simulated sequentially on a sample of rows."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1804_01698_gb300 import binding as sg
    from paper_1804_01698_gb300 import inputs

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    er16 = inputs.rmat(16, 16, abcd=(0.25, 0.25, 0.25, 0.25), seed=inputs.SEED_BASE + 8)
    cases = [("rmat16_ef16_f64", *inputs.workload("rmat16_ef16_f64")[:2]), ("er_rmat16_ef16_f64", er16, er16),
             ("tc_rmat16_lu_f64", *inputs.workload("tc_rmat16_lu_f64")[:2])]
    steps = max(1, min(args.steps, 10))
    rows_out, launches = [], 0
    rng = np.random.default_rng(5)
    with ClockSampler(0) as clocks:
        for name, A, B in cases:
            dA = sg.to_device(A, dev)
            dB = dA if B is A else sg.to_device(B, dev)
            row = {"workload": name, "flop": None}
            for probe, hsh in (("linear", "low"), ("chunk4", "low"), ("linear", "high"), ("chunk4", "high")):
                tag = probe if hsh == "low" else f"{probe}_high"   # plain names: the paper's low-bits hash
                for timing in (False, True):
                    ts, kt = [], {}
                    for it in range(steps + 1):
                        flush.fill_(it & 0xFF)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        plan = sg.Plan(dA, dB, True, stream=stream, timing=timing, serial=timing, probe=probe,
                                       hash=hsh)
                        plan.symbolic()
                        C = plan.numeric()
                        e1.record(stream)
                        e1.synchronize()
                        st = plan.stats()
                        if st["status"] != 0:
                            raise RuntimeError(f"device error status {st['status']}")
                        if it > 0:
                            ts.append(e0.elapsed_time(e1))
                            launches += st["kernel_launches"]
                            if timing:
                                for k, (ms, _) in plan.kernel_times().items():
                                    kt[k] = kt.get(k, 0.0) + ms / steps
                        if tag == "linear" and not timing and it == 0:
                            row_nnz = plan.row_nnz().cpu().numpy()
                        plan.destroy()
                        del C
                    if timing:
                        hash_ms = sum(v for k, v in kt.items() if k.startswith(("sym_warp", "sym_block", "num_warp",
                                                                                   "num_block", "sym_global",
                                                                                   "num_global")))
                        row[tag + "_hash_kernels_ms"] = hash_ms
                    else:
                        row[tag + "_step_ms"] = statistics.median(ts)
                row["flop"] = st["total_flop"]
                # the collision factor measured on the device (SPGEMM_COUNT_PROBES, an untimed run)
                with sg.Plan(dA, dB, True, stream=stream, probe=probe, hash=hsh, count_probes=True) as cp:
                    cp.symbolic()
                    cp.numeric()
                    cs = cp.stats()
                row[f"c_gpu_{tag}"] = {
                    "symbolic": cs["sym_probes"] / cs["sym_inserts"] if cs["sym_inserts"] else None,
                    "numeric": cs["num_probes"] / cs["num_inserts"] if cs["num_inserts"] else None,
                    "hash_inserts": cs["sym_inserts"] + cs["num_inserts"]}
            hash_rows = np.nonzero((row_nnz > 0) & (row_nnz <= 12288))[0]
            sample = rng.choice(hash_rows, size=min(300, len(hash_rows)), replace=False) if len(hash_rows) else []
            row["c_linear"] = collision_factor(A, B, row_nnz, sample, False)
            row["c_chunk4"] = collision_factor(A, B, row_nnz, sample, True)
            row["c_linear_high"] = collision_factor(A, B, row_nnz, sample, False, True)
            row["c_chunk4_high"] = collision_factor(A, B, row_nnz, sample, True, True)
            row["c_sample_rows"] = len(sample)
            rows_out.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
            del dA, dB
    head = rows_out[0]
    line = {
        "metric": "SpGEMM GFLOP/s (2*flop per second)", "value": 2 * head["flop"] / (head["linear_step_ms"] * 1e-3) / 1e9,
        "unit": "GFLOP/s", "n_gpus": 1, "steps": steps, "warmup": 1, "ms_per_step": head["linear_step_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "probing ablation: linear (Sec. 4.2.1) vs 4-slot chunks (Sec. 4.2.2), each with the "
                               "low-bits and the high-bits hash, on R-MAT16 A*A, "
                               "ER (R-MAT .25) scale 16 EF 16 A*A and triangle L*U of R-MAT16; FP64, sorted",
                   "l2": "256 MiB flush between steps", "timing": "median over steps"},
        "ablation": rows_out,
        "e2e": None,
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_numeric_repeat(args) -> int:
    """Repeated products of one structure with new values (as in multigrid
    setup): the whole product (plan, symbolic, numeric) against the numeric
    phase alone re-run on the same plan, and replayed as a CUDA graph
    (spgemm_numeric_graph).  FP64, sorted; values change between steps."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1804_01698_gb300 import binding as sg
    from paper_1804_01698_gb300 import inputs

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    cases = [("er4096_k8_f64", *inputs.workload("er4096_k8_f64")[:2]),
             ("amg_poisson7_g48_times_aggregation", inputs.poisson7(48), inputs.aggregation(48)),
             ("rmat16_ef16_f64", *inputs.workload("rmat16_ef16_f64")[:2])]
    steps = max(3, args.steps)
    rows, launches = [], 0

    def timed(fn):
        fn()
        ts = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    with ClockSampler(0) as clocks:
        for name, A, B in cases:
            dA = sg.to_device(A, dev)
            dB = dA if B is A else sg.to_device(B, dev)
            gen = torch.Generator(device=dev)
            gen.manual_seed(7)

            def new_values():
                dA.vals.uniform_(-1.0, 1.0, generator=gen)

            def whole():
                new_values()
                with sg.Plan(dA, dB, True, stream=stream) as p:
                    p.symbolic()
                    p.numeric()
            plan = sg.Plan(dA, dB, True, stream=stream)
            plan.symbolic()
            C = plan.numeric()

            def again():
                new_values()
                plan.numeric(C.col_idx, C.vals)

            def graph():
                new_values()
                plan.numeric_graph(C)
            t_whole, t_again, t_graph = timed(whole), timed(again), timed(graph)
            st = plan.stats()
            launches += st["kernel_launches"]
            flop = st["total_flop"]
            plan.destroy()
            rows.append({"workload": name, "flop": flop, "whole_product_ms": t_whole, "numeric_again_ms": t_again,
                         "numeric_graph_ms": t_graph, "graph_gflops": 2 * flop / (t_graph * 1e-3) / 1e9})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    head = rows[-1]
    line = {
        "metric": "SpGEMM GFLOP/s (2*flop per second)", "value": head["graph_gflops"], "unit": "GFLOP/s",
        "n_gpus": 1, "steps": steps, "warmup": 1, "ms_per_step": head["numeric_graph_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "repeated numeric phases of one structure with new A values: ER n=4096 k=8, AMG A*P "
                               "g=48, R-MAT16 A*A; FP64 sorted; whole product vs numeric re-run vs CUDA-graph replay",
                   "headline_point": "R-MAT16 graph replay", "l2": "inputs of R-MAT16 larger than L2",
                   "timing": "median over steps; each step includes drawing new values of A on the device"},
        "repeat": rows, "e2e": None, "gpu_launches": launches, "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------- GPU arm

def main() -> int:
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload.startswith("batch_"):
        return run_batch(args)
    if args.workload.startswith("serve_mix"):
        return run_serve(args)
    if args.workload == "sweep_rmat":
        return run_sweep(args)
    if args.workload == "ablate_probe":
        return run_ablate_probe(args)
    if args.workload == "numeric_repeat":
        return run_numeric_repeat(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        print(json.dumps({"error": f"--gpus {args.gpus} needs WORLD_SIZE={args.gpus} (torch.distributed.run)"}))
        return 2
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 2
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    import __graft_entry__
    __graft_entry__.build()
    from paper_1804_01698_gb300 import binding as sg
    from paper_1804_01698_gb300 import inputs
    from paper_1804_01698_gb300.shard import max_over_ranks

    A, B, sorted_default = inputs.workload(args.workload)
    sorted_output = sorted_default and not args.unsorted
    vdtype = {np.dtype(np.float64): torch.float64, np.dtype(np.float32): torch.float32,
              np.dtype(np.int64): torch.int64}[A.vals.dtype]
    vsize = A.vals.dtype.itemsize
    same = A is B
    dev = torch.device("cuda", local_rank)
    dA = sg.to_device(A, dev)
    dB = dA if same else sg.to_device(B, dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def step(sorted_flag: bool, timing: bool, marks=None):
        # timing=True records an event pair around every kernel and runs the
        # bins of each phase one after another (per-kernel durations alone);
        # `marks` (two events) are recorded after the plan and after the
        # symbolic phase, for the phases' spans in the concurrent step
        plan = sg.Plan(dA, dB, sorted_flag, stream=stream, timing=timing, serial=timing)
        if marks:
            marks[0].record(stream)
        nnz = plan.symbolic()
        if marks:
            marks[1].record(stream)
        C = plan.numeric()
        return plan, nnz, C

    def timed_steps(sorted_flag: bool, k: int, w: int, timing: bool = False):
        for _ in range(w):
            plan, nnz, C = step(sorted_flag, timing)
            plan.destroy()
            del C
        barrier()
        times, kt, launches, stats = [], {}, 0, None
        spans = []
        t_wall0 = time.perf_counter()
        for it in range(k):
            flush.fill_(it & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            marks = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
            e0.record(stream)
            plan, nnz, C = step(sorted_flag, timing, marks)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            spans.append((e0.elapsed_time(marks[0]), marks[0].elapsed_time(marks[1]), marks[1].elapsed_time(e1)))
            if timing:
                for name, (ms, n) in plan.kernel_times().items():
                    a, b = kt.get(name, (0.0, 0))
                    kt[name] = (a + ms, b + n)
            stats = plan.stats()
            if stats["status"] != 0:
                raise RuntimeError(f"device error status {stats['status']}")
            launches += stats["kernel_launches"]
            plan.destroy()
            del C
        barrier()
        wall = time.perf_counter() - t_wall0
        timed_steps.spans = spans
        return times, kt, launches, stats, nnz, wall

    with ClockSampler(local_rank) as clocks:
        times, _, launches, stats, nnz_c, wall = timed_steps(sorted_output, args.steps, args.warmup)
    clock_summary = clocks.summary()
    # spans of the phases inside the timed (concurrent) steps, each ending at
    # the host synchronisation that closes it
    sp = timed_steps.spans
    phase_wall = {name: round(sum(x[j] for x in sp) / len(sp), 4)
                  for j, name in enumerate(("plan (flop pass, bins; host reads the bin counts)",
                                            "symbolic (host reads nnz(C))", "numeric"))}
    # per-kernel durations: the same K steps again, bins serialised, an event pair per kernel
    ktimes, kt, _, _, _, _ = timed_steps(sorted_output, args.steps, 1, timing=True)

    total_ms = max_over_ranks(sum(times), world, dist if world > 1 else None, dev)
    acc = workload_accounting(A, B, nnz_c, vsize)
    flop = acc["flop"]
    ms_per_step = total_ms / args.steps
    value = world * args.steps * 2 * flop / (total_ms * 1e-3) / 1e9

    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    hbm_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or HBM_FALLBACK_GBS

    # dominant kernel and its roofline
    dom = max(kt.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms_total, dom_launches) = dom
    dom_ms = dom_ms_total / max(dom_launches, 1)
    units, phase = kernel_units(dom_name, stats)
    units_per_launch = units / max(dom_launches / args.steps, 1)
    if phase == "numeric" and vdtype == torch.float64:
        achieved = 2 * units_per_launch / (dom_ms * 1e-3) / 1e12
        roofline = {"kernel": dom_name, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2.07 GHz x 2",
                    "work_per_launch": f"{units_per_launch:.0f} multiply-adds (FP64 FMA)"}
    elif phase == "other":
        # a planning step: its algorithmic bytes (per launch of its scope)
        bytes_l, what = planning_bytes(dom_name, A, B, stats)
        achieved_b = bytes_l / (dom_ms * 1e-3) / 1e9
        roofline = {"kernel": dom_name, "bound": "hbm", "achieved": achieved_b, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved_b / hbm_peak, "peak_source": hbm_src, "work_per_launch": what}
    else:
        # bytes that kernel must move: the B entries it reads once per product
        # are L2 hits; its HBM share is bounded by its output and input rows.
        achieved_b = (units_per_launch * (4 + vsize)) / (dom_ms * 1e-3) / 1e9
        roofline = {"kernel": dom_name, "bound": "hbm", "achieved": achieved_b, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved_b / hbm_peak, "peak_source": hbm_src,
                    "work_per_launch": f"{units_per_launch:.0f} products x {4 + vsize} B"}
    roofline["launch_ms"] = dom_ms
    roofline["measured_in"] = (f"{args.steps} steps with the bins of each phase serialised and a CUDA event pair "
                               f"around every kernel on its stream ({sum(ktimes) / len(ktimes):.3f} ms/step)")
    roofline["traffic"] = committed_traffic(dom_name, args.workload)
    path_gbs = acc["bytes_alg"] / (ms_per_step * 1e-3) / 1e9
    hbm_roofline = {"bytes_alg": acc["bytes_alg"], "achieved_gbs": path_gbs, "peak_gbs": hbm_peak,
                    "frac": path_gbs / hbm_peak, "frac_of_8tbs": path_gbs / 8000.0, "peak_source": hbm_src}

    phases = {name: round(ms / args.steps, 4) for name, (ms, n) in sorted(kt.items(), key=lambda kv: -kv[1][0])}

    def phase_of(name):
        if name.startswith(("row_flop", "bin_rows_sym")):
            return "plan: flop pass and binning (Sec. 4.1)"
        if name.startswith(("sym_", "scan_", "num_classify", "bm_items_count")):
            return "symbolic: counts, row_ptr scan (Sec. 4.2.1)"
        return "numeric: accumulation and sort (Sec. 4.2.1)"
    phase_totals = {}
    for name, (ms, _) in kt.items():
        phase_totals[phase_of(name)] = phase_totals.get(phase_of(name), 0.0) + ms / args.steps
    phase_totals = {k: round(v, 4) for k, v in phase_totals.items()}
    kt_total = sum(ms for ms, _ in kt.values())
    shares = {name: round(ms / kt_total, 4) for name, (ms, n) in sorted(kt.items(), key=lambda kv: -kv[1][0])}

    # the autotuner's pick for this product (tuning runs untimed), then the
    # same K steps with it; the headline value stays the default plan's
    tuned = None
    if not args.no_variant:
        from paper_1804_01698_gb300.tune import _split, model_autotune
        t0 = time.perf_counter()
        best, table, model_meas = model_autotune(dA, dB, sorted_output, top=3, steps=2, stream=stream)
        tune_s = time.perf_counter() - t0
        kw, tuning = _split(best)
        tt = []
        for it in range(args.steps + 1):
            flush.fill_(it & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with sg.Plan(dA, dB, sorted_output, stream=stream, tuning=tuning, **kw) as tp:
                tp.symbolic()
                tC = tp.numeric()
            e1.record(stream)
            e1.synchronize()
            del tC
            if it > 0:
                tt.append(e0.elapsed_time(e1))
        tms = sum(tt) / len(tt)
        default_ms = next(ms for c, _, ms in table if c == {"long_row_min": 0})
        tuned = {"candidate": best, "ms_per_step": tms, "value": 2 * flop / (tms * 1e-3) / 1e9,
                 "autotune_seconds": tune_s, "candidates": len(table),
                 "model": {"kind": "Eq. 2: u[kind] * flop * c + bitmap word cost, calibrated on one default run",
                           "measured": model_meas,
                           "table": [{"candidate": c, "predicted_ms": round(pr, 4), "measured_ms": round(ms, 4)}
                                     for c, pr, ms in table]},
                 "gain_over_default": default_ms / min(ms for _, _, ms in table)}

    variant = None
    if not args.no_variant:
        vt, _, _, _, _, _ = timed_steps(not sorted_output, args.steps, 1)
        vms = sum(vt) / len(vt)
        variant = {"sorted": not sorted_output, "ms_per_step": vms, "value": 2 * flop / (vms * 1e-3) / 1e9}

    # end to end through the C entry point spgemm_host: operands in pinned
    # host memory, C written to a pinned host arena, every copy inside the
    # timed region (the copy of C overlaps the numeric phase block by block)
    e2e = None
    if not args.no_e2e:
        def pin(x):
            return torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        hA = inputs.CSR(A.nrows, A.ncols, pin(A.row_ptr), pin(A.col_idx), pin(A.vals))
        hB = hA if same else inputs.CSR(B.nrows, B.ncols, pin(B.row_ptr), pin(B.col_idx), pin(B.vals))
        arena = sg.HostArena(sg.HostArena.bytes_for(A.nrows, nnz_c, vsize))
        h2d = sum(t.numel() * t.element_size() for t in (hA.row_ptr, hA.col_idx, hA.vals)) + (0 if same else sum(
            t.numel() * t.element_size() for t in (hB.row_ptr, hB.col_idx, hB.vals)))
        d2h = (A.nrows + 1) * 4 + nnz_c * (4 + vsize)

        def e2e_step():
            arena.reset()
            C = sg.spgemm_host(hA, hB, sorted_output, row_blocks=args.row_blocks, arena=arena, stream=stream)
            if C.nnz != nnz_c:
                raise RuntimeError("end-to-end product differs in size from the device product")

        for _ in range(args.warmup):
            e2e_step()
        barrier()
        et = []
        for it in range(args.steps):
            flush.fill_(it & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            e2e_step()
            e1.record(stream)
            e1.synchronize()
            et.append(e0.elapsed_time(e1))
        barrier()
        ems = max_over_ranks(sum(et), world, dist if world > 1 else None, dev)
        e2e = {"value": world * args.steps * 2 * flop / (ems * 1e-3) / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ems / args.steps,
               "api": "spgemm_host", "row_blocks": args.row_blocks or "default"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        cores = len(os.sched_getaffinity(0))
        t0 = time.perf_counter()
        oracle.spgemm(A, B, nthreads=cores)
        dt = time.perf_counter() - t0
        cpu = {"value": 2 * flop / dt / 1e9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
               "sample": "the whole product once (dense-SPA Gustavson, rows split by RowsToThreads)",
               "seconds": dt}
        # the same oracle on one thread, and scipy's CSR product as a library
        # reference point (not the oracle; timed once each)
        t0 = time.perf_counter()
        oracle.spgemm(A, B, nthreads=1)
        dt1 = time.perf_counter() - t0
        cpu["single_thread"] = {"value": 2 * flop / dt1 / 1e9, "unit": "GFLOP/s", "cores": 1, "seconds": dt1}
        try:
            import scipy.sparse as sp
            sa = sp.csr_matrix((A.vals, A.col_idx, A.row_ptr), shape=(A.nrows, A.ncols))
            sb = sa if same else sp.csr_matrix((B.vals, B.col_idx, B.row_ptr), shape=(B.nrows, B.ncols))
            t0 = time.perf_counter()
            sc = sa @ sb
            if sorted_output:
                sc.sort_indices()
            dts = time.perf_counter() - t0
            cpu["scipy"] = {"value": 2 * flop / dts / 1e9, "unit": "GFLOP/s", "cores": 1, "seconds": dts,
                            "note": "scipy.sparse CSR product, a library reference point"}
        except ImportError:
            cpu["scipy"] = None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {torch.float64: "f64", torch.float32: "f32", torch.int64: "int64"}[vdtype],
            "data": "synthetic",
            "config": workload_config(args.workload, A, B, flop, nnz_c, sorted_output, world),
            "roofline": roofline,
            "hbm_roofline_path": hbm_roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches * world,
            "clocks": clock_summary,
            "phases_ms": phases,
            "phase_totals_ms": phase_totals,
            "phase_wall_ms": phase_wall,
            "ms_per_step_median": round(statistics.median(times), 4),
            "kernel_share": shares,
            "variant": variant,
            "tuned": tuned,
            "wall_s_timed_region": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
