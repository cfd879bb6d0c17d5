"""Continuous-batching server for SpGEMM requests.

Requests (C = A*B with A and B already resident on the device) arrive over
time.  The server loop, on one host thread:

  1. polls the batches running on the device and retires the finished ones
     (their memory is released and each request's latency is recorded);
  2. takes the requests that have arrived, up to `max_batch` and within a
     memory bound taken before the symbolic pass (nnz(C) <= flop), and
     prepares them as one batch: packing, flop pass and symbolic pass
     (spgemm_batch_*), which gives the exact output size;
  3. admits the prepared batch when its exact memory (packed inputs, plan
     workspace and C) fits under `mem_cap` next to the batches in flight,
     and launches its numeric phase asynchronously on its own stream.  A
     batch whose exact memory alone exceeds the cap is given back and
     prepared again with half as many requests.

Requests that arrive while earlier batches run on the GPU are prepared and
launched on other streams, so their work overlaps on the device.  The
one-call-per-product baseline (`serve_one_by_one`) handles each request
alone, in arrival order, on one stream.

The device work goes through a backend; `GpuBackend` uses the library's
batch API, and tests of the scheduling logic use a fake backend on the CPU.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    A: object            # DeviceCSR (or anything the backend understands)
    B: object
    arrival: float       # seconds after the start of the run
    flop: int            # sum over stored a_ik of nnz(b_k*): bounds nnz(C)


@dataclass
class Completion:
    rid: int
    arrival: float
    start: float         # when its batch was launched
    done: float          # when the server saw its batch finish
    batch: int
    result: object = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class Stats:
    completions: list = field(default_factory=list)
    batches: int = 0
    peak_mem: int = 0
    wall: float = 0.0

    def latencies(self):
        return sorted(c.latency for c in self.completions)

    def percentile(self, q: float) -> float:
        lat = self.latencies()
        if not lat:
            return float("nan")
        idx = min(len(lat) - 1, max(0, int(round(q / 100.0 * (len(lat) - 1)))))
        return lat[idx]

    def solves_per_s(self) -> float:
        return len(self.completions) / self.wall if self.wall > 0 else float("nan")

    def summary(self) -> dict:
        return {"requests": len(self.completions), "batches": self.batches, "wall_s": self.wall,
                "solves_per_s": self.solves_per_s(), "p50_ms": 1e3 * self.percentile(50),
                "p99_ms": 1e3 * self.percentile(99), "peak_mem_bytes": self.peak_mem}


def upper_bound_bytes(req: Request, vsize: int = 8) -> int:
    """Memory of a request before its symbolic pass: nnz(C) <= flop."""
    rows = getattr(req.A, "nrows", 0)
    nnz_a = getattr(req.A, "nnz", 0)
    nnz_b = getattr(req.B, "nnz", 0)
    return (rows + 1) * 4 + req.flop * (4 + vsize) + (nnz_a + nnz_b) * (4 + vsize) + rows * 32


class Server:
    def __init__(self, backend, mem_cap: int = 40 << 30, max_batch: int = 64, max_inflight: int = 3):
        self.backend = backend
        self.mem_cap = mem_cap
        self.max_batch = max_batch
        self.max_inflight = max_inflight

    def run(self, requests, keep_results: bool = False, clock=time.perf_counter) -> Stats:
        reqs = sorted(requests, key=lambda r: r.arrival)
        stats = Stats()
        t0 = clock()
        nxt = 0                  # next request not yet arrived
        pending = []             # arrived, not prepared
        prepared = None          # (handle, reqs) waiting for memory
        inflight = []            # (handle, reqs, start, bytes)
        used = 0
        limit = self.max_batch   # requests per batch, halved after an oversized one

        def now():
            return clock() - t0

        while nxt < len(reqs) or pending or prepared is not None or inflight:
            # 1. retire finished batches
            still = []
            for h, rs, start, nbytes in inflight:
                if self.backend.done(h):
                    t = now()
                    results = self.backend.results(h) if keep_results else [None] * len(rs)
                    for r, res in zip(rs, results):
                        stats.completions.append(Completion(r.rid, r.arrival, start, t, stats.batches, res))
                    self.backend.release(h)
                    used -= nbytes
                else:
                    still.append((h, rs, start, nbytes))
            inflight = still
            # arrivals
            t = now()
            while nxt < len(reqs) and reqs[nxt].arrival <= t:
                pending.append(reqs[nxt])
                nxt += 1
            # 2. prepare the next batch from the arrived requests
            if prepared is None and pending and len(inflight) < self.max_inflight:
                take, bound = [], 0
                for r in pending:
                    ub = upper_bound_bytes(r, self.backend.vsize)
                    if take and (len(take) >= limit or bound + ub > self.mem_cap):
                        break
                    take.append(r)
                    bound += ub
                pending = pending[len(take):]
                h = self.backend.prepare(take)
                prepared = (h, take, self.backend.bytes(h))
                if prepared[2] > self.mem_cap and len(take) > 1:
                    # the workspace made the batch larger than the cap on its
                    # own: give it back and prepare half as many requests
                    self.backend.release(h)
                    pending = take + pending
                    limit = max(1, len(take) // 2)
                    prepared = None
                    continue
            # 3. admit and launch when its exact memory fits (a batch larger
            #    than the cap, of one request, runs when nothing else does)
            if prepared is not None:
                h, rs, nbytes = prepared
                if not inflight or used + nbytes <= self.mem_cap:
                    limit = self.max_batch
                    start = now()
                    self.backend.launch(h)
                    inflight.append((h, rs, start, nbytes))
                    used += nbytes
                    stats.peak_mem = max(stats.peak_mem, used)
                    stats.batches += 1
                    prepared = None
                    continue
            if not pending and prepared is None and nxt < len(reqs) and not inflight:
                # idle until the next arrival
                wait = reqs[nxt].arrival - now()
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        stats.wall = now()
        return stats


def serve_one_by_one(backend, requests, keep_results: bool = False, clock=time.perf_counter) -> Stats:
    """Baseline: every request alone, in arrival order, one after the other."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    stats = Stats()
    t0 = clock()
    for r in reqs:
        t = clock() - t0
        if r.arrival > t:
            time.sleep(r.arrival - t)
        start = clock() - t0
        h = backend.prepare([r])
        backend.launch(h)
        backend.wait(h)
        done = clock() - t0
        res = backend.results(h) if keep_results else [None]
        stats.completions.append(Completion(r.rid, r.arrival, start, done, stats.batches, res[0]))
        stats.peak_mem = max(stats.peak_mem, backend.bytes(h))
        backend.release(h)
        stats.batches += 1
    stats.wall = clock() - t0
    return stats


class GpuBackend:
    """Runs request batches through the library on a pool of CUDA streams:
    a batch of several requests uses the batch API (one packed plan), a
    single request the plain plan API (the one-call-per-product path).
    Each prepared batch takes a stream no other live batch holds, so its
    symbolic pass (which waits for its own stream) never waits for another
    batch's numeric phase."""

    def __init__(self, sorted_output: bool = True, nstreams: int = 4, device=None):
        import torch

        from . import binding as sg
        self.torch, self.sg = torch, sg
        self.sorted = sorted_output
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.free = [torch.cuda.Stream(device=self.device) for _ in range(nstreams)]
        self.vsize = 8
        self.kernel_launches = 0

    def prepare(self, reqs):
        torch, sg = self.torch, self.sg
        s = self.free.pop() if self.free else torch.cuda.Stream(device=self.device)
        self.vsize = reqs[0].A.vals.element_size()
        with torch.cuda.stream(s):
            if len(reqs) == 1:
                work = sg.Plan(reqs[0].A, reqs[0].B, self.sorted, stream=s)
            else:
                work = sg.Batch([r.A for r in reqs], [r.B for r in reqs], self.sorted, stream=s)
            work.symbolic()
        return {"work": work, "stream": s, "n": len(reqs), "event": None, "out": None}

    def bytes(self, h) -> int:
        w = h["work"]
        nnz = w.nnz_c
        rows = w.c_row_ptr.numel()
        # a batch also holds its packed copies of the operands
        packed = 0 if h["n"] == 1 else sum(a.nnz + b.nnz for a, b in zip(w.As, w.Bs)) * (4 + self.vsize)
        return w.workspace_bytes() + packed + rows * 4 + nnz * (4 + self.vsize)

    def launch(self, h):
        torch = self.torch
        s = h["stream"]
        with torch.cuda.stream(s):
            h["out"] = h["work"].numeric()
            ev = torch.cuda.Event()
            ev.record(s)
        h["event"] = ev

    def done(self, h) -> bool:
        return h["event"].query()

    def wait(self, h):
        h["event"].synchronize()

    def results(self, h):
        """The batch's products, for use on the caller's current stream (the
        batch ran on its own stream, whose memory pool must not reuse the
        results while the caller still works on them)."""
        w = h["work"]
        if h["n"] == 1:
            C = h["out"]
            self.sg.hand_over(h["stream"], C.row_ptr, C.col_idx, C.vals)
            return [C]
        rp = w.c_row_ptr.cpu().numpy()
        return [w.product(p, rp) for p in range(h["n"])]

    def release(self, h):
        w = h["work"]
        if h["event"] is not None:
            st = w.stats() if h["n"] == 1 else w.plan_stats()
            self.kernel_launches += st["kernel_launches"] + (2 if h["n"] > 1 else 0)   # + pack, unpack
        w.destroy()
        h["out"] = None
        self.free.append(h["stream"])
