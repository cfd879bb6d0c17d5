"""Autotuner: picks a plan's tuning (spgemm_tuning) by timing candidates.

The decisions a plan exposes are the lanes that share one stored a_ik in
the block kernels' row loop (G), the symbolic bound above which rows take
the column-bitmap path, the hash probing (one slot or chunks of four per
probe) and the hash (low or high bits of the product); the better choices
depend on the input's collision factor.  Defaults come from rules measured on R-MAT
and ER products; `autotune` times a grid of candidates on the caller's own
product (or a sample batch) with CUDA events and returns the fastest.  The
result of a product does not depend on the tuning, only its time.
"""
from __future__ import annotations

import statistics

import numpy as np

import torch

from . import binding as sg

DEFAULT_GRID = [{"lanes_per_entry": g, "bitmap_min_bound": b, "probe": pr, "hash": h}
                for g in (0, 32) for b in (0, 512, 2048, -1) for pr in ("linear", "chunk4") for h in ("low", "high")]


def _split(candidate):
    """(plan keyword arguments: probe and hash schemes, spgemm_tuning dict) of a candidate."""
    t = dict(candidate)
    return {"probe": t.pop("probe", "linear"), "hash": t.pop("hash", "high")}, t


def _time(run, steps: int, stream) -> float:
    run()  # warm-up
    ts = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def autotune(A, B, sorted_output: bool = True, candidates=None, steps: int = 3, stream=None):
    """Times whole products (plan, symbolic, C allocation, numeric) of A*B
    for every candidate tuning; returns (best tuning, [(tuning, ms), ...])."""
    stream = stream if stream is not None else torch.cuda.current_stream(A.row_ptr.device)

    def run_with(t):
        kw, tuning = _split(t)

        def run():
            with sg.Plan(A, B, sorted_output, stream=stream, tuning=tuning, **kw) as p:
                p.symbolic()
                p.numeric()
        return run

    table = [(t, _time(run_with(t), steps, stream)) for t in (candidates or DEFAULT_GRID)]
    return min(table, key=lambda r: r[1])[0], table


def autotune_batch(As, Bs, sorted_output: bool = True, candidates=None, steps: int = 3, stream=None):
    """As autotune, for one packed batch of products (a sample of a larger
    stream of products of the same kind)."""
    stream = stream if stream is not None else torch.cuda.current_stream(As[0].row_ptr.device)

    def run_with(t):
        kw, tuning = _split(t)

        def run():
            with sg.Batch(As, Bs, sorted_output, stream=stream, tuning=tuning, **kw) as b:
                b.symbolic()
                b.numeric()
        return run

    table = [(t, _time(run_with(t), steps, stream)) for t in (candidates or DEFAULT_GRID)]
    return min(table, key=lambda r: r[1])[0], table


# ---------------------------------------------------------------------------
# Model-seeded tuning.  Sec. 4.2.4 (Eq. 2) prices hash SpGEMM as flop * c
# (c: probes per insertion, the collision factor) plus the sort term
# sum nnz(c_i) log nnz(c_i).  On the GPU every row goes to a kernel kind by
# its bin (warp or block hash tables, column bitmaps, global tables), so the
# model prices row i as u[kind] * flop_i * c[kind] (the sort of a hash row
# folded into its kind's unit cost, measured on the same output order) plus,
# for bitmap rows, a fixed cost per bitmap word.  One measured run of the
# default plan (kernel times, per-bin flop, the probe counters) calibrates
# u, w and c; the model then ranks a grid of bin thresholds and table loads
# by predicted time, and only the best few are timed.

# Kernel kinds of the model: per phase, hash tables in a warp or a block,
# column-bitmap rows in the library's size classes (symbolic: middle and
# heavy bounds; numeric: small, medium and large value arrays, the ranks of
# a large row beyond its array added straight into C), and global-memory
# tables.
SYM_KINDS = ("warp", "block", "bitmap_mid", "bitmap_heavy", "global")
NUM_KINDS = ("warp", "block", "bitmap_s", "bitmap_m", "bitmap_l", "global")
HASH_SLOTS = [64 << t for t in range(9)]       # warp tables 64..1024, block tables 2048..16384
BLOCK_SYM_MAX = 24576                          # 3/4 of the 32768-slot symbolic table
BITMAP_MAX_COLS = 1 << 18
MID_MAX = 24576
STATIC_SMEM = 256 * 24 + 2048                  # shared memory a bitmap block keeps for its static arrays
SMEM_BUDGETS = (72 * 1024, 110 * 1024, 232448)  # numeric bitmap classes: small, medium, large (1 block per SM)


def hash_caps(warp_load_pct: int = 0, block_load_pct: int = 0) -> list[int]:
    """Largest key bound of each hash bin (as the C library's rule)."""
    wp = warp_load_pct or 50
    bp = block_load_pct or 75
    return [s * (wp if t < 5 else bp) // 100 for t, s in enumerate(HASH_SLOTS)]


def bitmap_threshold(k: int, bitmap_min_bound: int = 0) -> int:
    """Rows whose symbolic bound exceeds this take column bitmaps (0: none)."""
    if k > BITMAP_MAX_COLS or bitmap_min_bound < 0:
        return 0
    if bitmap_min_bound > 0:
        return bitmap_min_bound
    return max(512, (k + 31) // 32 // 2)


def bitmap_caps(k: int, value_size: int = 8) -> list[int]:
    """Values per block of the numeric bitmap classes (as the library's rule)."""
    words = (k + 31) // 32
    return [max(0, (b - STATIC_SMEM - words * 8) // value_size // 256 * 256) for b in SMEM_BUDGETS]


def bin_kinds(flop, nnz, k: int, cand: dict, value_size: int = 8):
    """Kernel kind of every row in the symbolic phase (index into SYM_KINDS)
    and the numeric phase (NUM_KINDS) under a candidate tuning, -1 for rows
    without work, and the work items of every numeric row per part (1: a
    large bitmap row keeps its first ranks in shared memory and adds the
    others straight into C, in the same pass)."""
    flop = np.asarray(flop, dtype=np.int64)
    nnz = np.asarray(nnz, dtype=np.int64)
    caps = np.array(hash_caps(cand.get("warp_load_pct", 0), cand.get("block_load_pct", 0)), dtype=np.int64)
    bound = np.minimum(flop, k)
    thr = bitmap_threshold(k, cand.get("bitmap_min_bound", 0))
    t = np.searchsorted(caps, bound, side="left")          # first bin whose cap holds the bound
    sym = np.where(t < 5, 0, np.where(t < 9, 1, np.where(bound <= BLOCK_SYM_MAX, 1, 4)))
    bitmap = (thr > 0) & (bound > thr)
    sym = np.where(bitmap, np.where(bound > MID_MAX, 3, 2), sym)
    sym = np.where(bound <= 0, -1, sym)
    tn = np.searchsorted(caps, nnz, side="left")
    num = np.where(tn < 5, 0, np.where(tn < 9, 1, 5))
    bc = bitmap_caps(k, value_size)
    bm_cls = np.where(nnz <= bc[0], 2, np.where(nnz <= bc[1], 3, 4))
    num = np.where(bitmap, bm_cls, num)
    num = np.where((nnz <= 0) & ~bitmap, -1, num)
    windows = np.ones_like(nnz)
    return sym, num, windows


def linear_probe_cost(load: float) -> float:
    """Expected slots read by an insertion into a linear-probing table at this
    load (Knuth's successful-search estimate, 1/2 (1 + 1/(1 - load)))."""
    load = min(max(load, 0.0), 0.95)
    return 0.5 * (1.0 + 1.0 / (1.0 - load))


# kernel name prefix -> (phase, kind)
KERNEL_KIND = [("sym_warp", 0, 0), ("sym_block", 0, 1), ("sym_bitmap_mid", 0, 2), ("sym_bitmap_heavy", 0, 3),
               ("sym_global", 0, 4), ("num_warp", 1, 0), ("num_block", 1, 1), ("num_bitmap_s", 1, 2),
               ("num_bitmap_m", 1, 3), ("num_bitmap_l", 1, 4), ("num_global", 1, 5)]
HASH = ((0, 1, 4), (0, 1, 5))   # hash-table kinds per phase (their cost follows c)
BITMAP = ((2, 3), (2, 3, 4))    # bitmap kinds per phase (a cost per word as well)


def _work(flop, kinds, windows, nk):
    """Products (times windows) and rows (times windows) of every kind."""
    f = flop.astype(np.float64) * windows
    F = np.array([f[kinds == j].sum() for j in range(nk)])
    R = np.array([windows[kinds == j].sum() for j in range(nk)], dtype=np.float64)
    return F, R


def calibrate(kernel_ms: dict, flop, nnz, k: int, c_meas: tuple[float, float], cand: dict | None = None,
              value_size: int = 8) -> dict:
    """Unit costs per phase and kind (ms per product, divided by c for hash
    kinds) and the per-word cost of bitmap rows per phase, from the kernel
    times of one measured run of `cand` (default tuning if None).  The word
    cost is the least-squares slope over the bitmap classes of the phase."""
    cand = cand or {}
    sym, num, win = bin_kinds(flop, nnz, k, cand, value_size)
    flop = np.asarray(flop, dtype=np.int64)
    words = (k + 31) // 32
    nks = (len(SYM_KINDS), len(NUM_KINDS))
    t = [np.zeros(nks[0]), np.zeros(nks[1])]
    for name, ms in kernel_ms.items():
        for prefix, ph, kind in KERNEL_KIND:
            if name.startswith(prefix):
                t[ph][kind] += ms
                break
    u = [np.zeros(nks[0]), np.zeros(nks[1])]
    w = np.zeros(2)
    for ph, (kinds, wins) in enumerate(((sym, np.ones_like(sym)), (num, win))):
        F, R = _work(flop, kinds, wins, nks[ph])
        c = c_meas[ph] if c_meas[ph] > 0 else 1.0
        bm = [j for j in BITMAP[ph] if F[j] > 0 and t[ph][j] > 0]
        if len(bm) >= 2:   # t_j = u_j F_j + w R_j words: a common word cost, one product cost per class
            X = np.column_stack([F[bm] / F[bm].sum(), R[bm] * words / max(R[bm].sum() * words, 1)])
            sol, *_ = np.linalg.lstsq(X, t[ph][bm], rcond=None)
            w[ph] = max(0.0, float(sol[1])) / max(R[bm].sum() * words, 1)
        for j in range(nks[ph]):
            if F[j] > 0 and t[ph][j] > 0:
                rest = t[ph][j] - (w[ph] * R[j] * words if j in BITMAP[ph] else 0.0)
                rest = max(rest, 0.25 * t[ph][j])
                u[ph][j] = rest / (F[j] * (c if j in HASH[ph] else 1.0))
        # kinds the calibration run did not use: measured ratios to the block kind
        ref = u[ph][1] if u[ph][1] > 0 else max(u[ph].max(), 1e-9)
        for j in range(nks[ph]):
            if u[ph][j] == 0:
                u[ph][j] = ref * (1.2 if j == 0 else 2.0 if j in HASH[ph][2:] else 1.0 / 3.0 if j in BITMAP[ph]
                                  else 1.0)
    nnz = np.asarray(nnz, dtype=np.float64)
    hash_rows = (num == 0) | (num == 1)
    rho = float(nnz[hash_rows].sum() / max(np.minimum(flop[hash_rows], k).sum(), 1.0))
    return {"u": u, "w": w, "c": c_meas, "rho": rho, "words": words, "cand": dict(cand), "value_size": value_size}


def _kind_load(cand: dict, kind: int, rho: float) -> float:
    pct = (cand.get("warp_load_pct", 0) or 50) if kind == 0 else (cand.get("block_load_pct", 0) or 75)
    return pct / 100.0 * rho


def predict_ms(model: dict, flop, nnz, k: int, cand: dict) -> float:
    """Eq. 2 on the GPU: the sum over rows of u[kind] * flop_i * c[kind], plus
    the bitmap rows' word cost, under a candidate tuning."""
    sym, num, win = bin_kinds(flop, nnz, k, cand, model["value_size"])
    flop = np.asarray(flop, dtype=np.int64)
    u, w, rho = model["u"], model["w"], model["rho"]
    base = model["cand"]
    total = 0.0
    for ph, (kinds, wins) in enumerate(((sym, np.ones_like(sym)), (num, win))):
        c0 = model["c"][ph] if model["c"][ph] > 0 else 1.0
        F, R = _work(flop, kinds, wins, len(u[ph]))
        for j in range(len(u[ph])):
            if F[j] == 0:
                continue
            c = 1.0
            if j in (0, 1):  # shared hash tables: the collision factor follows the load
                c = c0 * linear_probe_cost(_kind_load(cand, j, rho)) / linear_probe_cost(_kind_load(base, j, rho))
            elif j in HASH[ph]:
                c = c0
            total += u[ph][j] * F[j] * c
            if j in BITMAP[ph]:
                total += w[ph] * R[j] * model["words"]
    return float(total)


MODEL_GRID = [{"bitmap_min_bound": b, "warp_load_pct": wl, "block_load_pct": bl}
              for b in (0, 256, 512, 1024, 2048, 4096, -1) for wl in (0, 30, 40, 65, 80)
              for bl in (0, 50, 60, 85, 95)]


def model_autotune(A, B, sorted_output: bool = True, top: int = 3, steps: int = 3, stream=None):
    """Calibrate the Eq. 2 model on the default plan (one run timing every
    kernel, one counting probes), rank MODEL_GRID by predicted time, then time
    the default and the `top` best predictions, each with and without long
    rows of B.  Returns (best candidate, [(candidate, predicted ms, measured
    ms)], measured collision factors)."""
    stream = stream if stream is not None else torch.cuda.current_stream(A.row_ptr.device)
    with sg.Plan(A, B, sorted_output, stream=stream, timing=True, serial=True) as p:
        p.symbolic()
        p.numeric()
        kt = {name: ms for name, (ms, n) in p.kernel_times().items()}
        flop = p.row_flop().cpu().numpy()
        nnz = p.row_nnz().cpu().numpy()
    with sg.Plan(A, B, sorted_output, stream=stream, count_probes=True) as p:
        p.symbolic()
        p.numeric()
        st = p.stats()
    c_sym = st["sym_probes"] / st["sym_inserts"] if st["sym_inserts"] else 1.0
    c_num = st["num_probes"] / st["num_inserts"] if st["num_inserts"] else 1.0
    k = B.ncols
    vs = A.vals.element_size()
    model = calibrate(kt, flop, nnz, k, (c_sym, c_num), value_size=vs)
    ranked = sorted(MODEL_GRID, key=lambda c: predict_ms(model, flop, nnz, k, c))
    default3 = {"bitmap_min_bound": 0, "warp_load_pct": 0, "block_load_pct": 0}
    picks = [{}] + [c for c in ranked if c != default3][:top]
    cands = []
    for c in picks:
        for lr in (0, -1):
            cands.append({**c, "long_row_min": lr})
    table = []
    for c in cands:
        kw, tuning = _split(c)

        def run(tuning=tuning, kw=kw):
            with sg.Plan(A, B, sorted_output, stream=stream, tuning=tuning, **kw) as q:
                q.symbolic()
                q.numeric()
        table.append((c, predict_ms(model, flop, nnz, k, {**default3, **c}), _time(run, steps, stream)))
    best = min(table, key=lambda r: r[2])[0]
    return best, table, {"c_sym": c_sym, "c_num": c_num, "rho": model["rho"]}
