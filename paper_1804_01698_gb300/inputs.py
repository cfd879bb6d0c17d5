"""Seeded synthetic CSR inputs shaped like the paper's workloads (Sec. 5.1, 5.5).

This module only builds input matrices. It holds none of the SpGEMM
arithmetic, so both the CUDA path and the CPU oracle may draw their inputs
from it without sharing any part of the method.

Randomness is counter based: every draw is SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
applied to a (seed, stream tag, counter) triple, so a given seed produces
the same matrix on any machine and in any order of evaluation.

Generators:
  * ``rmat``: R-MAT (Chakrabarti et al. 2004) with seed parameters
    (a, b, c, d); ER uses a=b=c=d=0.25, G500 uses 0.57/0.19/0.19/0.05
    (Sec. 5.1).  ``edge_factor * 2**scale`` edge samples, one uniform draw
    per recursion level, no noise, no vertex relabelling, self-loops kept,
    duplicates merged.
  * ``er_exact``: Erdos-Renyi rows with exactly ``k`` distinct uniformly
    random columns per row (Floyd's sampling algorithm).
  * ``frontier``: an n x f tall-skinny matrix whose column c holds
    r_c ~ U{lo..hi} distinct uniformly random rows (the stack of BFS
    frontiers of Sec. 5.5).
  * ``poisson7``/``aggregation``: the 3D 7-point Laplacian on a g^3 grid and
    the 2x2x2 aggregation prolongator (AMG-style A*P inputs).

Values are drawn per stored entry after duplicates are merged, indexed by
the entry's position in row-major sorted order.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream tags keep unrelated draws of one seed independent.
TAG_RMAT = 1
TAG_VALS = 2
TAG_ER = 3
TAG_FRONTIER_COUNT = 4
TAG_FRONTIER_ROWS = 5
TAG_SHUFFLE = 6
TAG_PERM = 7
TAG_BATCH = 8
TAG_ARRIVAL = 9
TAG_MIX = 10


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on uint64 arrays (wrapping arithmetic)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def draw_bits(seed: int, tag: int, counter: np.ndarray) -> np.ndarray:
    """64 random bits for each counter value of stream (seed, tag)."""
    with np.errstate(over="ignore"):
        key = splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(tag) * _GOLDEN))
        return splitmix64(key + np.asarray(counter, dtype=np.uint64))


def draw_unit(seed: int, tag: int, counter: np.ndarray) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1)."""
    bits = draw_bits(seed, tag, counter) >> np.uint64(11)
    return (bits.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


@dataclass
class CSR:
    """Host CSR matrix: int32 row_ptr/col_idx, values of any numpy dtype."""

    nrows: int
    ncols: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.nrows > 0 else 0

    def astype(self, dtype) -> "CSR":
        return CSR(self.nrows, self.ncols, self.row_ptr, self.col_idx, self.vals.astype(dtype))

    def with_vals(self, vals: np.ndarray) -> "CSR":
        return CSR(self.nrows, self.ncols, self.row_ptr, self.col_idx, vals)


def from_coo(nrows: int, ncols: int, rows: np.ndarray, cols: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Merge duplicate (row, col) pairs and return (row_ptr, col_idx), rows sorted by column."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    keys = np.unique(rows * np.int64(max(ncols, 1)) + cols)
    r = keys // max(ncols, 1)
    c = keys - r * max(ncols, 1)
    counts = np.bincount(r, minlength=nrows) if nrows > 0 else np.zeros(0, np.int64)
    row_ptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 indexing")
    return row_ptr.astype(np.int32), c.astype(np.int32)


def values(n: int, seed: int, kind: str) -> np.ndarray:
    """Per-entry values: 'uniform' doubles in (-1, 1), 'ones', or small 'ints' in [-8, 8]."""
    idx = np.arange(n, dtype=np.uint64)
    if kind == "uniform":
        return 2.0 * draw_unit(seed, TAG_VALS, idx) - 1.0
    if kind == "ones":
        return np.ones(n, dtype=np.float64)
    if kind == "ints":
        return (draw_bits(seed, TAG_VALS, idx) % np.uint64(17)).astype(np.int64) - 8
    raise ValueError(kind)


def _with_values(nrows, ncols, row_ptr, col_idx, seed, kind, dtype) -> CSR:
    v = values(len(col_idx), seed, kind).astype(dtype)
    return CSR(nrows, ncols, row_ptr, col_idx, v)


def rmat(scale: int, edge_factor: int, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 0,
         kind: str = "uniform", dtype=np.float64) -> CSR:
    """R-MAT 2^scale x 2^scale with edge_factor * 2^scale samples, duplicates merged (Sec. 5.1)."""
    a, b, c, _ = abcd
    n = 1 << scale
    ne = edge_factor * n
    rows = np.zeros(ne, dtype=np.int64)
    cols = np.zeros(ne, dtype=np.int64)
    e = np.arange(ne, dtype=np.uint64)
    ab, abc = a + b, a + b + c
    for level in range(scale):
        u = draw_unit(seed, TAG_RMAT, e * np.uint64(scale) + np.uint64(level))
        rbit = u >= ab
        cbit = ((u >= a) & (u < ab)) | (u >= abc)
        shift = scale - 1 - level
        rows |= rbit.astype(np.int64) << shift
        cols |= cbit.astype(np.int64) << shift
    row_ptr, col_idx = from_coo(n, n, rows, cols)
    return _with_values(n, n, row_ptr, col_idx, seed, kind, dtype)


def _floyd_rows(nrows: int, universe: np.ndarray, k: np.ndarray, seed: int, tag: int) -> np.ndarray:
    """Floyd's sampling: for each row r, k[r] distinct values in [0, universe[r]).

    Returns an (nrows, kmax) int64 array, padded with -1 past k[r].
    """
    kmax = int(k.max()) if nrows > 0 else 0
    out = np.full((nrows, kmax), -1, dtype=np.int64)
    ridx = np.arange(nrows, dtype=np.uint64)
    for it in range(kmax):
        active = k > it
        # j runs over universe-k .. universe-1 for each row.
        j = universe - k + it
        u = draw_unit(seed, tag, ridx * np.uint64(kmax) + np.uint64(it))
        t = np.minimum((u * (j + 1)).astype(np.int64), j)
        present = (out[:, :it] == t[:, None]).any(axis=1) if it > 0 else np.zeros(nrows, bool)
        pick = np.where(present, j, t)
        out[:, it] = np.where(active, pick, -1)
    return out


def er_exact(n: int, k: int, seed: int = 0, kind: str = "uniform", dtype=np.float64,
             ncols: int | None = None) -> CSR:
    """n x ncols matrix with exactly k distinct uniform random columns per row."""
    ncols = n if ncols is None else ncols
    if k > ncols:
        raise ValueError("k exceeds the column count")
    sel = _floyd_rows(n, np.full(n, ncols, np.int64), np.full(n, k, np.int64), seed, TAG_ER)
    sel.sort(axis=1)
    row_ptr = (np.arange(n + 1, dtype=np.int64) * k).astype(np.int32)
    return _with_values(n, ncols, row_ptr, sel.reshape(-1).astype(np.int32), seed, kind, dtype)


def frontier(n: int, f: int, lo: int = 1, hi: int = 4, seed: int = 0, kind: str = "ones",
             dtype=np.float32) -> CSR:
    """n x f frontier stack: column c holds r_c ~ U{lo..hi} distinct random rows (Sec. 5.5)."""
    cidx = np.arange(f, dtype=np.uint64)
    r = lo + np.minimum((draw_unit(seed, TAG_FRONTIER_COUNT, cidx) * (hi - lo + 1)).astype(np.int64), hi - lo)
    sel = _floyd_rows(f, np.full(f, n, np.int64), r, seed, TAG_FRONTIER_ROWS)
    cc = np.repeat(np.arange(f, dtype=np.int64), sel.shape[1]).reshape(sel.shape)
    mask = sel >= 0
    row_ptr, col_idx = from_coo(n, f, sel[mask], cc[mask])
    return _with_values(n, f, row_ptr, col_idx, seed, kind, dtype)


def poisson7(g: int, dtype=np.float64) -> CSR:
    """3D 7-point Laplacian on a g^3 grid: 6 on the diagonal, -1 to each grid neighbour."""
    n = g * g * g
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx % g, (idx // g) % g, idx // (g * g)
    rows, cols, vals = [idx], [idx], [np.full(n, 6.0)]
    for d, coord, step in ((0, x, 1), (1, y, g), (2, z, g * g)):
        for sgn in (-1, 1):
            ok = (coord + sgn >= 0) & (coord + sgn < g)
            rows.append(idx[ok])
            cols.append(idx[ok] + sgn * step)
            vals.append(np.full(int(ok.sum()), -1.0))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=row_ptr[1:])
    return CSR(n, n, row_ptr.astype(np.int32), c.astype(np.int32), v.astype(dtype))


def aggregation(g: int, dtype=np.float64) -> CSR:
    """2x2x2 aggregation prolongator from a g^3 grid to a ceil(g/2)^3 grid, values 1.0."""
    n = g * g * g
    gc = (g + 1) // 2
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx % g, (idx // g) % g, idx // (g * g)
    col = (x // 2) + (y // 2) * gc + (z // 2) * gc * gc
    row_ptr = np.arange(n + 1, dtype=np.int32)
    return CSR(n, gc ** 3, row_ptr, col.astype(np.int32), np.ones(n, dtype=dtype))


def shuffle_rows(m: CSR, seed: int) -> CSR:
    """Randomly permute the stored order inside every row (unsorted input, Sec. 5.1)."""
    nnz = m.nnz
    key = draw_bits(seed, TAG_SHUFFLE, np.arange(nnz, dtype=np.uint64))
    rowid = np.repeat(np.arange(m.nrows, dtype=np.int64), np.diff(m.row_ptr.astype(np.int64)))
    order = np.lexsort((key, rowid))
    return CSR(m.nrows, m.ncols, m.row_ptr, m.col_idx[order], m.vals[order])


def column_permutation(n: int, seed: int) -> np.ndarray:
    """A uniformly random permutation of range(n) (relabelling of columns)."""
    key = draw_bits(seed, TAG_PERM, np.arange(n, dtype=np.uint64))
    return np.argsort(key, kind="stable").astype(np.int32)


def relabel_columns(m: CSR, perm: np.ndarray) -> CSR:
    """Column j of the result is column perm^-1(j) of m, i.e. new col = perm[old col]."""
    return CSR(m.nrows, m.ncols, m.row_ptr, perm[m.col_idx].astype(np.int32), m.vals)


def batch_sizes(count: int, seed: int, n_lo: int = 256, n_hi: int = 65536, k_lo: int = 2, k_hi: int = 32):
    """Sizes of a batch of Erdos-Renyi products: n_i log-uniform in [n_lo, n_hi]
    and k_i (nonzeros per row) uniform in {k_lo..k_hi}, k_i <= n_i."""
    idx = np.arange(count, dtype=np.uint64)
    un = draw_unit(seed, TAG_BATCH, 2 * idx)
    uk = draw_unit(seed, TAG_BATCH, 2 * idx + np.uint64(1))
    n = np.floor(np.exp(np.log(n_lo) + un * (np.log(n_hi) - np.log(n_lo)))).astype(np.int64)
    n = np.clip(n, n_lo, n_hi)
    k = k_lo + np.minimum((uk * (k_hi - k_lo + 1)).astype(np.int64), k_hi - k_lo)
    return n, np.minimum(k, n)


def er_batch(count: int, seed: int, n_lo: int = 256, n_hi: int = 65536, k_lo: int = 2, k_hi: int = 32,
             kind: str = "uniform", dtype=np.float64) -> list:
    """`count` square Erdos-Renyi matrices with the sizes of batch_sizes (each
    with its own seed), for products A_i * A_i."""
    n, k = batch_sizes(count, seed, n_lo, n_hi, k_lo, k_hi)
    return [er_exact(int(n[i]), int(k[i]), seed=seed * 7919 + i + 1, kind=kind, dtype=dtype) for i in range(count)]


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    u = draw_unit(seed, TAG_ARRIVAL, np.arange(count, dtype=np.uint64))
    return np.cumsum(-np.log(u) / rate)


def serving_mix(count: int, seed: int, g_lo: int = 8, g_hi: int = 48, n_lo: int = 256, n_hi: int = 65536) -> list:
    """The serving mix: request i is, with probability 1/2 each, an
    Erdos-Renyi product A*A (sizes as er_batch) or an AMG-style product A*P
    (3D 7-point Poisson matrix on a g^3 grid, g uniform in {g_lo..g_hi}, times
    the 2x2x2 aggregation prolongator).  Returns a list of (A, B) pairs."""
    idx = np.arange(count, dtype=np.uint64)
    pick = draw_unit(seed, TAG_MIX, 2 * idx) < 0.5
    ug = draw_unit(seed, TAG_MIX, 2 * idx + np.uint64(1))
    g = g_lo + np.minimum((ug * (g_hi - g_lo + 1)).astype(np.int64), g_hi - g_lo)
    n, k = batch_sizes(count, seed, n_lo, n_hi)
    out = []
    for i in range(count):
        if pick[i]:
            a = er_exact(int(n[i]), int(k[i]), seed=seed * 7919 + i + 1)
            out.append((a, a))
        else:
            out.append((poisson7(int(g[i])), aggregation(int(g[i]))))
    return out


def undirected(m: CSR, dtype=np.float64) -> CSR:
    """Adjacency matrix of the undirected simple graph behind m's pattern:
    the pattern of m + m^T without the diagonal, values 1."""
    rows = np.repeat(np.arange(m.nrows, dtype=np.int64), np.diff(m.row_ptr))
    cols = m.col_idx.astype(np.int64)
    off = rows != cols
    r = np.concatenate([rows[off], cols[off]])
    c = np.concatenate([cols[off], rows[off]])
    rp, ci = from_coo(m.nrows, m.nrows, r, c)
    return CSR(m.nrows, m.nrows, rp, ci, np.ones(len(ci), dtype=dtype))


def degree_order(g: CSR) -> np.ndarray:
    """Vertices by increasing degree (ties by index): order[new] = old."""
    deg = np.diff(g.row_ptr)
    return np.lexsort((np.arange(g.nrows), deg)).astype(np.int64)


def permute_symmetric(g: CSR, order: np.ndarray) -> CSR:
    """P g P^T for the relabelling new = position of old in `order`."""
    new_of_old = np.empty(g.nrows, dtype=np.int64)
    new_of_old[order] = np.arange(g.nrows, dtype=np.int64)
    rows = new_of_old[np.repeat(np.arange(g.nrows, dtype=np.int64), np.diff(g.row_ptr))]
    cols = new_of_old[g.col_idx.astype(np.int64)]
    rp, ci = from_coo(g.nrows, g.nrows, rows, cols)
    return CSR(g.nrows, g.nrows, rp, ci, np.ones(len(ci), dtype=g.vals.dtype))


def triangular_split(g: CSR) -> tuple[CSR, CSR]:
    """(L, U): the strictly lower and strictly upper parts of g."""
    rows = np.repeat(np.arange(g.nrows, dtype=np.int64), np.diff(g.row_ptr))
    cols = g.col_idx.astype(np.int64)
    parts = []
    for keep in (cols < rows, cols > rows):
        rp, ci = from_coo(g.nrows, g.nrows, rows[keep], cols[keep])
        parts.append(CSR(g.nrows, g.nrows, rp, ci, np.ones(len(ci), dtype=g.vals.dtype)))
    return parts[0], parts[1]


def triangle_lu(scale: int, edge_factor: int, seed: int, dtype=np.float64) -> tuple[CSR, CSR, CSR]:
    """The triangle-counting product of Sec. 5.6 on an R-MAT graph: the
    undirected graph of R-MAT(scale, edge_factor), relabelled by increasing
    degree, split into strictly lower L and strictly upper U.  Returns
    (L, U, G) with G the relabelled adjacency matrix; (L*U)_ij counts the
    wedges i-k-j with k < min(i, j)."""
    g0 = undirected(rmat(scale, edge_factor, seed=seed, kind="ones"), dtype)
    g = permute_symmetric(g0, degree_order(g0))
    L, U = triangular_split(g)
    return L, U, g


# Workloads named by what they are, with their sizes.
WORKLOADS = {
    "er4096_k8_f64": dict(desc="Erdos-Renyi A*A, n=4096, 8 distinct columns per row, FP64 U(-1,1), sorted output"),
    "rmat16_ef16_f64": dict(desc="R-MAT A*A, scale 16, edge factor 16, (.57,.19,.19,.05), FP64 U(-1,1)"),
    "rmat18_frontier1024_f32": dict(desc="R-MAT scale 18 EF 16 (values 1.0) times an n x 1024 frontier stack (1-4 per column), FP32, unsorted"),
    "tc_rmat16_lu_f64": dict(desc="triangle counting L*U: undirected R-MAT scale 16 EF 16 graph ordered by increasing "
                                  "degree, strictly lower times strictly upper part, values 1.0 FP64, sorted output"),
}

SEED_BASE = 20180404


def workload(name: str, dtype=None):
    """Return (A, B, sorted_output) for a named workload."""
    if name == "er4096_k8_f64":
        a = er_exact(4096, 8, seed=SEED_BASE + 0, kind="uniform", dtype=dtype or np.float64)
        return a, a, True
    if name == "rmat16_ef16_f64":
        a = rmat(16, 16, seed=SEED_BASE + 1, kind="uniform", dtype=dtype or np.float64)
        return a, a, True
    if name == "rmat18_frontier1024_f32":
        dt = dtype or np.float32
        a = rmat(18, 16, seed=SEED_BASE + 2, kind="ones", dtype=dt)
        f = frontier(a.ncols, 1024, 1, 4, seed=SEED_BASE + 2, kind="ones", dtype=dt)
        return a, f, False
    if name == "tc_rmat16_lu_f64":
        L, U, _ = triangle_lu(16, 16, seed=SEED_BASE + 6, dtype=dtype or np.float64)
        return L, U, True
    raise KeyError(name)
