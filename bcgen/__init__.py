"""Seeded synthetic inputs for betweenness-centrality workloads (int32 CSR).

This package produces graphs, source lists and request streams only; it holds
none of the centrality arithmetic.  Both the CPU oracle (``oracle/``) and the
CUDA library consume its output, so a parity test feeds both sides exactly the
same arrays.  The generators live in ``gen.c`` (compiled on first use with
gcc) and are described there: SplitMix64-finalised counter-based draws, R-MAT
(Chakrabarti et al. 2004) with the paper's a=.57 b=.19 c=.19 d=.05, a 2-D grid
with a seeded fraction of edges removed, and uniform source sampling without
replacement over vertices of degree >= 1.

Every CSR returned here is undirected and simple: both directions of each
edge, no self-loops, no duplicates, rows sorted ascending.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "libbcgen.so")
_lock = threading.Lock()
_lib = None

RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19


def build(force: bool = False) -> str:
    """Compile gen.c into libbcgen.so next to it (no-op when up to date)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            lib.bcg_mix64.restype = u64
            lib.bcg_mix64.argtypes = [u64]
            lib.bcg_draw.restype = u64
            lib.bcg_draw.argtypes = [u64, u64, u64]
            lib.bcg_unit.restype = f64
            lib.bcg_unit.argtypes = [u64, u64, u64]
            lib.bcg_units.restype = None
            lib.bcg_units.argtypes = [u64, u64, i64, i64, P]
            lib.bcg_rmat_edges.restype = None
            lib.bcg_rmat_edges.argtypes = [ctypes.c_int, i64, f64, f64, f64, u64, P, P]
            lib.bcg_random_perm.restype = None
            lib.bcg_random_perm.argtypes = [i64, u64, u64, P]
            lib.bcg_apply_perm.restype = None
            lib.bcg_apply_perm.argtypes = [i64, P, P, P]
            lib.bcg_edges_to_csr.restype = i64
            lib.bcg_edges_to_csr.argtypes = [i32, i64, P, P, P, P, P]
            lib.bcg_grid.restype = i64
            lib.bcg_grid.argtypes = [i32, i32, f64, u64, P, P]
            lib.bcg_sample_sources.restype = i32
            lib.bcg_sample_sources.argtypes = [i32, P, i32, u64, P]
            lib.bcg_gnp_edges.restype = i64
            lib.bcg_gnp_edges.argtypes = [i32, f64, u64, P, P, i64]
            lib.bcg_random_tree.restype = None
            lib.bcg_random_tree.argtypes = [i32, u64, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class CSR:
    """Simple graph in CSR form: ``off`` (n+1) and ``adj`` (m), int32.  Undirected
    (symmetric) unless built by ``directed_csr`` / ``orient`` (then out-adjacency)."""
    off: np.ndarray
    adj: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.adj.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.off.astype(np.int64))


def draw(seed: int, stream: int, t: int) -> int:
    return int(_L().bcg_draw(seed, stream, t))


def unit(seed: int, stream: int, t: int) -> float:
    return float(_L().bcg_unit(seed, stream, t))


def units(seed: int, stream: int, t0: int, count: int) -> np.ndarray:
    """unit(seed, stream, t0 + i) for i < count."""
    out = np.empty(max(count, 1), np.float64)
    _L().bcg_units(seed, stream, t0, count, _p(out))
    return out[:count]


def directed_csr(n: int, src, dst, name: str = "") -> CSR:
    """Out-adjacency CSR of the arcs (src[i] -> dst[i]): rows sorted, duplicates and
    self-loops dropped, no symmetrisation."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    key = np.unique(src[keep] * n + dst[keep])
    s, d = key // n, key % n
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, s + 1, 1)
    return CSR(np.cumsum(off).astype(np.int32), d.astype(np.int32), name)


def orient(g: CSR, seed: int = 1, p_both: float = 0.25) -> CSR:
    """A directed graph from an undirected one: each edge {u, v} (u < v, k-th in CSR
    order) keeps both arcs when r < p_both, else u -> v when r < (1 + p_both) / 2,
    else v -> u, with r = unit(seed, 9, k)."""
    deg = np.diff(g.off.astype(np.int64))
    row = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    col = g.adj.astype(np.int64)
    sel = row < col
    u, v = row[sel], col[sel]
    r = units(seed, 9, 0, int(u.shape[0]))
    both = r < p_both
    uv = both | (r < (1.0 + p_both) / 2.0)
    vu = both | ~uv
    return directed_csr(g.n, np.concatenate([u[uv], v[vu]]), np.concatenate([v[uv], u[vu]]),
                        f"orient({g.name}, {seed}, {p_both})")


def edges_to_csr(n: int, u, v, name: str = "") -> CSR:
    """Symmetrise, drop self-loops and duplicates, sort rows."""
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    ne = int(u.shape[0])
    off = np.zeros(n + 1, dtype=np.int32)
    adj = np.empty(max(2 * ne, 1), dtype=np.int32)
    pos = np.empty(n + 1, dtype=np.int64)
    m = _L().bcg_edges_to_csr(n, ne, _p(u), _p(v), _p(off), _p(adj), _p(pos))
    if m >= 2**31:
        raise ValueError("graph too large for int32 CSR")
    return CSR(off, adj[:m].copy(), name)


def rmat(scale: int, edge_factor: float, seed: int = 1, a: float = RMAT_A, b: float = RMAT_B,
         c: float = RMAT_C, permute: bool = True) -> CSR:
    """Undirected R-MAT graph: 2^scale vertices, edge_factor * 2^scale raw edges.

    After generation the vertex ids are relabelled by a seeded uniform random
    permutation (so that raw R-MAT's id/degree correlation is gone), then the
    edge list is symmetrised, self-loops and duplicates removed, rows sorted.
    """
    n = 1 << scale
    ne = int(round(edge_factor * n))
    L = _L()
    u = np.empty(ne, dtype=np.int32)
    v = np.empty(ne, dtype=np.int32)
    L.bcg_rmat_edges(scale, ne, a, b, c, seed, _p(u), _p(v))
    if permute:
        perm = np.empty(n, dtype=np.int32)
        L.bcg_random_perm(n, seed, 2, _p(perm))
        L.bcg_apply_perm(ne, _p(perm), _p(u), _p(v))
    return edges_to_csr(n, u, v, name=f"rmat{scale}_ef{edge_factor:g}_s{seed}")


def edge_weights(g: CSR, lo: int = 1, hi: int = 100, seed: int = 1, per_arc: bool = False) -> np.ndarray:
    """Positive int32 weights parallel to g.adj, uniform in [lo, hi] per
    undirected edge (both arcs of an edge get the same weight): a SplitMix64
    hash of (min(u, v), max(u, v), seed).  per_arc: per arc instead, a hash of
    (u, v, seed), so u -> v and v -> u differ (directed graphs)."""
    n = g.n
    deg = np.diff(g.off.astype(np.int64))
    u = np.repeat(np.arange(n, dtype=np.uint64), deg)
    v = g.adj.astype(np.uint64)
    a, b = (u, v) if per_arc else (np.minimum(u, v), np.maximum(u, v))
    with np.errstate(over="ignore"):
        z = a * np.uint64(n) + b + np.uint64(seed) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (np.uint64(lo) + z % np.uint64(hi - lo + 1)).astype(np.int32)


def grid(rows: int, cols: int, remove_frac: float = 0.0, seed: int = 1) -> CSR:
    """rows x cols 4-neighbour grid (id = r*cols + c) with round(remove_frac*E) edges removed."""
    n = rows * cols
    E = rows * (cols - 1) + (rows - 1) * cols
    off = np.zeros(n + 1, dtype=np.int32)
    adj = np.empty(max(2 * E, 1), dtype=np.int32)
    m = _L().bcg_grid(rows, cols, float(remove_frac), seed, _p(off), _p(adj))
    return CSR(off, adj[:m].copy(), f"grid{rows}x{cols}_rm{remove_frac:g}_s{seed}")


def sample_sources(g: CSR, k: int, seed: int = 1) -> np.ndarray:
    """k distinct sources, uniform over vertices of degree >= 1 (fewer if not enough)."""
    out = np.empty(max(k, 1), dtype=np.int32)
    off = np.ascontiguousarray(g.off, dtype=np.int32)
    got = _L().bcg_sample_sources(g.n, _p(off), k, seed, _p(out))
    return out[:got].copy()


def gnp(n: int, p: float, seed: int = 1) -> CSR:
    """Erdos-Renyi G(n, p)."""
    cap = max(n * (n - 1) // 2, 1)
    u = np.empty(cap, dtype=np.int32)
    v = np.empty(cap, dtype=np.int32)
    ne = _L().bcg_gnp_edges(n, float(p), seed, _p(u), _p(v), cap)
    return edges_to_csr(n, u[:ne], v[:ne], name=f"gnp{n}_p{p:g}_s{seed}")


def random_tree(n: int, seed: int = 1) -> CSR:
    """Uniform random labelled tree (random Pruefer sequence)."""
    if n == 1:
        return CSR(np.zeros(2, dtype=np.int32), np.zeros(0, dtype=np.int32), "tree1")
    u = np.empty(n - 1, dtype=np.int32)
    v = np.empty(n - 1, dtype=np.int32)
    _L().bcg_random_tree(n, seed, _p(u), _p(v))
    return edges_to_csr(n, u, v, name=f"tree{n}_s{seed}")


# ---- small deterministic families (closed-form shapes) ----

def path(n: int) -> CSR:
    i = np.arange(n - 1, dtype=np.int32)
    return edges_to_csr(n, i, i + 1, name=f"path{n}")


def star(n: int) -> CSR:
    """Centre 0, leaves 1..n-1."""
    i = np.arange(1, n, dtype=np.int32)
    return edges_to_csr(n, np.zeros_like(i), i, name=f"star{n}")


def cycle(n: int) -> CSR:
    i = np.arange(n, dtype=np.int32)
    return edges_to_csr(n, i, (i + 1) % n, name=f"cycle{n}")


def complete(n: int) -> CSR:
    iu, ju = np.triu_indices(n, 1)
    return edges_to_csr(n, iu.astype(np.int32), ju.astype(np.int32), name=f"K{n}")


def complete_bipartite(a: int, b: int) -> CSR:
    """Side A = 0..a-1, side B = a..a+b-1."""
    ii, jj = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return edges_to_csr(a + b, ii.ravel().astype(np.int32), jj.ravel().astype(np.int32),
                        name=f"K{a},{b}")


def disjoint_union(*gs: CSR) -> CSR:
    offs, adjs, base, abase = [np.zeros(1, dtype=np.int64)], [], 0, 0
    for g in gs:
        offs.append(g.off[1:].astype(np.int64) + abase)
        adjs.append(g.adj.astype(np.int64) + base)
        base += g.n
        abase += g.m
    off = np.concatenate(offs).astype(np.int32)
    adj = np.concatenate(adjs).astype(np.int32) if adjs else np.zeros(0, np.int32)
    return CSR(off, adj, "+".join(g.name for g in gs))


def empty_graph(n: int) -> CSR:
    return CSR(np.zeros(n + 1, dtype=np.int32), np.zeros(0, dtype=np.int32), f"empty{n}")


# ---- workloads ----

def rmat_sizes_pool(count: int, seed: int = 1, lo_log2: float = 10.0, hi_log2: float = 18.0,
                    ef_lo: int = 4, ef_hi: int = 32):
    """Sizes for a pool of uneven R-MAT graphs: n = round(2^U[lo,hi]), ef ~ U{ef_lo..ef_hi}.

    Returns a list of (n, edge_factor, graph_seed) with graph_seed = seed + i.
    """
    out = []
    for i in range(count):
        x = lo_log2 + (hi_log2 - lo_log2) * unit(seed, 7, 2 * i)
        n = int(round(2.0 ** x))
        ef = ef_lo + int(draw(seed, 7, 2 * i + 1) % (ef_hi - ef_lo + 1))
        out.append((n, ef, seed + i))
    return out


def rmat_n(n: int, edge_factor: float, seed: int) -> CSR:
    """R-MAT on the smallest power of two >= n, restricted to ids < n.

    Edges are drawn on 2^ceil(log2 n) vertices and then mapped to [0, n) by the
    seeded permutation; endpoints that land at or above n are dropped, so the
    graph keeps R-MAT's skew at any vertex count.
    """
    scale = max(1, int(math.ceil(math.log2(max(n, 2)))))
    N = 1 << scale
    ne = int(round(edge_factor * N))
    L = _L()
    u = np.empty(ne, dtype=np.int32)
    v = np.empty(ne, dtype=np.int32)
    L.bcg_rmat_edges(scale, ne, RMAT_A, RMAT_B, RMAT_C, seed, _p(u), _p(v))
    perm = np.empty(N, dtype=np.int32)
    L.bcg_random_perm(N, seed, 2, _p(perm))
    L.bcg_apply_perm(ne, _p(perm), _p(u), _p(v))
    keep = (u < n) & (v < n)
    return edges_to_csr(n, u[keep], v[keep], name=f"rmatn{n}_ef{edge_factor:g}_s{seed}")


def poisson_requests(rate: float, duration_s: float, n_graphs: int, seed: int = 1,
                     k_lo_log2: float = 0.0, k_hi_log2: float = 10.0):
    """Open-loop request stream: exponential inter-arrival times at ``rate`` req/s.

    Each request is (arrival_time_s, graph_index, k) with graph_index uniform
    over the pool and k = round(2^U[k_lo_log2, k_hi_log2]).
    """
    out, t, i = [], 0.0, 0
    while True:
        t += -math.log(1.0 - unit(seed, 8, 3 * i)) / rate
        if t >= duration_s:
            break
        gi = int(draw(seed, 8, 3 * i + 1) % n_graphs)
        k = int(round(2.0 ** (k_lo_log2 + (k_hi_log2 - k_lo_log2) * unit(seed, 8, 3 * i + 2))))
        out.append((t, gi, k))
        i += 1
    return out
