"""ORACLE -- test infrastructure, not part of the library.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_2305_03317_b300``) and never imports it; the only module both sides
use is ``bcgen`` (seeded inputs, no centrality arithmetic).

Contents:
  * ``bc`` / ``bc_ld`` / ``source_detail`` -- plain single-threaded Brandes in
    double or long double (``brandes.c``), following the paper's computeBC
    (Appendix A, BC listing) with iterateInBFS / iterateInReverse semantics
    (Section 2.3.2): sigma summed over BFS-DAG predecessors, delta pulled from
    DAG successors in reverse BFS order as (sigma_v/sigma_w)(1+delta_w), and
    BC the raw sum of delta over the listed sources (source excluded).
  * ``brute_force_bc`` -- exact rational BC from explicit enumeration of every
    shortest path (tiny graphs only; undirected or directed, paths follow arcs);
    the definition
    BC(v) = sum_s sum_{t != s, v} sigma_st(v) / sigma_st written out.
  * ``sum_dm1`` -- per source, the sum of (d(s,t) - 1) over reached t != s, by
    breadth-first search alone (distances, no path counts; threads over
    sources): the sum of the raw BC over all vertices, at any graph size;
    ``sum_dm1_bits`` the same by bit-parallel search, 64 sources per pass.
  * ``relabel`` / ``validate`` -- the ingest rules (degree-descending stable
    relabelling; CSR validity) in their plain definitions.
  * ``wbc`` / ``wsource_detail`` -- weighted BC (positive integer arc
    weights, ``weighted.c``): the same accumulation over the shortest-path DAG
    of Dijkstra distances, vertices taken in (distance, id) order; and
    ``brute_force_wbc``, its exact rational definition by path enumeration
    over Bellman-Ford distances.
  * ``pagerank`` -- PageRank by its definition, the power iteration
    x <- (1 - delta)/n + delta P^T x with P = D^-1 A (``pagerank.c``), with
    the parameters and stopping rule of the paper's computePR (Appendix A):
    damping, an L1-change tolerance and an iteration cap; double precision.
Every function here is pinned by ``tests/test_oracle*.py`` against closed
forms, brute force and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from collections import deque
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brandes.c")
_SRCS = [_SRC, os.path.join(_HERE, "pagerank.c"), os.path.join(_HERE, "weighted.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class _Detail(ctypes.Structure):
    _fields_ = [("level", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("delta", ctypes.c_void_p),
                ("edag", ctypes.c_int64), ("reached", ctypes.c_int64), ("sum_dm1", ctypes.c_int64),
                ("max_level", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile brandes.c into liboracle.so (plain -O2; no fast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", tmp, *_SRCS, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            for name in ("oracle_bc_f64", "oracle_bc_ld"):
                f = getattr(lib, name)
                f.restype = ctypes.c_int
                f.argtypes = [i32, P, P, i32, P, P, P]
            lib.oracle_bc_ld_out_f64.restype = ctypes.c_int
            lib.oracle_bc_ld_out_f64.argtypes = [i32, P, P, i32, P, P]
            lib.oracle_source_ld.restype = ctypes.c_int
            lib.oracle_source_ld.argtypes = [i32, P, P, i32, P, P, P, P]
            lib.oracle_bc_f64_threads.restype = ctypes.c_int
            lib.oracle_bc_f64_threads.argtypes = [i32, P, P, i32, P, P, ctypes.c_int]
            lib.oracle_sum_dm1_threads.restype = ctypes.c_int
            lib.oracle_sum_dm1_threads.argtypes = [i32, P, P, i32, P, P, ctypes.c_int]
            lib.oracle_sum_dm1_bits.restype = ctypes.c_int
            lib.oracle_sum_dm1_bits.argtypes = [i32, P, P, i32, P, P, ctypes.c_int]
            lib.oracle_relabel.restype = None
            lib.oracle_relabel.argtypes = [i32, P, P, P, P, P, P]
            lib.oracle_validate_csr.restype = ctypes.c_int
            lib.oracle_validate_csr.argtypes = [i32, i64, P, P, ctypes.c_int]
            lib.oracle_wbc_f64.restype = ctypes.c_int
            lib.oracle_wbc_f64.argtypes = [i32, P, P, P, i32, P, P]
            lib.oracle_wsource.restype = ctypes.c_int
            lib.oracle_wsource.argtypes = [i32, P, P, P, i32, P, P, P]
            lib.oracle_pagerank.restype = ctypes.c_int
            lib.oracle_pagerank.argtypes = [i32, P, P, ctypes.c_double, ctypes.c_double, i32, P, P]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(off, adj):
    return (np.ascontiguousarray(off, dtype=np.int32), np.ascontiguousarray(adj, dtype=np.int32))


def bc(off, adj, sources, threads: int = 1) -> np.ndarray:
    """Raw BC (double) summed over ``sources`` (one entry per occurrence)."""
    off, adj = _csr(off, adj)
    src = np.ascontiguousarray(sources, dtype=np.int32)
    n = off.shape[0] - 1
    out = np.zeros(max(n, 1), dtype=np.float64)
    if threads > 1:
        rc = _L().oracle_bc_f64_threads(n, _p(off), _p(adj), src.shape[0], _p(src), _p(out), threads)
    else:
        rc = _L().oracle_bc_f64(n, _p(off), _p(adj), src.shape[0], _p(src), _p(out), None)
    if rc:
        raise ValueError(f"oracle rc={rc}")
    return out[:n]


def sum_dm1(off, adj, sources, threads: int = 1) -> np.ndarray:
    """Per source s: sum over the vertices t != s reached from s of (d(s,t) - 1), by BFS
    (int64).  Summed over a source list it equals the sum of the raw BC over all vertices."""
    off, adj = _csr(off, adj)
    src = np.ascontiguousarray(sources, dtype=np.int32)
    n = off.shape[0] - 1
    out = np.zeros(max(src.shape[0], 1), dtype=np.int64)
    rc = _L().oracle_sum_dm1_threads(n, _p(off), _p(adj), src.shape[0], _p(src), _p(out), max(1, threads))
    if rc:
        raise ValueError(f"oracle rc={rc}")
    return out[: src.shape[0]]


def sum_dm1_bits(off, adj, sources, threads: int = 1) -> np.ndarray:
    """sum_dm1 by bit-parallel breadth-first search, 64 sources per pass (for full-size graphs)."""
    off, adj = _csr(off, adj)
    src = np.ascontiguousarray(sources, dtype=np.int32)
    n = off.shape[0] - 1
    out = np.zeros(max(src.shape[0], 1), dtype=np.int64)
    rc = _L().oracle_sum_dm1_bits(n, _p(off), _p(adj), src.shape[0], _p(src), _p(out), max(1, threads))
    if rc:
        raise ValueError(f"oracle rc={rc}")
    return out[: src.shape[0]]


def bc_ld(off, adj, sources) -> np.ndarray:
    """Raw BC computed in long double (80-bit on x86-64), returned as np.longdouble."""
    off, adj = _csr(off, adj)
    src = np.ascontiguousarray(sources, dtype=np.int32)
    n = off.shape[0] - 1
    out = np.zeros(max(n, 1), dtype=np.longdouble)
    rc = _L().oracle_bc_ld(n, _p(off), _p(adj), src.shape[0], _p(src), _p(out), None)
    if rc:
        raise ValueError(f"oracle rc={rc}")
    return out[:n]


def wbc(off, adj, wt, sources) -> np.ndarray:
    """Raw weighted BC (double) over ``sources``; ``wt`` parallel to ``adj``, positive int32."""
    off, adj = _csr(off, adj)
    wt = np.ascontiguousarray(wt, dtype=np.int32)
    src = np.ascontiguousarray(sources, dtype=np.int32)
    n = off.shape[0] - 1
    out = np.zeros(max(n, 1), dtype=np.float64)
    rc = _L().oracle_wbc_f64(n, _p(off), _p(adj), _p(wt), src.shape[0], _p(src), _p(out))
    if rc:
        raise ValueError(f"oracle rc={rc}")
    return out[:n]


def wsource_detail(off, adj, wt, s: int) -> dict:
    """dist (int64, -1 unreached), sigma and delta of one source, weighted."""
    off, adj = _csr(off, adj)
    wt = np.ascontiguousarray(wt, dtype=np.int32)
    n = off.shape[0] - 1
    dist = np.empty(max(n, 1), np.int64)
    sigma = np.empty(max(n, 1), np.float64)
    delta = np.empty(max(n, 1), np.float64)
    rc = _L().oracle_wsource(n, _p(off), _p(adj), _p(wt), int(s), _p(dist), _p(sigma), _p(delta))
    if rc:
        raise ValueError(f"oracle rc={rc}")
    return {"dist": dist[:n], "sigma": sigma[:n], "delta": delta[:n]}


def source_detail(off, adj, s: int, long_double: bool = False) -> dict:
    """Levels, sigma, delta and counts for one source.

    Returns dict(level int32[n] (-1 unreachable), sigma, delta (float64 or
    longdouble), edag, reached, sum_dm1, max_level).
    """
    off, adj = _csr(off, adj)
    n = off.shape[0] - 1
    dt = np.longdouble if long_double else np.float64
    level = np.empty(max(n, 1), np.int32)
    sigma = np.empty(max(n, 1), dt)
    delta = np.empty(max(n, 1), dt)
    bcv = np.empty(max(n, 1), dt)
    d = _Detail(level.ctypes.data, sigma.ctypes.data, delta.ctypes.data, 0, 0, 0, 0)
    src = np.array([s], np.int32)
    f = _L().oracle_bc_ld if long_double else _L().oracle_bc_f64
    rc = f(n, _p(off), _p(adj), 1, _p(src), _p(bcv), ctypes.byref(d))
    if rc:
        raise ValueError(f"oracle rc={rc}")
    return dict(level=level[:n], sigma=sigma[:n], delta=delta[:n], edag=int(d.edag),
                reached=int(d.reached), sum_dm1=int(d.sum_dm1), max_level=int(d.max_level))


def source_sigma_split(off, adj, s: int):
    """Long-double levels / sigma as (mantissa in [0.5,1), exponent) / delta for one source."""
    off, adj = _csr(off, adj)
    n = off.shape[0] - 1
    level = np.empty(max(n, 1), np.int32)
    mant = np.empty(max(n, 1), np.float64)
    ex = np.empty(max(n, 1), np.int32)
    delta = np.empty(max(n, 1), np.float64)
    rc = _L().oracle_source_ld(n, _p(off), _p(adj), s, _p(level), _p(mant), _p(ex), _p(delta))
    if rc:
        raise ValueError(f"oracle rc={rc}")
    return level[:n], mant[:n], ex[:n], delta[:n]


def relabel(off, adj):
    """(perm, inv, new_off, new_adj): degree-descending, ties by id; rows sorted."""
    off, adj = _csr(off, adj)
    n = off.shape[0] - 1
    m = adj.shape[0]
    perm = np.empty(max(n, 1), np.int32)
    inv = np.empty(max(n, 1), np.int32)
    noff = np.empty(n + 1, np.int32)
    nadj = np.empty(max(m, 1), np.int32)
    _L().oracle_relabel(n, _p(off), _p(adj), _p(perm), _p(inv), _p(noff), _p(nadj))
    return perm[:n], inv[:n], noff, nadj[:m]


def pagerank(off, adj, delta: float = 0.85, beta: float = 1e-10, max_iter: int = 100):
    """PageRank by power iteration (pagerank.c): (ranks float64[n], iterations run, last L1 change)."""
    off, adj = _csr(off, adj)
    n = off.shape[0] - 1
    pr = np.zeros(max(n, 1), np.float64)
    diff = ctypes.c_double()
    it = _L().oracle_pagerank(n, _p(off), _p(adj), delta, beta, max_iter, _p(pr), ctypes.byref(diff))
    if it < 0:
        raise MemoryError("oracle_pagerank")
    return pr[:n], int(it), float(diff.value)


def validate(off, adj, undirected: bool = True) -> int:
    """0 if the CSR is valid, else a reason code (1 offsets, 2 range, 3 self-loop,
    4 duplicate, 5 asymmetric)."""
    off, adj = _csr(off, adj)
    n = off.shape[0] - 1
    return int(_L().oracle_validate_csr(n, adj.shape[0], _p(off), _p(adj), 1 if undirected else 0))


# ---------------------------------------------------------------------------
# Brute force: explicit enumeration of every shortest path (tiny graphs only).
# ---------------------------------------------------------------------------

def _bfs_dist(off, adj, s):
    n = len(off) - 1
    d = [-1] * n
    d[s] = 0
    q = deque([s])
    while q:
        v = q.popleft()
        for e in range(off[v], off[v + 1]):
            w = adj[e]
            if d[w] < 0:
                d[w] = d[v] + 1
                q.append(w)
    return d


def _reverse(off, adj):
    """CSR of the reversed arcs (the same graph when it is undirected)."""
    n = len(off) - 1
    rows = [[] for _ in range(n)]
    for v in range(n):
        for e in range(off[v], off[v + 1]):
            rows[adj[e]].append(v)
    roff, radj = [0], []
    for r in rows:
        radj.extend(sorted(r))
        roff.append(len(radj))
    return roff, radj


def shortest_paths(off, adj, s, t):
    """Every shortest s-t path (following arcs) as a tuple of vertices: DFS over
    the vertices w with d(s, w) + d(w, t) = d(s, t)."""
    off = [int(x) for x in off]
    adj = [int(x) for x in adj]
    ds = _bfs_dist(off, adj, s)
    if ds[t] < 0:
        return []
    roff, radj = _reverse(off, adj)
    dt = _bfs_dist(roff, radj, t)  # distance to t: BFS from t over reversed arcs
    out = []

    def walk(path):
        v = path[-1]
        if v == t:
            out.append(tuple(path))
            return
        for e in range(off[v], off[v + 1]):
            w = adj[e]
            if ds[w] == ds[v] + 1 and dt[w] == dt[v] - 1:
                path.append(w)
                walk(path)
                path.pop()

    walk([s])
    return out


def brute_force_bc(off, adj, sources):
    """Exact rational BC: sum over s in sources, t != s of (#paths through v)/(#paths)."""
    n = len(off) - 1
    res = [Fraction(0)] * n
    for s in sources:
        s = int(s)
        for t in range(n):
            if t == s:
                continue
            ps = shortest_paths(off, adj, s, t)
            if not ps:
                continue
            cnt = [0] * n
            for p in ps:
                for v in p[1:-1]:
                    cnt[v] += 1
            for v in range(n):
                if cnt[v]:
                    res[v] += Fraction(cnt[v], len(ps))
    return res


def brute_force_sigma(off, adj, s):
    """(level, sigma) for one source by explicit path enumeration."""
    n = len(off) - 1
    level = [-1] * n
    sigma = [0] * n
    for t in range(n):
        if t == s:
            level[t], sigma[t] = 0, 1
            continue
        ps = shortest_paths(off, adj, s, t)
        if ps:
            level[t] = len(ps[0]) - 1
            sigma[t] = len(ps)
    return level, sigma


def _bellman_ford(off, adj, wt, s):
    """Weighted distances from s by repeated relaxation of every arc (None = unreached)."""
    n = len(off) - 1
    d = [None] * n
    d[s] = 0
    for _ in range(n):
        changed = False
        for v in range(n):
            if d[v] is None:
                continue
            for e in range(off[v], off[v + 1]):
                x, c = adj[e], d[v] + wt[e]
                if d[x] is None or c < d[x]:
                    d[x] = c
                    changed = True
        if not changed:
            break
    return d


def weighted_shortest_paths(off, adj, wt, s, t):
    """Every minimum-weight s-t path (following arcs): DFS over arcs v -> x with
    d(s, v) + w = d(s, x) and d(x, t) = d(v, t) - w."""
    off = [int(x) for x in off]
    adj = [int(x) for x in adj]
    wt = [int(x) for x in wt]
    ds = _bellman_ford(off, adj, wt, s)
    if ds[t] is None:
        return []
    n = len(off) - 1
    rows = [[] for _ in range(n)]
    for v in range(n):
        for e in range(off[v], off[v + 1]):
            rows[adj[e]].append((v, wt[e]))
    roff, radj, rwt = [0], [], []
    for r in rows:
        for v, w in r:
            radj.append(v)
            rwt.append(w)
        roff.append(len(radj))
    dt = _bellman_ford(roff, radj, rwt, t)
    out = []

    def walk(path):
        v = path[-1]
        if v == t:
            out.append(tuple(path))
            return
        for e in range(off[v], off[v + 1]):
            x = adj[e]
            if ds[x] is not None and dt[x] is not None and ds[x] == ds[v] + wt[e] and dt[x] == dt[v] - wt[e]:
                path.append(x)
                walk(path)
                path.pop()

    walk([s])
    return out


def brute_force_wbc(off, adj, wt, sources):
    """Exact rational weighted BC: sum over s in sources, t != s of
    (#minimum-weight s-t paths through v) / (#minimum-weight s-t paths)."""
    n = len(off) - 1
    res = [Fraction(0)] * n
    for s in sources:
        s = int(s)
        for t in range(n):
            if t == s:
                continue
            ps = weighted_shortest_paths(off, adj, wt, s, t)
            if not ps:
                continue
            cnt = [0] * n
            for p in ps:
                for v in p[1:-1]:
                    cnt[v] += 1
            for v in range(n):
                if cnt[v]:
                    res[v] += Fraction(cnt[v], len(ps))
    return res
