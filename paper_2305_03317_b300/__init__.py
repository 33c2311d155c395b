"""Python binding of libbc (exact Brandes betweenness centrality on one B300).

Argument marshalling only: every step of the computation runs in the CUDA
library ``libbc.so`` built from ``csrc/`` (see ``include/bc.h`` for the C ABI,
whose names this module mirrors).  PyTorch provides device memory for outputs
and the CUDA stream handles.  There is no fallback: if the library is missing
or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbc.so")

BC_OK = 0
BC_PENDING = 1
BC_W_SIGMA_INEXACT = 2
BC_E_INVALID_ARG = -1
BC_E_INVALID_GRAPH = -2
BC_E_SOURCE = -3
BC_E_NOMEM = -4
BC_E_TIMEOUT = -5
BC_E_CUDA = -6
BC_E_SIGMA_RANGE = -7
BC_E_LIMIT = -8
BC_E_BUSY = -9
BC_E_CANCELLED = -10

BC_UNDIRECTED = 1
BC_INPUT_ON_DEVICE = 2
BC_SKIP_VALIDATION = 4

_lib = None


class BCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status) if _lib else status}: {msg}")
        self.status = status


class bc_options(ctypes.Structure):
    _fields_ = [("batch_width", ctypes.c_int32), ("direction", ctypes.c_int32), ("alpha", ctypes.c_float),
                ("beta", ctypes.c_float), ("group_vertices", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("barrier_budget", ctypes.c_int64), ("trace", ctypes.c_int32), ("teams", ctypes.c_int32),
                ("dense_min", ctypes.c_int32), ("source_order", ctypes.c_int32),
                ("deep_form", ctypes.c_int32)]


class bc_run_stats(ctypes.Structure):
    _fields_ = [("batch_width", ctypes.c_int32), ("batches", ctypes.c_int32), ("max_levels", ctypes.c_int32),
                ("pull_levels", ctypes.c_int32), ("push_levels", ctypes.c_int32), ("ext_batches", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("kernel_ms", ctypes.c_float), ("teams", ctypes.c_int32), ("order_ms", ctypes.c_float),
                ("arcs_visited", ctypes.c_int64), ("rows_visited", ctypes.c_int64),
                ("mask_arcs", ctypes.c_int64), ("mask_lanes", ctypes.c_int64), ("dag_arcs", ctypes.c_int64),
                ("reached", ctypes.c_int64), ("deep_sources", ctypes.c_int32)]


class bc_item(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("sources", ctypes.c_void_p), ("nsrc", ctypes.c_int32),
                ("out_bc", ctypes.c_void_p)]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libbc.so and declare its signatures (raises if the file is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libbc.so not built ({path}); run python -m paper_2305_03317_b300.build")
    lib = ctypes.CDLL(path)
    P, i32, i64, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
    st = ctypes.c_int
    sig = {
        "bc_set_allocator": [P, P, P],
        "bc_graph_create": [P, P, i32, i64, u32, P, ctypes.POINTER(P)],
        "bc_graph_destroy": [P],
        "bc_graph_create_weighted": [P, P, P, i32, i64, u32, P, ctypes.POINTER(P)],
        "bc_compute_weighted": [P, P, i32, P, P],
        "bc_graph_info": [P, P, P, P, P],
        "bc_graph_export": [P, P, P, P],
        "bc_compute": [P, P, i32, P, P],
        "bc_compute_ex": [P, P, i32, P, P, ctypes.POINTER(bc_options)],
        "bc_bfs": [P, P, i32, P, P, P, P],
        "bc_pagerank": [P, ctypes.c_double, ctypes.c_double, i32, P, ctypes.POINTER(i32),
                        ctypes.POINTER(ctypes.c_double), P],
        "bc_last_run_stats": [P, ctypes.POINTER(bc_run_stats)],
        "bc_batch_submit": [P, P, i32, P, ctypes.POINTER(u64)],
        "bc_poll": [u64],
        "bc_poll_ex": [u64, ctypes.POINTER(ctypes.c_double)],
        "bc_wait": [u64, i64],
        "bc_wait_ex": [u64, i64, ctypes.POINTER(ctypes.c_double)],
        "bc_server_stats": [P, P],
        "bc_server_reset_stats": [],
        "bc_cancel": [u64],
        "bc_server_config": [i32, i64],
        "bc_team_rule": [i64, i32, i32, i32, u64, u64, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "bc_debug_source": [P, i32, P, P, P],
        "bc_last_trace": [P, P, i32, P],
        "bc_compute_noalloc": [P, P, i32, i64, P, i32, P, P],
        "bc_source_batches": [P, P, i32, ctypes.POINTER(bc_options), P, ctypes.POINTER(i32), P],
        "bc_reduce_ranks": [P, i32, i64, P, P],
        "bc_autotune": [P, P, i32, P, ctypes.POINTER(bc_options), ctypes.POINTER(ctypes.c_double)],
        "bc_tuning_cache": [ctypes.c_char_p, i32],
        "bc_many_create": [ctypes.POINTER(bc_item), i32, ctypes.POINTER(bc_options), P, ctypes.POINTER(P)],
        "bc_many_run": [P, P, P],
        "bc_many_destroy": [P],
        "bc_many_info": [P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = st
    lib.bc_status_string.argtypes = [st]
    lib.bc_status_string.restype = ctypes.c_char_p
    lib.bc_last_error.argtypes = []
    lib.bc_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def status_string(s: int) -> str:
    return load().bc_status_string(s).decode()


def last_error() -> str:
    return load().bc_last_error().decode()


def _check(s: int, allow=(BC_OK, BC_W_SIGMA_INEXACT)) -> int:
    if s not in allow:
        raise BCError(s, last_error())
    return s


def _ptr(x) -> int:
    """Data pointer of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def tuning_cache(path: str, save: bool) -> None:
    """Load or write the autotuner's settings (JSON)."""
    _check(load().bc_tuning_cache(path.encode(), 1 if save else 0))


def reduce_ranks(parts, out=None, stream=None):
    """out[v] = parts[0][v] + ... + parts[R-1][v] in rank order (bc_reduce_ranks); parts: [R][n] float64 cuda."""
    import torch
    R, n = int(parts.shape[0]), int(parts.shape[1])
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.float64, device=parts.device)[:n]
    parts = parts.contiguous()
    _check(load().bc_reduce_ranks(_ptr(parts) if n else None, R, n, _ptr(out) if n else None,
                                  _stream_handle(stream)))
    return out


def server_config(slots: int = 1, memory_budget: int = 0) -> None:
    _check(load().bc_server_config(slots, memory_budget))


def team_rule(m: int, batch_width: int, nbatch: int, blocks: int, team_bytes: int, free_bytes: int,
              teams: int = 0):
    """(teams, blocks per team) of a traversal (bc_team_rule: host arithmetic, no device work)."""
    T = ctypes.c_int32()
    B = ctypes.c_int32()
    _check(load().bc_team_rule(m, batch_width, nbatch, blocks, team_bytes, free_bytes, teams, ctypes.byref(T),
                               ctypes.byref(B)))
    return int(T.value), int(B.value)


def server_stats():
    peak = ctypes.c_int32()
    done = ctypes.c_int64()
    _check(load().bc_server_stats(ctypes.byref(peak), ctypes.byref(done)))
    return int(peak.value), int(done.value)


def server_reset_stats() -> None:
    _check(load().bc_server_reset_stats())


@dataclass
class Job:
    id: int
    graph: "Graph"
    out: object
    sources: np.ndarray

    def poll(self):
        """None while pending, else (status, latency_seconds)."""
        lat = ctypes.c_double()
        s = load().bc_poll_ex(self.id, ctypes.byref(lat))
        if s == BC_PENDING:
            return None
        _check(s)
        return s, float(lat.value)

    def wait(self, timeout_ms: int = -1):
        lat = ctypes.c_double()
        s = load().bc_wait_ex(self.id, timeout_ms, ctypes.byref(lat))
        if s == BC_PENDING:
            return None
        _check(s)
        return s, float(lat.value)

    def cancel(self) -> bool:
        """Withdraw the job if it is still queued (True); False when it already runs or ran."""
        s = load().bc_cancel(self.id)
        if s == BC_E_BUSY:
            return False
        _check(s)
        return True


class Graph:
    """A graph resident on the device (relabelled CSR; see bc_graph_create)."""

    def __init__(self, off, adj, validate: bool = True, stream=None, directed: bool = False, weights=None):
        """weights: positive int32 per arc, parallel to adj (rows sorted; equal on the two arcs of an
        undirected edge, free per arc when directed)."""
        lib = load()
        self._h = ctypes.c_void_p()
        flags = (0 if directed else BC_UNDIRECTED) | (0 if validate else BC_SKIP_VALIDATION)
        if isinstance(off, np.ndarray):
            off = np.ascontiguousarray(off, dtype=np.int32)
            adj = np.ascontiguousarray(adj, dtype=np.int32)
            if weights is not None:
                weights = np.ascontiguousarray(weights, dtype=np.int32)
            self._keep = (off, adj, weights)
            n, m = off.shape[0] - 1, adj.shape[0]
        else:  # torch tensors on the device
            flags |= BC_INPUT_ON_DEVICE
            n, m = off.numel() - 1, adj.numel()
            self._keep = (off, adj, weights)
        st = _stream_handle(stream) if _has_cuda() else 0
        if weights is None:
            _check(lib.bc_graph_create(_ptr(off), _ptr(adj) if m > 0 else None, n, m, flags, st,
                                       ctypes.byref(self._h)))
        else:
            _check(lib.bc_graph_create_weighted(_ptr(off), _ptr(adj) if m > 0 else None,
                                                _ptr(weights) if m > 0 else None, n, m, flags, st,
                                                ctypes.byref(self._h)))
        self.weighted = weights is not None
        self._keep = None
        n_, m_, md, nnz = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib.bc_graph_info(self._h, ctypes.byref(n_), ctypes.byref(m_), ctypes.byref(md), ctypes.byref(nnz)))
        self.n, self.m, self.max_degree, self.n_nonisolated = n_.value, m_.value, md.value, nnz.value

    def close(self):
        """Frees the device graph; BCError(BC_E_BUSY) while a plan or an unfinished job uses it."""
        if getattr(self, "_h", None):
            _check(load().bc_graph_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compute(self, sources, out=None, stream=None, batch_width: int = 0, direction: int = 0,
                alpha: float = 0.0, beta: float = 0.0, group_vertices: int = 0, blocks_per_sm: int = 0,
                barrier_budget: int = 0, trace: bool = False, teams: int = 0, dense_min: int = 0,
                source_order: int = 0, deep_form: int = 0):
        """BC over ``sources`` (host numpy or device int32 tensor). Returns (out, status)."""
        import torch
        if out is None:
            out = torch.empty(max(self.n, 1), dtype=torch.float64, device="cuda")[: self.n]
        if isinstance(sources, np.ndarray):
            sources = np.ascontiguousarray(sources, dtype=np.int32)
        nsrc = int(sources.shape[0]) if isinstance(sources, np.ndarray) else int(sources.numel())
        opt = bc_options(batch_width, direction, alpha, beta, group_vertices, blocks_per_sm, barrier_budget,
                         1 if trace else 0, teams, dense_min, source_order, deep_form)
        s = load().bc_compute_ex(self._h, _ptr(sources) if nsrc else None, nsrc, _ptr(out) if self.n else None,
                                 _stream_handle(stream), ctypes.byref(opt))
        _check(s)
        return out, s

    def source_batches(self, sources, stream=None, batch_width: int = 0, source_order: int = 0):
        """The order in which compute() would batch ``sources`` and its batch width: (order, K)."""
        if isinstance(sources, np.ndarray):
            sources = np.ascontiguousarray(sources, dtype=np.int32)
        nsrc = int(sources.shape[0]) if isinstance(sources, np.ndarray) else int(sources.numel())
        order = np.empty(max(nsrc, 1), np.int32)
        K = ctypes.c_int32()
        opt = bc_options()
        opt.batch_width, opt.source_order = batch_width, source_order
        _check(load().bc_source_batches(self._h, _ptr(sources) if nsrc else None, nsrc, ctypes.byref(opt),
                                        order.ctypes.data, ctypes.byref(K), _stream_handle(stream)))
        return order[:nsrc], K.value

    def compute_weighted(self, sources, out=None, stream=None):
        """Weighted BC over ``sources`` (host numpy or device int32 tensor). Returns (out, status)."""
        import torch
        if out is None:
            out = torch.empty(max(self.n, 1), dtype=torch.float64, device="cuda")[: self.n]
        if isinstance(sources, np.ndarray):
            sources = np.ascontiguousarray(sources, dtype=np.int32)
        nsrc = int(sources.shape[0]) if isinstance(sources, np.ndarray) else int(sources.numel())
        s = load().bc_compute_weighted(self._h, _ptr(sources) if nsrc else None, nsrc, _ptr(out) if self.n else None,
                                       _stream_handle(stream))
        _check(s)
        return out, s

    def autotune(self, sources, stream=None) -> dict:
        """Tune this graph's size bucket on a sample of ``sources`` (host); returns the chosen knobs."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        best = bc_options()
        rate = ctypes.c_double()
        _check(load().bc_autotune(self._h, src.ctypes.data, int(src.size), _stream_handle(stream), ctypes.byref(best),
                                  ctypes.byref(rate)))
        return {"batch_width": best.batch_width, "alpha": best.alpha, "group_vertices": best.group_vertices,
                "rate": rate.value}

    def stats(self) -> dict:
        st = bc_run_stats()
        _check(load().bc_last_run_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    TRACE_KINDS = {1: "init", 2: "pull", 3: "push", 4: "sigma", 5: "back", 6: "bc", 7: "prefix"}

    def trace(self):
        """Phase trace of the last compute(trace=True): list of (kind, level, t_ns)."""
        cap = 1 << 16
        buf = np.empty(2 * cap, np.int64)
        cnt = ctypes.c_int32()
        _check(load().bc_last_trace(self._h, buf.ctypes.data, cap, ctypes.byref(cnt)))
        out = []
        for i in range(cnt.value):
            tag, t = int(buf[2 * i]), int(buf[2 * i + 1])
            out.append((self.TRACE_KINDS.get(tag >> 24, str(tag >> 24)), tag & 0xFFFFFF, t))
        return out

    def export(self):
        perm = np.empty(max(self.n, 1), np.int32)
        off = np.empty(self.n + 1, np.int32)
        adj = np.empty(max(self.m, 1), np.int32)
        _check(load().bc_graph_export(self._h, perm.ctypes.data, off.ctypes.data, adj.ctypes.data))
        return perm[: self.n], off, adj[: self.m]

    def bfs(self, sources, sigma: bool = True, exponent: bool = False, stream=None):
        """Multi-source BFS (bc_bfs): level int32[nsrc][n] (-1 unreachable) and, when asked,
        path counts float64[nsrc][n] (with ``exponent``: mantissas and int32 exponents)."""
        import torch
        if isinstance(sources, np.ndarray):
            sources = np.ascontiguousarray(sources, dtype=np.int32)
        nsrc = int(sources.shape[0]) if isinstance(sources, np.ndarray) else int(sources.numel())
        shape = (nsrc, self.n)
        lev = torch.empty(shape, dtype=torch.int32, device="cuda")
        sg = torch.empty(shape, dtype=torch.float64, device="cuda") if sigma else None
        ex = torch.empty(shape, dtype=torch.int32, device="cuda") if (sigma and exponent) else None
        s = load().bc_bfs(self._h, _ptr(sources) if nsrc else None, nsrc, _ptr(lev) if lev.numel() else None,
                          _ptr(sg) if sg is not None and sg.numel() else None,
                          _ptr(ex) if ex is not None and ex.numel() else None, _stream_handle(stream))
        _check(s)
        return lev, sg, ex, s

    def pagerank(self, delta: float = 0.85, beta: float = 1e-10, max_iter: int = 100, out=None, stream=None):
        """The paper's computePR (bc_pagerank): (ranks float64[n] on the device, sweeps run, last L1 change)."""
        import torch
        if out is None:
            out = torch.empty(max(self.n, 1), dtype=torch.float64, device="cuda")[: self.n]
        it = ctypes.c_int32()
        diff = ctypes.c_double()
        _check(load().bc_pagerank(self._h, float(delta), float(beta), int(max_iter), _ptr(out) if self.n else None,
                                  ctypes.byref(it), ctypes.byref(diff), _stream_handle(stream)))
        return out, int(it.value), float(diff.value)

    def debug_source(self, s: int):
        """(level int32[n], sigma_mant float64[n], sigma_exp int32[n]) for one source."""
        lev = np.empty(max(self.n, 1), np.int32)
        mant = np.empty(max(self.n, 1), np.float64)
        ex = np.empty(max(self.n, 1), np.int32)
        r = load().bc_debug_source(self._h, int(s), lev.ctypes.data, mant.ctypes.data, ex.ctypes.data)
        _check(r)
        return lev[: self.n], mant[: self.n], ex[: self.n], r

    def submit(self, sources, out) -> Job:
        """Queue a serving job (host sources); ``out`` is a device float64 tensor of n."""
        src = np.ascontiguousarray(sources, dtype=np.int32)
        jid = ctypes.c_uint64()
        _check(load().bc_batch_submit(self._h, src.ctypes.data if src.size else None, int(src.size),
                                      _ptr(out) if self.n else None, ctypes.byref(jid)))
        return Job(int(jid.value), self, out, src)


class ManyPlan:
    """Many (graph, sources, output) items recorded once into a CUDA graph (bc_many_create)."""

    def __init__(self, items, stream=None, **opts):
        """items: list of (Graph, host int32 sources, device float64 output tensor)."""
        lib = load()
        self._keep = [(g, np.ascontiguousarray(s, dtype=np.int32), o) for g, s, o in items]
        arr = (bc_item * max(len(items), 1))()
        for i, (g, s, o) in enumerate(self._keep):
            arr[i] = bc_item(g._h, s.ctypes.data if s.size else None, int(s.size), _ptr(o) if g.n else None)
        opt = bc_options(opts.get("batch_width", 0), opts.get("direction", 0), 0.0, 0.0, 0, opts.get("blocks_per_sm", 0),
                         0, 0, opts.get("teams", 0), 0, opts.get("source_order", 0), opts.get("deep_form", 0))
        self._h = ctypes.c_void_p()
        _check(lib.bc_many_create(arr, len(items), ctypes.byref(opt), _stream_handle(stream), ctypes.byref(self._h)))

    def run(self, stream=None):
        """Replay; returns the per-item statuses."""
        st = np.zeros(max(len(self._keep), 1), np.int32)
        _check(load().bc_many_run(self._h, _stream_handle(stream), st.ctypes.data))
        return st[: len(self._keep)]

    def info(self):
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(load().bc_many_info(self._h, ctypes.byref(a), ctypes.byref(b)))
        return {"items": a.value, "kernel_launches": b.value}

    def close(self):
        if getattr(self, "_h", None):
            load().bc_many_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _has_cuda() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


__all__ = ["Graph", "Job", "ManyPlan", "BCError", "load", "status_string", "last_error", "server_config", "server_stats"]
