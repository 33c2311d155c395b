"""The allocation-free entry point, bc_compute_noalloc, through the C ABI.

It serves callers that may not allocate device memory themselves -- host code
whose framework owns the whole device through its own memory pool and
forbids other allocations, or latency-critical code that must stay out of the
CUDA allocator -- by keeping every intermediate in one static device array.

Checked here, each against the CPU oracle (and the first against the regular
entry point, bc_compute, too), at the parity tolerance of the other GPU tests:
  * two calls in a row with different sources (the shared array keeps the
    previous call's contents, so the second call shows that each call starts
    clean);
  * rows above 1024 arcs (this entry point sums rows whole);
  * path counts beyond 2^64, which send every batch to the extended-range rerun;
  * a row that repeats one arc 140,000 times: its sums stay below 2^64 only
    because the longest row, not the vertex count, bounds the terms;
  * more than 65,536 sources (several launches adding into one output);
  * bad offsets, indices and sources, refused with their status and followed by
    a good call; a graph beyond the fixed capacity, refused before device work.
The file sorts last so that a stop-at-first-failure run has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import bcgen
import oracle

pytestmark = pytest.mark.gpu

REL = 1e-9  # same per-vertex relative tolerance as tests/test_gpu_parity.py


@pytest.fixture(scope="module")
def bc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_03317_b300 as m
    m.load()
    return m


def close(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    zero = want == 0
    assert np.all(got[zero] == 0)
    rel = np.abs(got[~zero] - want[~zero]) / np.abs(want[~zero])
    assert rel.max() <= REL, rel.max()


def noalloc(bc, off, adj, src, n=None, m=None):
    """One bc_compute_noalloc call on device copies of the inputs: (status, BC on the host)."""
    import torch
    lib = bc.load()
    n = len(off) - 1 if n is None else n
    m = len(adj) if m is None else m
    d_off = torch.from_numpy(np.ascontiguousarray(off, dtype=np.int32)).cuda()
    d_adj = torch.from_numpy(np.ascontiguousarray(adj, dtype=np.int32)).cuda()
    d_src = torch.from_numpy(np.ascontiguousarray(src, dtype=np.int32)).cuda()
    out = torch.full((max(n, 1),), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.bc_compute_noalloc(d_off.data_ptr(), d_adj.data_ptr(), n, m, d_src.data_ptr(), len(src),
                                out.data_ptr(), ctypes.c_void_p(stream))
    return st, out.cpu().numpy()[:n]


def csr_from_arcs(n, u, v):
    """CSR of the arc list (u[i] -> v[i]), rows sorted, repeated arcs kept."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    order = np.lexsort((v, u))
    off = np.zeros(n + 1, dtype=np.int32)
    np.add.at(off, u + 1, 1)
    return np.cumsum(off).astype(np.int32), v[order].astype(np.int32)


def test_noalloc_matches_regular_entry_point_twice(bc):
    g = bcgen.disjoint_union(bcgen.rmat(12, 8, 1), bcgen.path(6))  # has isolated vertices too
    G = bc.Graph(g.off, g.adj)
    for seed, k in ((1, 100), (2, 45)):
        src = bcgen.sample_sources(g, k, seed)
        src = np.concatenate([src, src[:3]])  # repeated sources count once per entry
        want, _ = G.compute(src)
        st, got = noalloc(bc, g.off, g.adj, src)
        assert st in (bc.BC_OK, bc.BC_W_SIGMA_INEXACT), bc.last_error()
        close(got, want.cpu().numpy())
        close(got, oracle.bc(g.off, g.adj, src))


def test_noalloc_rows_above_1024_arcs(bc):
    g = bcgen.disjoint_union(bcgen.star(2001), bcgen.rmat(10, 8, 1))  # the hub's row has 2000 arcs
    assert int(np.diff(g.off).max()) == 2000
    src = np.concatenate([[0, 1, 2], bcgen.sample_sources(g, 150, 3)]).astype(np.int32)
    st, got = noalloc(bc, g.off, g.adj, src)
    assert st == bc.BC_OK, bc.last_error()
    close(got, oracle.bc(g.off, g.adj, src))


def test_noalloc_extended_range_rerun(bc):
    # 24 layers of 8 vertices, consecutive layers completely joined: from a
    # layer-0 source the counts are 8^(k-1) in layer k, up to 8^22 = 2^66
    L, w = 24, 8
    u, v = [], []
    for k in range(L - 1):
        for a in range(w):
            for b in range(w):
                u += [k * w + a, (k + 1) * w + b]
                v += [(k + 1) * w + b, k * w + a]
    off, adj = csr_from_arcs(L * w, u, v)
    src = np.array([0, 3, 8 * 12 + 5, L * w - 1, 0], dtype=np.int32)
    st, got = noalloc(bc, off, adj, src)
    assert st == bc.BC_W_SIGMA_INEXACT, bc.last_error()
    close(got, oracle.bc_ld(off, adj, src).astype(np.float64))


def test_noalloc_repeated_arc_rows_bound_the_sums(bc):
    # a path 0-1-2-3-4 whose every edge is repeated M times in both rows: from
    # source 0 the counts are M^k at vertex k.  With M = 70,000, M^3 < 2^49 but
    # the 70,000-term sum at vertex 4 is M^4 > 2^64: only a bound taken from the
    # longest row (140,000 arcs) sends the batch to the extended form in time
    M = 70000
    u = np.concatenate([np.full(M, k) for k in range(4)] + [np.full(M, k + 1) for k in range(4)])
    v = np.concatenate([np.full(M, k + 1) for k in range(4)] + [np.full(M, k) for k in range(4)])
    off, adj = csr_from_arcs(5, u, v)
    assert int(np.diff(off).max()) == 2 * M
    src = np.arange(5, dtype=np.int32)
    st, got = noalloc(bc, off, adj, src)
    assert st == bc.BC_W_SIGMA_INEXACT, bc.last_error()
    want = oracle.bc_ld(off, adj, src).astype(np.float64)
    close(got, want)
    close(got, [0, 6, 8, 6, 0])  # the path's raw BC: repeated arcs cancel in sigma_v / sigma_w


def test_noalloc_more_sources_than_one_launch(bc):
    g = bcgen.rmat(8, 4, 2)
    base = bcgen.sample_sources(g, 100, 4)
    src = np.resize(base, 70001).astype(np.int32)  # 65,536 sources per launch: two launches
    st, got = noalloc(bc, g.off, g.adj, src)
    assert st == bc.BC_OK, bc.last_error()
    close(got, oracle.bc(g.off, g.adj, src))


def test_noalloc_rejects_bad_inputs_then_runs(bc):
    g = bcgen.rmat(9, 4, 1)
    src = bcgen.sample_sources(g, 40, 1)
    off = g.off.copy()
    off[6] = off[5] - 1  # offsets no longer monotone
    st, _ = noalloc(bc, off, g.adj, src)
    assert st == bc.BC_E_INVALID_GRAPH
    adj = g.adj.copy()
    adj[-1] = g.n  # an index outside [0, n)
    st, _ = noalloc(bc, g.off, adj, src)
    assert st == bc.BC_E_INVALID_GRAPH
    st, _ = noalloc(bc, g.off, g.adj, np.concatenate([src, [g.n]]).astype(np.int32))
    assert st == bc.BC_E_SOURCE
    st, _ = noalloc(bc, g.off, g.adj, np.array([-1], dtype=np.int32))
    assert st == bc.BC_E_SOURCE
    st, got = noalloc(bc, g.off, g.adj, src)
    assert st == bc.BC_OK, bc.last_error()
    close(got, oracle.bc(g.off, g.adj, src))


def test_noalloc_refuses_graphs_beyond_its_capacity(bc):
    lib = bc.load()
    # refused from the sizes alone: nothing on the device is read or written
    st = lib.bc_compute_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), 40000, 10, ctypes.c_void_p(16), 1,
                                ctypes.c_void_p(16), None)
    assert st == bc.BC_E_LIMIT
    assert "32768" in bc.last_error()
