"""GPU parity for weighted BC (bc_graph_create_weighted / bc_compute_weighted)
against the weighted CPU oracle (Dijkstra distances, the same accumulation),
on undirected graphs and on directed ones (per-arc weights).

Tolerance as for the unweighted path: 1e-9 relative per vertex, exact zeros
exact.  Weights 1..3 on the small graphs make many equal-weight paths of
different hop counts; R-MAT weights 1..100 give long relaxation chains.
"""
import numpy as np
import pytest

import bcgen
import oracle

pytestmark = pytest.mark.gpu

REL = 1e-9


@pytest.fixture(scope="module")
def bc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_03317_b300 as m
    m.load()
    return m


def assert_bc_close(got, want, rel=REL):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape
    zero = want == 0
    assert np.all(got[zero] == 0), "exact zeros must stay zero"
    err = np.abs(got - want) / np.maximum(np.abs(want), 1e-300)
    assert np.all(err[~zero] <= rel), f"max rel err {err[~zero].max()}"


def wgpu(bc, g, wt, src):
    G = bc.Graph(g.off, g.adj, weights=wt)
    out, st = G.compute_weighted(np.asarray(src, np.int32))
    res = out.cpu().numpy().copy()
    stats = G.stats()
    G.close()
    return res, st, stats


SMALL = [bcgen.gnp(n, p, seed) for n, p, seed in ((8, 0.5, 1), (30, 0.2, 2), (120, 0.05, 3), (200, 0.03, 4))] + \
        [bcgen.path(40), bcgen.cycle(33), bcgen.grid(9, 11, 0.1, 2), bcgen.random_tree(300, 5),
         bcgen.disjoint_union(bcgen.path(5), bcgen.empty_graph(3), bcgen.cycle(6))]


@pytest.mark.parametrize("g", SMALL, ids=lambda g: g.name)
@pytest.mark.parametrize("wmax", [1, 3])
def test_small_graphs_all_sources(bc, g, wmax):
    wt = bcgen.edge_weights(g, 1, wmax, seed=g.n)
    got, st, _ = wgpu(bc, g, wt, np.arange(g.n))
    assert st == bc.BC_OK
    assert_bc_close(got, oracle.wbc(g.off, g.adj, wt, np.arange(g.n)))


def test_tiny_graph_brute_force(bc):
    g = bcgen.gnp(8, 0.6, 5)
    wt = bcgen.edge_weights(g, 1, 2, 9)
    got, _, _ = wgpu(bc, g, wt, np.arange(g.n))
    want = oracle.brute_force_wbc(g.off, g.adj, wt, range(g.n))
    assert_bc_close(got, [float(x) for x in want])


def test_rmat_all_sources_and_repeatable(bc):
    g = bcgen.rmat(12, 8, 1)
    wt = bcgen.edge_weights(g, 1, 100, 1)
    src = np.arange(g.n)
    G = bc.Graph(g.off, g.adj, weights=wt)
    a, st = G.compute_weighted(src)
    a = a.cpu().numpy().copy()
    stats = G.stats()
    b, _ = G.compute_weighted(src)
    assert np.array_equal(a.view(np.uint64), b.cpu().numpy().view(np.uint64))
    assert st == bc.BC_OK and stats["batches"] == (g.n + 31) // 32
    assert stats["max_levels"] >= 2 and stats["pull_levels"] >= 2 and stats["push_levels"] >= 2
    # the first pass of each of the three loops reads every arc of every batch
    assert stats["arcs_visited"] >= 3 * stats["batches"] * g.m * 0.9 and stats["rows_visited"] >= 3 * g.n
    assert_bc_close(a, oracle.wbc(g.off, g.adj, wt, src))


def test_long_rows_take_the_chunk_path(bc):
    # hubs above 1024 arcs: a weighted star and an R-MAT graph with big hubs
    s = bcgen.star(3000)
    wt = bcgen.edge_weights(s, 1, 5, 2)
    got, _, _ = wgpu(bc, s, wt, np.arange(0, 3000, 7))
    assert_bc_close(got, oracle.wbc(s.off, s.adj, wt, np.arange(0, 3000, 7)))
    g = bcgen.rmat(15, 16, 2)
    assert np.diff(g.off).max() > 1024
    wt = bcgen.edge_weights(g, 1, 7, 2)
    src = bcgen.sample_sources(g, 70, 3)
    got, _, _ = wgpu(bc, g, wt, src)
    assert_bc_close(got, oracle.wbc(g.off, g.adj, wt, src))


def test_equal_weights_match_unweighted_bc(bc):
    g = bcgen.rmat(11, 8, 4)
    src = bcgen.sample_sources(g, 100, 4)
    got, _, _ = wgpu(bc, g, np.full(g.m, 5, np.int32), src)
    G = bc.Graph(g.off, g.adj)
    unw, _ = G.compute(src, source_order=1)
    assert_bc_close(got, unw.cpu().numpy())


def test_duplicates_empty_and_isolated_sources(bc):
    g = bcgen.disjoint_union(bcgen.rmat(8, 6, 2), bcgen.empty_graph(5))
    wt = bcgen.edge_weights(g, 1, 4, 1)
    src = np.array([3, 3, g.n - 1, 10, 3], np.int32)  # g.n - 1 is isolated
    got, _, _ = wgpu(bc, g, wt, src)
    assert_bc_close(got, oracle.wbc(g.off, g.adj, wt, src))
    zero, st, _ = wgpu(bc, g, wt, np.zeros(0, np.int32))
    assert st == bc.BC_OK and not zero.any()


def _layers(a, layers):
    u, v = [], []
    for j in range(a):
        u.append(0); v.append(1 + j)
    for i in range(layers - 1):
        for j in range(a):
            for k in range(a):
                u.append(1 + i * a + j); v.append(1 + (i + 1) * a + k)
    return bcgen.edges_to_csr(1 + a * layers, np.array(u), np.array(v))


def test_path_count_range(bc):
    g = _layers(16, 16)  # counts up to 2^60: inexact beyond 2^53, still below 2^64
    wt = np.full(g.m, 3, np.int32)
    got, st, _ = wgpu(bc, g, wt, [0, 5])
    assert st == bc.BC_W_SIGMA_INEXACT
    assert_bc_close(got, oracle.wbc(g.off, g.adj, wt, [0, 5]))
    g = _layers(16, 18)  # 2^68
    with pytest.raises(bc.BCError) as ei:
        wgpu(bc, g, np.full(g.m, 1, np.int32), [0])
    assert ei.value.status == bc.BC_E_SIGMA_RANGE


def test_invalid_weighted_inputs(bc):
    g = bcgen.gnp(40, 0.2, 7)
    wt = bcgen.edge_weights(g, 1, 9, 7)
    bad = wt.copy(); bad[3] = 0
    with pytest.raises(bc.BCError) as ei:
        bc.Graph(g.off, g.adj, weights=bad)
    assert ei.value.status == bc.BC_E_INVALID_GRAPH
    bad = wt.copy(); bad[3] += 1  # one arc of an edge differs from its twin
    with pytest.raises(bc.BCError) as ei:
        bc.Graph(g.off, g.adj, weights=bad)
    assert ei.value.status == bc.BC_E_INVALID_GRAPH
    adj = g.adj.copy()
    r = int(np.argmax(np.diff(g.off)))
    adj[g.off[r]:g.off[r + 1]] = adj[g.off[r]:g.off[r + 1]][::-1]  # a row out of order
    with pytest.raises(bc.BCError) as ei:
        bc.Graph(g.off, adj, weights=wt)
    assert ei.value.status == bc.BC_E_INVALID_GRAPH
    with pytest.raises(bc.BCError) as ei:  # directed: weights are per arc, still positive
        bc.Graph(g.off, g.adj, weights=np.where(np.arange(g.m) == 5, -2, wt).astype(np.int32), directed=True)
    assert ei.value.status == bc.BC_E_INVALID_GRAPH
    G = bc.Graph(g.off, g.adj)
    with pytest.raises(bc.BCError) as ei:
        G.compute_weighted(np.arange(3))
    assert ei.value.status == bc.BC_E_INVALID_ARG
    W = bc.Graph(g.off, g.adj, weights=wt)
    with pytest.raises(bc.BCError) as ei:
        W.compute_weighted(np.array([0, 40], np.int32))
    assert ei.value.status == bc.BC_E_SOURCE
    out, _ = W.compute_weighted(np.arange(5))  # the library is usable after the errors
    assert_bc_close(out.cpu().numpy(), oracle.wbc(g.off, g.adj, wt, np.arange(5)))
    # the unweighted calls ignore the weights
    a, _ = W.compute(np.arange(5))
    b, _ = G.compute(np.arange(5))
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_device_inputs_and_skip_validation(bc):
    import torch
    g = bcgen.rmat(10, 8, 6)
    wt = bcgen.edge_weights(g, 1, 30, 6)
    src = bcgen.sample_sources(g, 40, 6)
    want = oracle.wbc(g.off, g.adj, wt, src)
    host, _, _ = wgpu(bc, g, wt, src)
    # CSR and weights already on the device (BC_INPUT_ON_DEVICE)
    G = bc.Graph(torch.from_numpy(g.off).cuda(), torch.from_numpy(g.adj).cuda(),
                 weights=torch.from_numpy(wt).cuda())
    dev, _ = G.compute_weighted(torch.from_numpy(src).cuda())
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), host.view(np.uint64))
    # valid input with the checks skipped gives the same result
    S = bc.Graph(g.off, g.adj, weights=wt, validate=False)
    skip, _ = S.compute_weighted(src)
    assert np.array_equal(skip.cpu().numpy().view(np.uint64), host.view(np.uint64))
    assert_bc_close(host, want)


# ------------------------------------------------------------ directed graphs

DSMALL = [bcgen.orient(g, seed=i + 1, p_both=0.3) for i, g in enumerate(SMALL)]


def wgpu_dir(bc, g, wt, src):
    G = bc.Graph(g.off, g.adj, weights=wt, directed=True)
    out, st = G.compute_weighted(np.asarray(src, np.int32))
    res = out.cpu().numpy().copy()
    stats = G.stats()
    G.close()
    return res, st, stats


@pytest.mark.parametrize("g", DSMALL, ids=lambda g: g.name)
@pytest.mark.parametrize("wmax", [1, 3])
def test_directed_small_graphs_all_sources(bc, g, wmax):
    wt = bcgen.edge_weights(g, 1, wmax, seed=g.n + 1, per_arc=True)
    got, st, _ = wgpu_dir(bc, g, wt, np.arange(g.n))
    assert st == bc.BC_OK
    assert_bc_close(got, oracle.wbc(g.off, g.adj, wt, np.arange(g.n)))


def test_directed_tiny_graph_brute_force(bc):
    g = bcgen.orient(bcgen.gnp(9, 0.6, 6), seed=2, p_both=0.4)
    wt = bcgen.edge_weights(g, 1, 2, 3, per_arc=True)
    got, _, _ = wgpu_dir(bc, g, wt, np.arange(g.n))
    assert_bc_close(got, [float(x) for x in oracle.brute_force_wbc(g.off, g.adj, wt, range(g.n))])


def _in_and_out_hubs(n, seed):
    # vertex 0: in-arcs from everyone, no out-arcs (relabelled last: a heavy
    # in-row outside the prefix); vertex 1: out-arcs to everyone (a heavy
    # out-row); plus an oriented random graph
    rest = bcgen.orient(bcgen.gnp(n, 4.0 / n, seed), seed=seed, p_both=0.2)
    deg = np.diff(rest.off.astype(np.int64))
    u = np.repeat(np.arange(n), deg)
    keep = (u != 0) & (rest.adj != 1) & (u != 1) & (rest.adj != 0)
    su = np.concatenate([np.arange(1, n), np.full(n - 2, 1), u[keep]])
    sv = np.concatenate([np.zeros(n - 1, np.int64), np.arange(2, n), rest.adj[keep]])
    return bcgen.directed_csr(n, su, sv, f"hubs{n}")


def test_directed_heavy_in_rows_outside_the_prefix(bc):
    g = _in_and_out_hubs(3000, 4)
    indeg = np.bincount(g.adj, minlength=g.n)
    assert indeg[0] > 2048 and np.diff(g.off)[0] == 0 and np.diff(g.off)[1] > 2048
    wt = bcgen.edge_weights(g, 1, 6, 5, per_arc=True)
    src = np.concatenate([[1, 0], bcgen.sample_sources(g, 62, 5)])
    got, st, stats = wgpu_dir(bc, g, wt, src)
    assert st == bc.BC_OK and stats["batches"] == 2
    assert_bc_close(got, oracle.wbc(g.off, g.adj, wt, src))


def test_directed_rmat_all_sources_repeatable(bc):
    g = bcgen.orient(bcgen.rmat(12, 8, 3), seed=4)
    wt = bcgen.edge_weights(g, 1, 100, 3, per_arc=True)
    src = np.arange(g.n)
    G = bc.Graph(g.off, g.adj, weights=wt, directed=True)
    a, st = G.compute_weighted(src)
    a = a.cpu().numpy().copy()
    stats = G.stats()
    b, _ = G.compute_weighted(src)
    assert np.array_equal(a.view(np.uint64), b.cpu().numpy().view(np.uint64))
    assert st == bc.BC_OK and stats["batches"] == (g.n + 31) // 32
    assert stats["arcs_visited"] >= 3 * stats["batches"] * g.m * 0.9
    assert_bc_close(a, oracle.wbc(g.off, g.adj, wt, src))


def test_directed_long_rows_both_directions(bc):
    g = bcgen.orient(bcgen.rmat(15, 16, 2), seed=3, p_both=0.5)
    indeg = np.bincount(g.adj, minlength=g.n)
    assert np.diff(g.off).max() > 1024 and indeg.max() > 1024
    wt = bcgen.edge_weights(g, 1, 7, 2, per_arc=True)
    src = bcgen.sample_sources(g, 40, 3)
    got, _, _ = wgpu_dir(bc, g, wt, src)
    assert_bc_close(got, oracle.wbc(g.off, g.adj, wt, src))


def test_directed_equal_weights_match_unweighted_bc(bc):
    g = bcgen.orient(bcgen.rmat(11, 8, 6), seed=7)
    src = bcgen.sample_sources(g, 90, 2)
    got, _, _ = wgpu_dir(bc, g, np.full(g.m, 3, np.int32), src)
    G = bc.Graph(g.off, g.adj, directed=True)
    unw, _ = G.compute(src)
    assert_bc_close(got, unw.cpu().numpy())
    # the transpose's arcs carry their own weights: an unweighted directed
    # call on the same graph ignores them
    W = bc.Graph(g.off, g.adj, weights=bcgen.edge_weights(g, 1, 9, 1, per_arc=True), directed=True)
    a, _ = W.compute(src)
    assert np.array_equal(a.cpu().numpy(), unw.cpu().numpy())


def test_directed_device_inputs_and_skip_validation(bc):
    import torch
    g = bcgen.orient(bcgen.rmat(10, 8, 8), seed=9)
    wt = bcgen.edge_weights(g, 1, 30, 8, per_arc=True)
    src = bcgen.sample_sources(g, 40, 8)
    host, _, _ = wgpu_dir(bc, g, wt, src)
    D = bc.Graph(torch.from_numpy(g.off).cuda(), torch.from_numpy(g.adj).cuda(),
                 weights=torch.from_numpy(wt).cuda(), directed=True)
    dev, _ = D.compute_weighted(torch.from_numpy(src).cuda())
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), host.view(np.uint64))
    S = bc.Graph(g.off, g.adj, weights=wt, validate=False, directed=True)
    skip, _ = S.compute_weighted(src)
    assert np.array_equal(skip.cpu().numpy().view(np.uint64), host.view(np.uint64))
    assert_bc_close(host, oracle.wbc(g.off, g.adj, wt, src))


def test_directed_sinks_isolated_and_edgeless(bc):
    # sources that are sinks (no out-arcs) or isolated give zero terms; a
    # graph with no arcs gives zeros
    g = bcgen.disjoint_union(bcgen.orient(bcgen.gnp(60, 0.08, 3), seed=2, p_both=0.1), bcgen.empty_graph(4))
    wt = bcgen.edge_weights(g, 1, 5, 4, per_arc=True)
    sinks = np.flatnonzero(np.diff(g.off) == 0)
    assert len(sinks) > 4
    src = np.concatenate([sinks[:6], np.arange(0, g.n, 5)]).astype(np.int32)
    got, st, _ = wgpu_dir(bc, g, wt, src)
    assert st == bc.BC_OK
    assert_bc_close(got, oracle.wbc(g.off, g.adj, wt, src))
    e = bcgen.empty_graph(7)
    zero, st, _ = wgpu_dir(bc, e, np.zeros(0, np.int32), np.arange(7))
    assert st == bc.BC_OK and not zero.any()
