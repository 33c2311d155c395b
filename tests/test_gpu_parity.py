"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerance (derived for the reading that BC is the raw sum of delta): every
delta term is non-negative, so no cancellation; double rounding of a sum of
k positive terms is bounded by ~k * 2^-53 relative.  The GPU forms the sum as
sigma_v * sum_w (1+delta_w)/sigma_w while the oracle forms per-arc ratios, so
the two differ by a few ulps per level of the DAG; 1e-9 relative per vertex
is far above that and exact zeros must stay exact zeros.  Levels and path
counts below 2^53 are compared bit for bit.
"""
import os

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


def gpu_bc(bc, g, src, **kw):
    G = bc.Graph(g.off, g.adj)
    out, st = G.compute(np.asarray(src, np.int32), **kw)
    res = out.cpu().numpy().copy()
    stats = G.stats()
    G.close()
    return res, st, stats


# ----------------------------------------------------------------- ingest

@pytest.mark.parametrize("g", [bcgen.rmat(12, 8, 1), bcgen.grid(30, 31, 0.05, 2), bcgen.star(50),
                               bcgen.disjoint_union(bcgen.path(5), bcgen.empty_graph(4), bcgen.cycle(9)),
                               bcgen.rmat_n(3000, 11, 5)], ids=lambda g: g.name)
def test_relabel_matches_oracle(bc, g):
    G = bc.Graph(g.off, g.adj)
    perm, off, adj = G.export()
    operm, _, ooff, oadj = oracle.relabel(g.off, g.adj)
    assert np.array_equal(perm, operm)
    assert np.array_equal(off, ooff)
    assert np.array_equal(adj, oadj)
    deg = g.degrees()
    assert G.max_degree == int(deg.max()) and G.n_nonisolated == int((deg > 0).sum())


def test_invalid_graphs_rejected(bc):
    g = bcgen.cycle(6)
    cases = []
    off = g.off.copy(); off[2] = off[1] - 1; cases.append((off, g.adj))
    adj = g.adj.copy(); adj[3] = 6; cases.append((g.off, adj))
    adj = g.adj.copy(); adj[0] = 0; cases.append((g.off, adj))
    adj = g.adj.copy(); adj[1] = adj[0]; cases.append((g.off, adj))
    h = bcgen.path(4)
    adj = h.adj.copy(); adj[1] = 3; cases.append((h.off, adj))
    for off, adj in cases:
        assert oracle.validate(off, adj) != 0
        with pytest.raises(bc.BCError) as ei:
            bc.Graph(off, adj)
        assert ei.value.status == bc.BC_E_INVALID_GRAPH


def test_source_out_of_range_and_empty(bc):
    g = bcgen.path(5)
    G = bc.Graph(g.off, g.adj)
    with pytest.raises(bc.BCError) as ei:
        G.compute(np.array([5], np.int32))
    assert ei.value.status == bc.BC_E_SOURCE
    out, st = G.compute(np.zeros(0, np.int32))
    assert st == bc.BC_OK and np.all(out.cpu().numpy() == 0)
    # the graph is still usable after a rejected call
    out, _ = G.compute(np.arange(5, dtype=np.int32))
    assert_bc_close(out.cpu().numpy(), oracle.bc(g.off, g.adj, np.arange(5)))


# ----------------------------------------------------------------- exact small cases

@pytest.mark.parametrize("K", [1, 32, 64, 128])
def test_golden_fixtures(bc, K):
    from golden_io import load
    for rec in load():
        got, _, _ = gpu_bc(bc, bcgen.CSR(rec["off"], rec["adj"]), rec["src"], batch_width=K)
        assert_bc_close(got, [float(x) for x in rec["bc"]], rel=1e-12)


@pytest.mark.parametrize("g,half", [
    (bcgen.path(300), lambda n: [i * (n - 1 - i) for i in range(n)]),
    (bcgen.star(200), lambda n: [(n - 1) * (n - 2) / 2] + [0] * (n - 1)),
    (bcgen.cycle(101), lambda n: [(n - 1) * (n - 3) / 8] * n),
    (bcgen.cycle(100), lambda n: [(n - 2) ** 2 / 8] * n),
    (bcgen.complete(12), lambda n: [0] * n),
], ids=["path300", "star200", "cycle101", "cycle100", "K12"])
def test_closed_forms(bc, g, half):
    got, _, _ = gpu_bc(bc, g, np.arange(g.n))
    assert_bc_close(got / 2, half(g.n), rel=1e-12)


def test_complete_bipartite_and_tree(bc):
    import math
    g = bcgen.complete_bipartite(4, 7)
    got, _, _ = gpu_bc(bc, g, np.arange(g.n))
    assert_bc_close(got / 2, [math.comb(7, 2) / 4] * 4 + [math.comb(4, 2) / 7] * 7, rel=1e-12)
    t = bcgen.random_tree(3000, 3)
    got, _, _ = gpu_bc(bc, t, np.arange(t.n))
    assert_bc_close(got, oracle.bc(t.off, t.adj, np.arange(t.n)), rel=1e-12)


# ----------------------------------------------------------------- R-MAT, all widths

@pytest.fixture(scope="module")
def rmat12():
    g = bcgen.rmat(12, 8, 1)
    return g, oracle.bc(g.off, g.adj, np.arange(g.n))


@pytest.mark.parametrize("K", [1, 32, 64, 128])
def test_rmat12_all_sources(bc, rmat12, K):
    g, want = rmat12
    got, st, stats = gpu_bc(bc, g, np.arange(g.n), batch_width=K)
    assert st == bc.BC_OK
    assert stats["batch_width"] == K
    assert_bc_close(got, want)


def test_rmat12_bitwise_across_widths_and_directions(bc, rmat12):
    g, _ = rmat12
    src = bcgen.sample_sources(g, 300, 4)
    ref, _, _ = gpu_bc(bc, g, src, batch_width=64)
    for kw in [dict(batch_width=1), dict(batch_width=32), dict(batch_width=128), dict(batch_width=64, direction=1),
               dict(batch_width=64, direction=2), dict(batch_width=64, group_vertices=1),
               dict(batch_width=32, group_vertices=7, direction=2), dict(batch_width=1, group_vertices=3),
               dict(batch_width=64, teams=1), dict(batch_width=32, teams=3), dict(batch_width=1, teams=7)]:
        got, _, _ = gpu_bc(bc, g, src, **kw)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), kw


def test_many_batches_team_counts_and_degree1_rule_keep_bits(bc):
    """Hundreds of batches on a medium graph: the automatic team count (several blocks per team),
    one team per batch and a few large teams give the same bits, with degree-1 vertices (left out of
    the reverse sweep) exactly 0 and the whole against the oracle."""
    g = bcgen.rmat(13, 8, 5)
    deg = np.diff(g.off)
    assert (deg == 1).sum() > 500  # many degree-1 vertices
    src = np.tile(np.nonzero(deg)[0].astype(np.int32), 2)[:9000]  # repeated sources: 71 batches of 128
    G = bc.Graph(g.off, g.adj)
    ref, st = G.compute(src)
    ref = ref.cpu().numpy().copy()
    auto_teams = G.stats()["teams"]
    assert 1 < auto_teams < 71
    for kw in (dict(teams=71), dict(teams=4), dict(batch_width=32), dict(batch_width=1), dict(deep_form=2)):
        out, st2 = G.compute(src, **kw)
        assert st2 == st
        assert np.array_equal(out.cpu().numpy().view(np.uint64), ref.view(np.uint64)), kw
    assert np.all(ref[deg == 1] == 0.0)
    assert_bc_close(ref, oracle.bc(g.off, g.adj, src))


def test_one_source_batches_on_a_large_graph_keep_bits(bc):
    """One-source batches on a graph large enough that their teams are capped
    (R-MAT 20: about one block per 2^19 arcs would give teams of 64 blocks; one-
    source batches keep at most about 32): the same bits as one 128-wide batch
    and as fewer, larger teams; over 8 of the sources, the oracle's values."""
    g = bcgen.rmat(20, 16, 1)
    src = bcgen.sample_sources(g, 64, 3)
    G = bc.Graph(g.off, g.adj)
    ref, st = G.compute(src, batch_width=128)
    assert st == bc.BC_OK
    ref = ref.cpu().numpy().copy()
    out, st1 = G.compute(src, batch_width=1)
    s = G.stats()
    assert st1 == st and s["batches"] == 64
    assert s["teams"] >= 12 and s["grid_blocks"] // s["teams"] <= 40, s
    assert np.array_equal(out.cpu().numpy().view(np.uint64), ref.view(np.uint64))
    out, st2 = G.compute(src, batch_width=1, teams=4)
    assert st2 == st and G.stats()["teams"] == 4
    assert np.array_equal(out.cpu().numpy().view(np.uint64), ref.view(np.uint64))
    few = src[:8]
    got, st3 = G.compute(few, batch_width=1)
    assert st3 == bc.BC_OK
    assert_bc_close(got.cpu().numpy(), oracle.bc(g.off, g.adj, few, threads=max(1, min(os.cpu_count() or 1, 64))))


def test_reduce_ranks_is_the_rank_order_sum(bc):
    import torch
    rng = np.random.default_rng(5)
    parts = rng.random((5, 1001)) * 10.0 ** rng.integers(-8, 8, (5, 1001))
    got = bc.reduce_ranks(torch.from_numpy(parts).cuda()).cpu().numpy()
    want = parts[0].copy()
    for r in parts[1:]:
        want = want + r
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    one = bc.reduce_ranks(torch.from_numpy(parts[:1]).cuda()).cpu().numpy()
    assert np.array_equal(one.view(np.uint64), parts[0].view(np.uint64))


def test_job_split_over_emulated_ranks(bc, rmat12):
    # the multi-GPU split run rank after rank on one GPU: each rank's share of
    # the job's batches through bc_compute_ex, then the rank-order sum
    import torch
    from grouping import grouped_order
    from paper_2305_03317_b300 import sharded
    g, _ = rmat12
    G = bc.Graph(g.off, g.adj)
    src = bcgen.sample_sources(g, 700, 3)
    order, K = G.source_batches(src)
    assert np.array_equal(order, src[grouped_order(g, G.export()[0], src)])  # the automatic grouping
    assert G.source_batches(src, source_order=1)[0].tolist() == src.tolist()
    full, _ = G.compute(src, batch_width=K)
    full = full.cpu().numpy().copy()
    want = oracle.bc(g.off, g.adj, src)
    for world in (1, 2, 3, 9):
        parts = []
        for r in range(world):
            mine = sharded.shard_of(order, K, r, world)
            part = torch.zeros(g.n, dtype=torch.float64, device="cuda")
            if len(mine):
                G.compute(mine, out=part, batch_width=K, source_order=1)
            parts.append(part)
        got = bc.reduce_ranks(torch.stack(parts)).cpu().numpy()
        assert_bc_close(got, want)
        if world == 1:
            assert np.array_equal(got.view(np.uint64), full.view(np.uint64))


def test_source_grouping_order_and_widths(bc, rmat12):
    g, _ = rmat12
    src = bcgen.sample_sources(g, 300, 4)
    want = oracle.bc(g.off, g.adj, src)
    ref, _, st = gpu_bc(bc, g, src, batch_width=64, source_order=2)
    assert st["order_ms"] > 0
    assert_bc_close(ref, want)
    # the grouping itself, from oracle levels: stable sort of the sources by their
    # distances to the 32 first relabelled (highest-degree) vertices, nearest first;
    # BC summed in that order, as given, must be the same bits
    from grouping import grouped_order
    G = bc.Graph(g.off, g.adj)
    perm = G.export()[0]
    G.close()
    order = grouped_order(g, perm, src)
    regrouped, _, st1 = gpu_bc(bc, g, src[order], batch_width=64, source_order=1)
    assert st1["order_ms"] == 0
    assert np.array_equal(regrouped.view(np.uint64), ref.view(np.uint64))
    for kw in [dict(batch_width=1), dict(batch_width=32), dict(batch_width=128), dict(batch_width=64, direction=2),
               dict(batch_width=32, teams=3)]:
        got, _, _ = gpu_bc(bc, g, src, source_order=2, **kw)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), kw
    with pytest.raises(bc.BCError):
        gpu_bc(bc, g, src, source_order=3)
    # auto: grouped on skewed undirected graphs with >= 256 sources, else as given
    _, _, st = gpu_bc(bc, g, src)
    assert st["order_ms"] > 0
    _, _, st = gpu_bc(bc, g, src[:255])
    assert st["order_ms"] == 0
    grid = bcgen.grid(60, 60, 0.0)
    gsrc = bcgen.sample_sources(grid, 300, 1)
    plain, _, st = gpu_bc(bc, grid, gsrc)
    assert st["order_ms"] == 0
    # a deep graph (more than 15 levels) takes the other sort of the grouping
    G = bc.Graph(grid.off, grid.adj)
    gorder = grouped_order(grid, G.export()[0], gsrc)
    G.close()
    got, _, st = gpu_bc(bc, grid, gsrc, source_order=2, batch_width=32)
    assert st["order_ms"] > 0 and st["max_levels"] > 16
    again, _, _ = gpu_bc(bc, grid, gsrc[gorder], source_order=1, batch_width=32)
    assert np.array_equal(got.view(np.uint64), again.view(np.uint64))
    assert_bc_close(got, plain)


def test_large_terms_in_column_mapped_sums_take_extended_form(bc):
    # s, then 16 layers of 16 vertices, consecutive layers complete bipartite:
    # sigma of layer i is 16^(i-1), so the last layer sums terms of 2^56.  128
    # copies of s match every column of every arc: all forward sums run
    # column-mapped, and a term >= 2^54 there must send the batch to the
    # extended form as it does in the pair path (whose 32-bit atomics may share
    # a sum with the column-mapped path).
    a, layers = 16, 16
    n = 1 + a * layers
    u, v = [], []
    for j in range(a):
        u.append(0); v.append(1 + j)
    for i in range(layers - 1):
        for j in range(a):
            for k in range(a):
                u.append(1 + i * a + j); v.append(1 + (i + 1) * a + k)
    g = bcgen.edges_to_csr(n, np.array(u), np.array(v), "layers16x16")
    src = np.zeros(128, np.int32)
    got, st, stats = gpu_bc(bc, g, src, batch_width=128, source_order=1)
    assert stats["ext_batches"] == 1 and st == bc.BC_W_SIGMA_INEXACT
    assert_bc_close(got, 128 * oracle.bc_ld(g.off, g.adj, src[:1]).astype(np.float64))


def test_duplicate_sources_count_twice(bc):
    g = bcgen.rmat(10, 6, 3)
    src = np.array([5, 9, 5, 5, 100, 9], np.int32)
    got, _, _ = gpu_bc(bc, g, src, batch_width=32)
    assert_bc_close(got, oracle.bc(g.off, g.adj, src))


def test_ragged_batches_and_isolated_sources(bc):
    g = bcgen.disjoint_union(bcgen.rmat(11, 8, 2), bcgen.empty_graph(3))
    src = np.concatenate([bcgen.sample_sources(g, 77, 9), np.array([g.n - 1, g.n - 2], np.int32)])
    for K in (32, 64):
        got, _, stats = gpu_bc(bc, g, src, batch_width=K)
        assert stats["batches"] == -(-len(src) // K)
        assert_bc_close(got, oracle.bc(g.off, g.adj, src))


# ----------------------------------------------------------------- levels and path counts

def test_debug_source_levels_and_sigma(bc):
    g = bcgen.rmat(12, 8, 1)
    G = bc.Graph(g.off, g.adj)
    for s in bcgen.sample_sources(g, 5, 2):
        lev, mant, ex, _ = G.debug_source(int(s))
        d = oracle.source_detail(g.off, g.adj, int(s))
        assert np.array_equal(lev, d["level"])
        sig = np.ldexp(mant, ex)
        assert np.array_equal(sig, d["sigma"])


def test_full_grid_extended_range(bc):
    """Path counts up to C(298,149) ~ 2^293: beyond 2^64, so the extended form runs."""
    g = bcgen.grid(150, 150, 0.0)
    src = np.array([0, 151, 150 * 75 + 75], np.int32)
    G = bc.Graph(g.off, g.adj)
    out, st = G.compute(np.concatenate([src] * 11), batch_width=1, teams=4)  # 33 batches over 4 teams
    assert st == bc.BC_W_SIGMA_INEXACT
    assert_bc_close(out.cpu().numpy(), 11 * oracle.bc_ld(g.off, g.adj, src).astype(np.float64))
    out, st = G.compute(src, batch_width=32)
    stats = G.stats()
    assert st == bc.BC_W_SIGMA_INEXACT and stats["ext_batches"] > 0
    want = oracle.bc_ld(g.off, g.adj, src).astype(np.float64)
    assert_bc_close(out.cpu().numpy(), want)
    # the extended form keeps every column's sums in CSR order too: the plain
    # per-source form and both batch widths agree bit for bit
    for kw in (dict(batch_width=1), dict(batch_width=64), dict(batch_width=32, direction=1)):
        other, _ = G.compute(src, **kw)
        assert np.array_equal(other.cpu().numpy().view(np.uint64), out.cpu().numpy().view(np.uint64)), kw
    lev, mant, ex, _ = G.debug_source(0)
    olev, omant, oex, _ = oracle.source_sigma_split(g.off, g.adj, 0)
    assert np.array_equal(lev, olev)
    rel = np.abs(mant * np.ldexp(1.0, ex - oex) - omant) / omant
    assert rel.max() <= 1e-12
    # counts below 2^53 stay exact in the extended form
    small = oex <= 53
    assert np.array_equal(np.ldexp(mant[small], ex[small]), np.ldexp(omant[small], oex[small]))


# ----------------------------------------------------------------- failure handling

def test_barrier_timeout_reports_and_recovers(bc):
    g = bcgen.rmat(11, 8, 1)
    G = bc.Graph(g.off, g.adj)
    src = bcgen.sample_sources(g, 64, 1)
    with pytest.raises(bc.BCError) as ei:
        G.compute(src, batch_width=64, barrier_budget=1)
    assert ei.value.status == bc.BC_E_TIMEOUT
    out, st = G.compute(src, batch_width=64)
    assert_bc_close(out.cpu().numpy(), oracle.bc(g.off, g.adj, src))


# ----------------------------------------------------------------- serving

def test_serving_alone_equals_mix(bc):
    import torch
    graphs = [bcgen.rmat(11, 8, 1), bcgen.rmat(12, 4, 2), bcgen.grid(40, 40, 0.05, 3)]
    Gs = [bc.Graph(g.off, g.adj) for g in graphs]
    reqs = [(i % 3, bcgen.sample_sources(graphs[i % 3], k, 10 + i)) for i, k in
            enumerate([1, 3, 40, 7, 130, 2, 64, 5, 17, 300, 1, 33])]

    def run(batch):
        outs, jobs = [], []
        for gi, src in batch:
            o = torch.empty(graphs[gi].n, dtype=torch.float64, device="cuda")
            outs.append(o)
            jobs.append(Gs[gi].submit(src, o))
        for j in jobs:
            assert j.wait(120000) is not None
        return [o.cpu().numpy().copy() for o in outs]

    alone = [run([r])[0] for r in reqs]
    mixed = run(reqs)  # one slot: jobs of a graph packed into shared batches
    for (gi, src), a, b in zip(reqs, alone, mixed):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
        assert_bc_close(b, oracle.bc(graphs[gi].off, graphs[gi].adj, src))
    bc.server_config(3)  # three concurrent traversals, several on the same graph
    mixed3 = run(reqs + reqs)
    for a, b in zip(alone + alone, mixed3):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    peak, done = bc.server_stats()
    assert done >= 4 * len(reqs)


def test_served_job_equals_direct_call_with_grouped_sources(bc):
    # a job large enough to be grouped (skewed graph, >= 256 sources): the same
    # bits served alone, served packed with other jobs, and from bc_compute
    import torch
    g = bcgen.rmat(13, 16, 7)
    G = bc.Graph(g.off, g.adj)
    big = bcgen.sample_sources(g, 600, 7)
    direct, _ = G.compute(big)
    assert G.stats()["order_ms"] > 0
    direct = direct.cpu().numpy().copy()
    outs = [torch.empty(g.n, dtype=torch.float64, device="cuda") for _ in range(3)]
    jobs = [G.submit(big, outs[0]), G.submit(bcgen.sample_sources(g, 40, 8), outs[1]), G.submit(big, outs[2])]
    for j in jobs:
        assert j.wait(120000) is not None
    for o in (outs[0], outs[2]):
        assert np.array_equal(o.cpu().numpy().view(np.uint64), direct.view(np.uint64))
    assert_bc_close(direct, oracle.bc(g.off, g.adj, big))


# ----------------------------------------------------------------- rows above 1024 arcs (chunk tasks)

@pytest.fixture(scope="module")
def heavy_graph():
    g = bcgen.rmat(14, 64, 3)  # 106 rows above 1024 arcs, the largest ~6.9K arcs (7 chunks)
    assert int(g.degrees().max()) > 4 * 1024
    src = bcgen.sample_sources(g, 160, 7)
    return g, src, oracle.bc(g.off, g.adj, src)


@pytest.mark.parametrize("kw", [dict(batch_width=1), dict(batch_width=32), dict(batch_width=64),
                                dict(batch_width=128), dict(batch_width=64, direction=1),
                                dict(batch_width=64, direction=2), dict(batch_width=32, group_vertices=5)],
                         ids=lambda kw: "-".join(f"{k}{v}" for k, v in kw.items()))
def test_heavy_rows_parity(bc, heavy_graph, kw):
    g, src, want = heavy_graph
    got, st, stats = gpu_bc(bc, g, src, **kw)
    assert_bc_close(got, want)


def test_heavy_rows_bitwise_across_forms(bc, heavy_graph):
    g, src, _ = heavy_graph
    ref, _, _ = gpu_bc(bc, g, src, batch_width=64)
    for kw in [dict(batch_width=1), dict(batch_width=128), dict(batch_width=32, direction=1),
               dict(batch_width=128, direction=2), dict(batch_width=32, teams=5), dict(batch_width=64, teams=1)]:
        got, _, _ = gpu_bc(bc, g, src, **kw)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), kw


def test_star_hub_all_sources(bc):
    """A hub of degree 3000 (3 chunks) reached at level 0 and level 1, all sources."""
    g = bcgen.disjoint_union(bcgen.star(3001), bcgen.path(3))
    for K in (1, 64):
        got, _, _ = gpu_bc(bc, g, np.arange(g.n), batch_width=K)
        half = np.zeros(g.n)
        half[0] = 3000 * 2999 / 2
        half[3002] = 1
        assert_bc_close(got / 2, half, rel=1e-12)


# ----------------------------------------------------------------- many graphs, one recorded sequence

def test_many_graphs_plan_matches_single_calls(bc):
    import torch
    sizes = [(300, 6, 11), (1000, 12, 12), (2500, 20, 13), (4000, 8, 14), (700, 31, 15), (5000, 16, 16)]
    graphs = [bcgen.rmat_n(n, ef, seed) for n, ef, seed in sizes] + [bcgen.grid(70, 70, 0.0),
                                                                      bcgen.star(2500), bcgen.rmat_n(6000, 16, 17)]
    items, refs, oracles = [], [], []
    for i, g in enumerate(graphs):
        # the last item (400 sources on a skewed graph) has its sources grouped, as bc_compute groups them
        nsrc = 400 if i == len(graphs) - 1 else 100
        src = np.arange(g.n, dtype=np.int32) if g.n <= 1200 else bcgen.sample_sources(g, nsrc, 30 + i)
        G = bc.Graph(g.off, g.adj)
        out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        items.append((G, src, out))
        ref, _ = bc.Graph(g.off, g.adj).compute(src)
        refs.append(ref.cpu().numpy().copy())
        want = oracle.bc_ld(g.off, g.adj, src).astype(np.float64) if g.n == 4900 else oracle.bc(g.off, g.adj, src)
        oracles.append(want)
    plan = bc.ManyPlan(items)
    assert plan.info()["items"] == len(items)
    for rep in range(2):  # replay twice
        st = plan.run()
        assert all(int(x) in (bc.BC_OK, bc.BC_W_SIGMA_INEXACT) for x in st)
        for (G, src, out), ref, want in zip(items, refs, oracles):
            got = out.cpu().numpy()
            assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
            assert_bc_close(got, want)
    # the 70x70 full grid needs the extended form (and, 138 levels deep, runs in the per-source form)
    assert int(st[len(sizes)]) == bc.BC_W_SIGMA_INEXACT
    G, src, _ = items[-1]
    G.compute(src)
    assert G.stats()["order_ms"] > 0  # the single call grouped the same sources
    # a graph a plan uses is not freed under it
    with pytest.raises(bc.BCError) as ei:
        items[0][0].close()
    assert ei.value.status == bc.BC_E_BUSY
    plan.close()
    items[0][0].close()


def test_graph_in_use_by_serving_job_is_not_freed(bc):
    import torch
    g = bcgen.rmat(13, 16, 5)
    G = bc.Graph(g.off, g.adj)
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    src = bcgen.sample_sources(g, 512, 5)
    job = G.submit(src, out)
    try:
        G.close()
        closed_early = True  # the job finished before the call: allowed
    except bc.BCError as e:
        assert e.status == bc.BC_E_BUSY
        closed_early = False
    assert job.wait(600000) is not None
    if not closed_early:
        G.close()
    assert_bc_close(out.cpu().numpy(), oracle.bc(g.off, g.adj, src))


def test_autotune_changes_speed_not_results(bc, rmat12, tmp_path):
    g, _ = rmat12
    src = bcgen.sample_sources(g, 300, 4)
    G = bc.Graph(g.off, g.adj)
    before, _ = G.compute(src)
    before = before.cpu().numpy().copy()
    best = G.autotune(src)
    assert best["batch_width"] in (1, 32, 64, 128) and best["rate"] > 0
    after, _ = G.compute(src)  # knobs now come from the tuned bucket
    assert G.stats()["batch_width"] == best["batch_width"]
    assert np.array_equal(after.cpu().numpy().view(np.uint64), before.view(np.uint64))
    bc.tuning_cache(str(tmp_path / "t.json"), True)
    assert '"batch_width": %d' % best["batch_width"] in (tmp_path / "t.json").read_text()


# ----------------------------------------------------------------- multi-source BFS (bc_bfs)

def test_bfs_levels_and_sigma_match_oracle(bc):
    g = bcgen.disjoint_union(bcgen.rmat(12, 8, 1), bcgen.path(5))  # unreachable parts and isolated vertices
    G = bc.Graph(g.off, g.adj)
    src = bcgen.sample_sources(g, 70, 3)  # a 64-wide batch and a ragged 6-source one
    src = np.concatenate([src, src[:2]])  # repeated sources get their own rows
    lev, sig, _, st = G.bfs(src)
    assert st == bc.BC_OK
    lev, sig = lev.cpu().numpy(), sig.cpu().numpy()
    for i, s in enumerate(src):
        d = oracle.source_detail(g.off, g.adj, int(s))
        assert np.array_equal(lev[i], d["level"]), i
        assert np.array_equal(sig[i], np.where(d["level"] >= 0, d["sigma"], 0.0)), i


def test_bfs_extended_range_and_errors(bc):
    g = bcgen.grid(150, 150, 0.0)
    G = bc.Graph(g.off, g.adj)
    src = np.array([0, 150 * 75 + 75], np.int32)
    lev, mant, ex, st = G.bfs(src, exponent=True)
    assert st == bc.BC_W_SIGMA_INEXACT
    lev, mant, ex = lev.cpu().numpy(), mant.cpu().numpy(), ex.cpu().numpy()
    for i, s in enumerate(src):
        olev, omant, oex, _ = oracle.source_sigma_split(g.off, g.adj, int(s))
        assert np.array_equal(lev[i], olev)
        rel = np.abs(mant[i] * np.ldexp(1.0, ex[i] - oex) - omant) / omant
        assert rel.max() <= 1e-12
    with pytest.raises(bc.BCError):
        G.bfs(np.array([g.n], np.int32))
    lev0, _, _, st0 = G.bfs(np.zeros(0, np.int32))
    assert st0 == bc.BC_OK and lev0.numel() == 0


# ----------------------------------------------------------------- directed graphs

@pytest.fixture(scope="module")
def directed_rmat():
    g = bcgen.orient(bcgen.rmat(11, 8, 1), 5, 0.3)
    return g, oracle.bc(g.off, g.adj, np.arange(g.n))


def test_directed_relabel_matches_oracle(bc, directed_rmat):
    g, _ = directed_rmat
    G = bc.Graph(g.off, g.adj, directed=True)
    perm, off, adj = G.export()
    operm, _, ooff, oadj = oracle.relabel(g.off, g.adj)
    assert np.array_equal(perm, operm) and np.array_equal(off, ooff) and np.array_equal(adj, oadj)


@pytest.mark.parametrize("kw", [dict(batch_width=1), dict(batch_width=32), dict(batch_width=64),
                                dict(batch_width=128), dict(batch_width=64, direction=1),
                                dict(batch_width=64, direction=2)],
                         ids=lambda kw: "-".join(f"{k}{v}" for k, v in kw.items()))
def test_directed_all_sources(bc, directed_rmat, kw):
    g, want = directed_rmat
    G = bc.Graph(g.off, g.adj, directed=True)
    got, st = G.compute(np.arange(g.n, dtype=np.int32), **kw)
    assert st == bc.BC_OK
    assert_bc_close(got.cpu().numpy(), want)


def test_directed_bitwise_across_forms_and_heavy_rows(bc):
    g = bcgen.orient(bcgen.rmat(14, 64, 3), 2, 0.5)  # rows above 1024 out-arcs and in-arcs
    assert int(np.diff(g.off).max()) > 2 * 1024
    src = bcgen.sample_sources(g, 96, 4)
    want = oracle.bc(g.off, g.adj, src)
    G = bc.Graph(g.off, g.adj, directed=True)
    ref = None
    for kw in (dict(batch_width=64), dict(batch_width=32, direction=1), dict(batch_width=128, direction=2),
               dict(batch_width=1), dict(batch_width=64, teams=3)):
        got, st = G.compute(src, **kw)
        got = got.cpu().numpy()
        assert_bc_close(got, want)
        if ref is None:
            ref = got
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), kw


def test_directed_closed_forms_and_bfs(bc):
    n = 200
    dpath = bcgen.directed_csr(n, np.arange(n - 1), np.arange(1, n))
    got, _ = bc.Graph(dpath.off, dpath.adj, directed=True).compute(np.arange(n, dtype=np.int32))
    assert_bc_close(got.cpu().numpy(), [i * (n - 1 - i) for i in range(n)], rel=1e-12)
    dcyc = bcgen.directed_csr(n, np.arange(n), (np.arange(n) + 1) % n)
    got, _ = bc.Graph(dcyc.off, dcyc.adj, directed=True).compute(np.arange(n, dtype=np.int32))
    assert_bc_close(got.cpu().numpy(), [(n - 1) * (n - 2) / 2] * n, rel=1e-12)
    g = bcgen.orient(bcgen.disjoint_union(bcgen.rmat(10, 8, 2), bcgen.path(4)), 3, 0.2)
    src = bcgen.sample_sources(g, 40, 6)
    lev, sig, _, _ = bc.Graph(g.off, g.adj, directed=True).bfs(src)
    lev, sig = lev.cpu().numpy(), sig.cpu().numpy()
    for i, s in enumerate(src):
        d = oracle.source_detail(g.off, g.adj, int(s))
        assert np.array_equal(lev[i], d["level"]) and np.array_equal(sig[i], np.where(d["level"] >= 0, d["sigma"], 0))


def test_directed_invalid_inputs(bc):
    g = bcgen.directed_csr(4, [0, 1, 2], [1, 2, 3])
    with pytest.raises(bc.BCError):  # a directed CSR is not symmetric
        bc.Graph(g.off, g.adj)
    dup = (np.array([0, 2, 2, 2, 2], np.int32), np.array([1, 1], np.int32))
    with pytest.raises(bc.BCError):
        bc.Graph(*dup, directed=True)
    loop = (np.array([0, 1, 1], np.int32), np.array([0], np.int32))
    with pytest.raises(bc.BCError):
        bc.Graph(*loop, directed=True)


def test_directed_long_in_row_sum_beyond_64_bits(bc):
    """A sink with 4000 in-arcs from vertices of sigma = 2^53: its count 4000 * 2^53
    passes 2^64.  Whole in-rows are summed unchunked, so the per-term bound that
    sends the batch to the extended form must leave room for 4000 terms."""
    L, M = 53, 4000
    src, dst = [0, 0], [1, 2]
    layer = lambda i: (1 + 2 * (i - 1), 2 + 2 * (i - 1))  # layer i in 1..L: sigma = 2^(i-1)
    for i in range(1, L):
        for a in layer(i):
            for b in layer(i + 1):
                src.append(a); dst.append(b)
    mid0 = 1 + 2 * L
    sink = mid0 + M
    for k in range(M):
        for a in layer(L):
            src.append(a); dst.append(mid0 + k)  # sigma(mid) = 2 * 2^(L-1) = 2^53
        src.append(mid0 + k); dst.append(sink)
    g = bcgen.directed_csr(sink + 1, np.array(src), np.array(dst))
    G = bc.Graph(g.off, g.adj, directed=True)
    lev, mant, ex, st = G.bfs(np.array([0], np.int32), exponent=True)
    assert st == bc.BC_W_SIGMA_INEXACT
    got = np.ldexp(float(mant[0, sink].item()), int(ex[0, sink].item()))
    assert got == M * 2.0 ** 53 and int(lev[0, sink].item()) == L + 2
    out, st = G.compute(np.array([0, 1, 2], np.int32), batch_width=32)
    assert st == bc.BC_W_SIGMA_INEXACT and G.stats()["ext_batches"] > 0
    assert_bc_close(out.cpu().numpy(), oracle.bc_ld(g.off, g.adj, np.array([0, 1, 2])).astype(np.float64))


# ----------------------------------------------------------------- PageRank (computePR)

@pytest.mark.parametrize("gname", ["rmat12", "directed", "isolated"])
def test_pagerank_matches_oracle_sweep_for_sweep(bc, gname):
    g = {"rmat12": lambda: bcgen.rmat(12, 8, 1),
         "directed": lambda: bcgen.orient(bcgen.rmat(11, 16, 2), 3, 0.3),  # has vertices without out-arcs
         "isolated": lambda: bcgen.disjoint_union(bcgen.rmat(10, 4, 4), bcgen.empty_graph(7), bcgen.star(40))}[gname]()
    G = bc.Graph(g.off, g.adj, directed=(gname == "directed"))
    for k in (1, 2, 17):
        got, it, diff = G.pagerank(0.85, 0.0, k)  # beta 0: exactly k sweeps unless a fixed point is hit
        want, oit, odiff = oracle.pagerank(g.off, g.adj, 0.85, 0.0, k)
        assert it == oit
        assert_bc_close(got.cpu().numpy(), want)
        assert abs(diff - odiff) <= 1e-9 * max(odiff, 1e-300) or odiff == 0.0


def test_pagerank_convergence_repeatability_and_errors(bc):
    g = bcgen.rmat(13, 16, 2)
    G = bc.Graph(g.off, g.adj)
    a, it, diff = G.pagerank(0.85, 1e-10, 500)
    want, oit, _ = oracle.pagerank(g.off, g.adj, 0.85, 1e-10, 500)
    assert diff <= 1e-10 and abs(it - oit) <= 1
    assert_bc_close(a.cpu().numpy(), want, rel=1e-8)
    b, it2, diff2 = G.pagerank(0.85, 1e-10, 500)
    assert it2 == it and diff2 == diff
    assert np.array_equal(a.cpu().numpy().view(np.uint64), b.cpu().numpy().view(np.uint64))
    assert abs(float(a.sum().item()) - float(want.sum())) < 1e-12  # isolated vertices leak rank, as in the listing
    grid = bcgen.grid(40, 40, 0.0)  # every vertex has out-arcs: the rank mass stays 1
    r, _, _ = bc.Graph(grid.off, grid.adj).pagerank(0.85, 1e-12, 1000)
    assert abs(float(r.sum().item()) - 1.0) < 1e-12
    for bad in (dict(delta=1.5), dict(beta=-1.0), dict(max_iter=0)):
        with pytest.raises(bc.BCError):
            G.pagerank(**bad)


# ----------------------------------------------------------------- depth limit (levels are 16-bit)

def test_deepest_supported_and_too_deep_paths(bc):
    n = 65000  # depth 64999 from an end: inside the 65534-level limit
    g = bcgen.path(n)
    G = bc.Graph(g.off, g.adj)
    out, st = G.compute(np.array([0], np.int32))
    assert st == bc.BC_OK
    want = np.array([0.0] + [float(n - 1 - v) for v in range(1, n - 1)] + [0.0])  # delta_0(v) = n - 1 - v
    assert np.array_equal(out.cpu().numpy(), want)
    assert G.stats()["max_levels"] == n
    deep = bcgen.path(70000)
    D = bc.Graph(deep.off, deep.adj)
    with pytest.raises(bc.BCError) as ei:
        D.compute(np.array([0], np.int32))
    assert ei.value.status == bc.BC_E_LIMIT
    # the middle source is only 35000 deep: fine, and the library stays usable
    s0, nd = 35000, deep.n
    mid, st = D.compute(np.array([s0], np.int32))
    v = np.arange(nd, dtype=np.float64)
    want_mid = np.where(v < s0, v, nd - 1 - v)  # vertices beyond v, seen from s0
    want_mid[s0] = 0.0
    assert st == bc.BC_OK and np.array_equal(mid.cpu().numpy(), want_mid)
    got, _ = G.compute(np.array([n - 1], np.int32))
    assert np.array_equal(got.cpu().numpy(), want[::-1])
