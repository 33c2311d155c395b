"""Pins for the CPU oracle: brute force, closed forms, invariants, special cases.

Each check ties the oracle to something other than itself -- explicit
shortest-path enumeration, textbook closed forms, scipy's independent BFS
distances, exact integer binomials -- so that a dropped term, a wrong sign or
index, or a swapped operand in ``oracle/brandes.c`` fails at least one test.

Convention (paper's computeBC, Appendix A): the oracle returns the raw sum
over the listed sources of the per-source dependency, with no halving.  For an
undirected graph with every vertex listed as a source, raw = 2 x the
unordered-pair betweenness that the closed forms below state.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import bcgen
import oracle

REL = 1e-12


def all_src(g):
    return np.arange(g.n, dtype=np.int32)


def close(a, b, rel=REL, abs_=1e-12):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.all(np.abs(a - b) <= rel * np.abs(b) + abs_)


def dist_matrix(g):
    A = sp.csr_matrix((np.ones(g.m), g.adj, g.off), shape=(g.n, g.n))
    return shortest_path(A, unweighted=True, directed=False)


# ---------------------------------------------------------------- brute force

SMALL = ([bcgen.gnp(n, p, seed) for n in (5, 6, 7, 8) for p in (0.3, 0.5, 0.8) for seed in (1, 2)]
         + [bcgen.path(6), bcgen.star(6), bcgen.cycle(7), bcgen.cycle(8), bcgen.complete(5),
            bcgen.complete_bipartite(2, 4), bcgen.random_tree(8, 3), bcgen.grid(2, 4),
            bcgen.disjoint_union(bcgen.path(3), bcgen.cycle(4)), bcgen.empty_graph(3)])


@pytest.mark.parametrize("g", SMALL, ids=lambda g: g.name)
def test_bc_matches_brute_force_all_sources(g):
    want = oracle.brute_force_bc(g.off, g.adj, range(g.n))
    got = oracle.bc(g.off, g.adj, all_src(g))
    assert close(got, [float(x) for x in want])
    got_ld = oracle.bc_ld(g.off, g.adj, all_src(g))
    assert close(got_ld.astype(np.float64), [float(x) for x in want])


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_bc_matches_brute_force_source_subset_with_duplicates(seed):
    g = bcgen.gnp(8, 0.45, seed)
    srcs = np.array([3, 1, 3, 7, 0], dtype=np.int32)  # 3 appears twice: counted twice
    want = oracle.brute_force_bc(g.off, g.adj, srcs)
    got = oracle.bc(g.off, g.adj, srcs)
    assert close(got, [float(x) for x in want])


@pytest.mark.parametrize("g", SMALL[:12], ids=lambda g: g.name)
def test_levels_and_sigma_match_enumeration(g):
    for s in range(g.n):
        lv, sg = oracle.brute_force_sigma(g.off, g.adj, s)
        d = oracle.source_detail(g.off, g.adj, s)
        assert list(d["level"]) == lv
        assert [int(x) for x in d["sigma"]] == sg


def test_no_sources_gives_zero():
    g = bcgen.gnp(7, 0.5, 1)
    assert np.all(oracle.bc(g.off, g.adj, np.zeros(0, np.int32)) == 0)


def test_source_out_of_range_rejected():
    g = bcgen.path(4)
    with pytest.raises(ValueError):
        oracle.bc(g.off, g.adj, np.array([4], np.int32))


# ---------------------------------------------------------------- closed forms
# unordered-pair betweenness, so the raw all-source oracle value is twice these.

@pytest.mark.parametrize("n", [2, 3, 7, 40, 501])
def test_path(n):
    g = bcgen.path(n)
    got = oracle.bc(g.off, g.adj, all_src(g)) / 2
    want = [i * (n - 1 - i) for i in range(n)]
    assert close(got, want)


@pytest.mark.parametrize("n", [3, 4, 9, 300])
def test_star(n):
    g = bcgen.star(n)
    got = oracle.bc(g.off, g.adj, all_src(g)) / 2
    want = [(n - 1) * (n - 2) / 2] + [0] * (n - 1)
    assert close(got, want)


@pytest.mark.parametrize("n", [2, 3, 6, 33])
def test_complete(n):
    g = bcgen.complete(n)
    assert np.all(oracle.bc(g.off, g.adj, all_src(g)) == 0)


@pytest.mark.parametrize("n", [3, 4, 5, 8, 11, 64, 101])
def test_cycle(n):
    g = bcgen.cycle(n)
    got = oracle.bc(g.off, g.adj, all_src(g)) / 2
    want = (n - 1) * (n - 3) / 8 if n % 2 else (n - 2) ** 2 / 8
    assert close(got, np.full(n, want))


@pytest.mark.parametrize("a,b", [(1, 5), (2, 3), (3, 3), (4, 7), (10, 13)])
def test_complete_bipartite(a, b):
    g = bcgen.complete_bipartite(a, b)
    got = oracle.bc(g.off, g.adj, all_src(g)) / 2
    want = [math.comb(b, 2) / a] * a + [math.comb(a, 2) / b] * b
    assert close(got, want)


def tree_bc_half(g):
    """Unordered-pair BC of a tree: sum over pairs of components of T - v of |Ci||Cj|,
    from subtree sizes of an iterative DFS rooted at 0."""
    n = g.n
    parent = np.full(n, -1)
    order = []
    seen = np.zeros(n, bool)
    stack = [0]
    seen[0] = True
    while stack:
        v = stack.pop()
        order.append(v)
        for w in g.adj[g.off[v]:g.off[v + 1]]:
            if not seen[w]:
                seen[w] = True
                parent[w] = v
                stack.append(w)
    size = np.ones(n, dtype=np.int64)
    for v in reversed(order):
        if parent[v] >= 0:
            size[parent[v]] += size[v]
    out = np.zeros(n)
    for v in range(n):
        comps = [int(size[w]) for w in g.adj[g.off[v]:g.off[v + 1]] if parent[w] == v]
        if parent[v] >= 0:
            comps.append(n - int(size[v]))
        s1 = sum(comps)
        s2 = sum(c * c for c in comps)
        out[v] = (s1 * s1 - s2) // 2
    return out


@pytest.mark.parametrize("n,seed", [(2, 1), (10, 1), (200, 2), (3000, 3)])
def test_random_tree(n, seed):
    g = bcgen.random_tree(n, seed)
    got = oracle.bc(g.off, g.adj, all_src(g)) / 2
    assert close(got, tree_bc_half(g))


@pytest.mark.parametrize("R,C", [(3, 4), (6, 6), (12, 9)])
def test_full_grid_sigma_is_binomial(R, C):
    g = bcgen.grid(R, C, 0.0)
    for s in [0, C + 1, R * C - 1, (R // 2) * C + C // 2]:
        d = oracle.source_detail(g.off, g.adj, s)
        sr, sc = divmod(s, C)
        for v in range(g.n):
            r, c = divmod(v, C)
            dx, dy = abs(r - sr), abs(c - sc)
            assert d["level"][v] == dx + dy
            assert int(d["sigma"][v]) == math.comb(dx + dy, dx)


def test_big_grid_sigma_long_double_binomial():
    """Path counts beyond 2^64 and beyond the double range: long double keeps them
    to about 1e-16 relative against exact integer binomials."""
    R = C = 600
    g = bcgen.grid(R, C, 0.0)
    s = 0
    level, mant, ex, delta = oracle.source_sigma_split(g.off, g.adj, s)
    for v in [1, 601, 599 * 600 + 599, 300 * 600 + 299, 599 * 600, 450 * 600 + 10]:
        r, c = divmod(v, C)
        exact = math.comb(r + c, r)
        # compare mant*2^ex with the exact integer via Fraction
        approx = Fraction(float(mant[v])) * (Fraction(2) ** int(ex[v]))
        assert abs(approx - exact) <= Fraction(1, 10**15) * exact
        assert level[v] == r + c
    assert math.comb(1198, 599) > 2**1024  # the corner's count leaves the double range


# ---------------------------------------------------------------- invariants

def test_per_source_delta_sum_equals_distance_sum_rmat12():
    g = bcgen.rmat(12, 8, 1)
    D = dist_matrix(g)
    srcs = bcgen.sample_sources(g, 48, 1)
    for s in srcs:
        d = oracle.source_detail(g.off, g.adj, int(s))
        row = D[s]
        reach = np.isfinite(row) & (np.arange(g.n) != s)
        want = int(np.sum(row[reach] - 1))
        assert abs(float(np.sum(d["delta"])) - d["delta"][s] - want) <= 1e-9 * max(want, 1)
        assert np.array_equal(np.where(np.isfinite(row), row, -1).astype(np.int32), d["level"])
        assert np.all(d["delta"] >= 0)
        assert np.all(d["sigma"][d["level"] == 1] == 1)


def test_all_pairs_bc_sum_equals_distance_sum():
    g = bcgen.rmat(10, 6, 5)
    D = dist_matrix(g)
    fin = np.isfinite(D) & (D > 0)
    want = np.sum(D[fin] - 1) / 2  # unordered connected pairs
    got = np.sum(oracle.bc(g.off, g.adj, all_src(g))) / 2
    assert abs(got - want) <= 1e-11 * want


def test_grid_dag_arcs_are_half_the_component_arcs():
    """A connected bipartite graph puts every edge between consecutive levels."""
    g = bcgen.grid(20, 17, 0.0)
    for s in [0, 5, 170]:
        d = oracle.source_detail(g.off, g.adj, s)
        assert d["reached"] == g.n and d["edag"] * 2 == g.m


@pytest.mark.parametrize("g", [bcgen.rmat(10, 8, 3), bcgen.grid(20, 23, 0.1, 4),
                               bcgen.disjoint_union(bcgen.path(7), bcgen.star(9), bcgen.empty_graph(3)),
                               bcgen.orient(bcgen.rmat(9, 8, 2), seed=2)], ids=lambda g: g.name)
def test_sum_dm1_against_scipy_distances(g):
    # the BFS-only path-length sum, from scipy's own unweighted shortest paths
    a = sp.csr_matrix((np.ones(g.m), g.adj, g.off), shape=(g.n, g.n))
    src = np.concatenate([np.arange(0, g.n, 3), [0, 0]]).astype(np.int32)  # repeats count per entry
    d = shortest_path(a, directed=True, unweighted=True, indices=src)
    want = np.array([np.sum(np.where(np.isfinite(row) & (row > 0), row - 1, 0)) for row in d], dtype=np.int64)
    got = oracle.sum_dm1(g.off, g.adj, src, threads=3)
    assert np.array_equal(got, want)
    assert np.array_equal(oracle.sum_dm1_bits(g.off, g.adj, src, threads=2), want)
    many = np.resize(src, 150)  # several 64-source groups, the last ragged, over 2 threads
    assert np.array_equal(oracle.sum_dm1_bits(g.off, g.adj, many, threads=2), oracle.sum_dm1(g.off, g.adj, many))
    # summed over the sources it is the sum of the raw BC over all vertices
    assert oracle.bc(g.off, g.adj, src).sum() == pytest.approx(float(got.sum()), rel=1e-12)


def test_long_double_and_double_agree_where_counts_fit():
    g = bcgen.rmat(11, 8, 2)
    srcs = bcgen.sample_sources(g, 64, 3)
    a = oracle.bc(g.off, g.adj, srcs)
    b = oracle.bc_ld(g.off, g.adj, srcs).astype(np.float64)
    assert close(a, b, rel=1e-13)


def test_threaded_wrapper_matches_single_thread():
    g = bcgen.rmat(10, 8, 4)
    srcs = bcgen.sample_sources(g, 37, 2)
    assert close(oracle.bc(g.off, g.adj, srcs, threads=4), oracle.bc(g.off, g.adj, srcs), rel=1e-13)


def test_bc_is_invariant_under_relabelling():
    g = bcgen.rmat(10, 8, 7)
    perm, inv, noff, nadj = oracle.relabel(g.off, g.adj)
    a = oracle.bc(g.off, g.adj, all_src(g))
    b = oracle.bc(noff, nadj, all_src(g))
    assert close(b[inv], a, rel=1e-12)


# ---------------------------------------------------------------- ingest rules

def test_relabel_definition():
    g = bcgen.rmat(11, 8, 9)
    perm, inv, noff, nadj = oracle.relabel(g.off, g.adj)
    deg = g.degrees()
    assert np.array_equal(np.sort(perm), np.arange(g.n))
    assert np.array_equal(inv[perm], np.arange(g.n))
    # independent definition: lexsort by (-degree, id)
    want = np.lexsort((np.arange(g.n), -deg))
    assert np.array_equal(perm, want)
    # relabelled rows = mapped neighbour sets, sorted
    for r in range(0, g.n, 37):
        v = perm[r]
        assert np.array_equal(nadj[noff[r]:noff[r + 1]], np.sort(inv[g.adj[g.off[v]:g.off[v + 1]]]))
    assert np.all(np.diff(np.diff(noff)) <= 0)


def test_validate_codes():
    g = bcgen.cycle(5)
    assert oracle.validate(g.off, g.adj) == 0
    off = g.off.copy(); off[2] = off[1] - 1
    assert oracle.validate(off, g.adj) == 1
    adj = g.adj.copy(); adj[3] = 5
    assert oracle.validate(g.off, adj) == 2
    adj = g.adj.copy(); adj[0] = 0
    assert oracle.validate(g.off, adj) == 3
    adj = g.adj.copy(); adj[1] = adj[0]
    assert oracle.validate(g.off, adj) == 4
    # arc 0->1 kept, arc 1->0 replaced by 1->3: asymmetric (and duplicate-free)
    h = bcgen.path(4)
    adj = h.adj.copy(); adj[1] = 3
    assert oracle.validate(h.off, adj) == 5
    assert oracle.validate(h.off, adj, undirected=False) == 0


# ---------------------------------------------------------------- golden fixtures

def test_golden_small_graphs():
    from golden_io import load
    for rec in load():
        got = oracle.bc(rec["off"], rec["adj"], rec["src"])
        assert close(got, [float(x) for x in rec["bc"]]), rec["name"]


# ----------------------------------------------------------------- directed graphs (arcs followed one way)

def test_directed_brute_force_matches_oracle():
    """Shortest paths follow arcs; brute force counts s -> t paths through v."""
    from fractions import Fraction
    for seed in range(6):
        g = bcgen.orient(bcgen.gnp(8, 0.45, seed + 20), seed, 0.3)
        want = oracle.brute_force_bc(g.off, g.adj, range(g.n))
        got = oracle.bc(g.off, g.adj, np.arange(g.n))
        for v in range(g.n):
            assert abs(got[v] - float(want[v])) <= 1e-12 * max(1.0, float(want[v])), (seed, v)
        for s in range(g.n):
            lev, sig = oracle.brute_force_sigma(g.off, g.adj, s)
            d = oracle.source_detail(g.off, g.adj, s)
            assert np.array_equal(d["level"], np.array(lev)) and np.array_equal(d["sigma"], np.array(sig, float))


def test_directed_closed_forms():
    n = 11
    dpath = bcgen.directed_csr(n, np.arange(n - 1), np.arange(1, n))
    # ordered pairs s < i < t: i * (n - 1 - i); no halving for directed graphs
    assert np.array_equal(oracle.bc(dpath.off, dpath.adj, np.arange(n)), [i * (n - 1 - i) for i in range(n)])
    dcyc = bcgen.directed_csr(n, np.arange(n), (np.arange(n) + 1) % n)
    # every ordered pair has one path of length (t - s) mod n: each vertex is interior (n-1)(n-2)/2 times
    assert np.all(oracle.bc(dcyc.off, dcyc.adj, np.arange(n)) == (n - 1) * (n - 2) / 2)
    out_star = bcgen.directed_csr(n, np.zeros(n - 1, int), np.arange(1, n))
    assert np.all(oracle.bc(out_star.off, out_star.adj, np.arange(n)) == 0)
    # orienting with p_both = 1 keeps every arc: the undirected graph itself
    g = bcgen.rmat(8, 4, 2)
    both = bcgen.orient(g, 1, 1.0)
    assert np.array_equal(both.off, g.off) and np.array_equal(both.adj, g.adj)


# ----------------------------------------------------------------- PageRank (computePR)

def _transition(g):
    """Dense column-stochastic-like matrix M[v, u] = 1/outdeg(u) for each arc u -> v."""
    n = g.n
    M = np.zeros((n, n))
    deg = np.diff(g.off)
    for u in range(n):
        for e in range(g.off[u], g.off[u + 1]):
            M[g.adj[e], u] += 1.0 / deg[u]
    return M


def test_pagerank_sweeps_equal_dense_power_iteration():
    """k sweeps of the listing = k steps of x <- (1-d)/n + d M x from x = 1/n (dense algebra)."""
    for g in (bcgen.rmat(6, 4, 3), bcgen.orient(bcgen.gnp(30, 0.15, 2), 4, 0.3), bcgen.directed_csr(5, [0, 1, 2, 3], [1, 2, 3, 4])):
        M = _transition(g)
        x = np.full(g.n, 1.0 / g.n)
        for k in range(1, 12):
            x = (1 - 0.85) / g.n + 0.85 * (M @ x)
            pr, it, diff = oracle.pagerank(g.off, g.adj, 0.85, 0.0, k)
            assert it == k or (it < k and diff == 0.0)  # an exact fixed point stops the sweeps early
            assert np.allclose(pr, x, rtol=1e-13, atol=0)


def test_pagerank_fixed_point_and_closed_forms():
    g = bcgen.rmat(7, 6, 5)
    pr, it, diff = oracle.pagerank(g.off, g.adj, 0.85, 1e-14, 1000)
    assert diff <= 1e-14 and it < 1000
    n = g.n
    want = np.linalg.solve(np.eye(n) - 0.85 * _transition(g), np.full(n, 0.15 / n))
    assert np.allclose(pr, want, rtol=1e-11, atol=0)
    # no vertex without out-arcs: rank mass stays 1
    assert abs(pr.sum() - 1.0) < 1e-12 or np.any(np.diff(g.off) == 0)
    # a regular graph keeps the uniform start: one sweep, no change
    c = bcgen.cycle(50)
    pr, it, diff = oracle.pagerank(c.off, c.adj, 0.85, 1e-12, 100)
    assert it == 1 and diff < 1e-15 and np.allclose(pr, 1 / 50, rtol=1e-14)
    # undirected star: centre c, leaves l solve c = (1-d)/n + d (n-1) l, l = (1-d)/n + d c/(n-1)
    n, d = 41, 0.85
    s = bcgen.star(n)
    pr, _, _ = oracle.pagerank(s.off, s.adj, d, 1e-15, 5000)
    A = np.array([[1.0, -d * (n - 1)], [-d / (n - 1), 1.0]])
    cc, ll = np.linalg.solve(A, [(1 - d) / n, (1 - d) / n])
    assert np.isclose(pr[0], cc, rtol=1e-12) and np.allclose(pr[1:], ll, rtol=1e-12)


# ---------------------------------------------------------------- weighted BC (positive integer weights)

WSMALL = [g for g in SMALL if g.m > 0]


@pytest.mark.parametrize("g", WSMALL, ids=lambda g: g.name)
@pytest.mark.parametrize("wmax", [1, 3])
def test_weighted_bc_matches_brute_force(g, wmax):
    # weights 1..3 make many ties between paths of different hop counts
    wt = bcgen.edge_weights(g, 1, wmax, seed=g.n + wmax)
    want = oracle.brute_force_wbc(g.off, g.adj, wt, range(g.n))
    assert close(oracle.wbc(g.off, g.adj, wt, all_src(g)), [float(x) for x in want])


def test_weighted_sigma_and_dist_match_enumeration():
    g = bcgen.gnp(8, 0.6, 5)
    wt = bcgen.edge_weights(g, 1, 2, 9)
    for s in range(g.n):
        d = oracle.wsource_detail(g.off, g.adj, wt, s)
        for t in range(g.n):
            ps = oracle.weighted_shortest_paths(g.off, g.adj, wt, s, t)
            if t == s:
                assert d["dist"][t] == 0 and d["sigma"][t] == 1
            elif not ps:
                assert d["dist"][t] == -1 and d["sigma"][t] == 0
            else:
                w = sum(int(wt[e]) for a, b in zip(ps[0], ps[0][1:])
                        for e in range(g.off[a], g.off[a + 1]) if g.adj[e] == b)
                assert d["dist"][t] == w and d["sigma"][t] == len(ps)


@pytest.mark.parametrize("c", [1, 7])
def test_equal_weights_give_unweighted_bc(c):
    g = bcgen.rmat(10, 8, 3)
    wt = np.full(g.m, c, np.int32)
    src = bcgen.sample_sources(g, 200, 2)
    assert close(oracle.wbc(g.off, g.adj, wt, src), oracle.bc(g.off, g.adj, src))


def test_weight_scaling_leaves_bc_unchanged_bitwise():
    g = bcgen.rmat(9, 8, 4)
    wt = bcgen.edge_weights(g, 1, 20, 4)
    src = all_src(g)
    a = oracle.wbc(g.off, g.adj, wt, src)
    b = oracle.wbc(g.off, g.adj, wt * 3, src)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.parametrize("n,seed", [(50, 1), (400, 2)])
def test_tree_plus_heavy_edges_is_the_tree(n, seed):
    # a tree has unique paths whatever its weights; extra edges heavier than any
    # tree path never lie on a shortest path, so BC is the tree's closed form
    t = bcgen.random_tree(n, seed)
    twt = bcgen.edge_weights(t, 1, 9, seed)
    extra = bcgen.gnp(n, 0.02, seed + 10)
    deg = np.diff(t.off.astype(np.int64))
    u = np.concatenate([np.repeat(np.arange(n), deg), np.repeat(np.arange(n), np.diff(extra.off.astype(np.int64)))])
    v = np.concatenate([t.adj, extra.adj])
    heavy = 10 * n
    w = {}
    for a, b, x in zip(np.repeat(np.arange(n), deg), t.adj, twt):
        w[(int(a), int(b))] = int(x)
    g = bcgen.edges_to_csr(n, u, v)
    gdeg = np.diff(g.off.astype(np.int64))
    gw = np.array([w.get((int(a), int(b)), heavy) for a, b in zip(np.repeat(np.arange(n), gdeg), g.adj)], np.int32)
    got = oracle.wbc(g.off, g.adj, gw, all_src(g)) / 2
    assert close(got, tree_bc_half(t))


def test_weighted_path_closed_form():
    g = bcgen.path(30)
    wt = bcgen.edge_weights(g, 1, 50, 1)
    got = oracle.wbc(g.off, g.adj, wt, all_src(g)) / 2
    assert close(got, [i * (29 - i) for i in range(30)])


# ------------------------------------------------ weighted BC on directed graphs (per-arc weights)

WDIR = [bcgen.orient(g, seed=i + 3, p_both=0.3) for i, g in enumerate(WSMALL[:5])]


@pytest.mark.parametrize("g", WDIR, ids=lambda g: g.name)
def test_directed_weighted_bc_matches_brute_force(g):
    wt = bcgen.edge_weights(g, 1, 3, seed=g.n, per_arc=True)
    want = oracle.brute_force_wbc(g.off, g.adj, wt, range(g.n))
    assert close(oracle.wbc(g.off, g.adj, wt, all_src(g)), [float(x) for x in want])


def test_directed_weighted_chain_closed_form():
    # 0 -> 1 -> ... -> n-1: one path per ordered pair s < t, through every v between
    n = 40
    g = bcgen.directed_csr(n, np.arange(n - 1), np.arange(1, n))
    wt = bcgen.edge_weights(g, 1, 50, 2, per_arc=True)
    assert close(oracle.wbc(g.off, g.adj, wt, all_src(g)), [v * (n - 1 - v) for v in range(n)])


def test_directed_equal_weights_give_unweighted_bc():
    g = bcgen.orient(bcgen.rmat(10, 8, 5), seed=2)
    src = bcgen.sample_sources(g, 150, 3)
    assert close(oracle.wbc(g.off, g.adj, np.full(g.m, 4, np.int32), src), oracle.bc(g.off, g.adj, src))


def test_directed_weighted_reversal_over_all_sources():
    # every s -> t shortest path of G is a t -> s shortest path of its transpose
    # (arcs keep their weights), so the all-source sums agree
    g = bcgen.orient(bcgen.gnp(60, 0.08, 11), seed=5, p_both=0.2)
    wt = bcgen.edge_weights(g, 1, 4, 7, per_arc=True)
    deg = np.diff(g.off.astype(np.int64))
    u = np.repeat(np.arange(g.n), deg)
    order = np.lexsort((u, g.adj))  # arcs sorted by (head, tail): the transpose's CSR order
    r = bcgen.directed_csr(g.n, g.adj[order], u[order])
    rw = wt[order]
    assert np.array_equal(r.adj, u[order])
    assert close(oracle.wbc(r.off, r.adj, rw, all_src(r)), oracle.wbc(g.off, g.adj, wt, all_src(g)))
