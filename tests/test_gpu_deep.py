"""GPU parity of the per-source form for graphs of large diameter (deep.cu).

The per-source form runs each source alone in one block with the batched
traversal's arithmetic and order of summation (extended-form path counts
summed over in-neighbours in CSR order, per 1024-arc chunk on heavy
undirected rows; rho sums over out-neighbours in CSR order; dependencies
added to BC in source-list order), so its BC must equal the batched form's
bit for bit, and the oracle within the parity tolerance of the batched tests.
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


def close(got, want, rel=REL):
    zero = want == 0
    assert np.all(got[zero] == 0), "exact zeros must stay zero"
    err = np.abs(got - want) / np.maximum(np.abs(want), 1e-300)
    assert np.all(err[~zero] <= rel), f"max rel err {err[~zero].max()}"


def both_forms(bc, G, src, **kw):
    out, st_deep = G.compute(src, deep_form=2, **kw)
    deep = out.cpu().numpy().copy()
    s_deep = G.stats()
    out, st_b = G.compute(src, deep_form=1, **kw)
    batched = out.cpu().numpy().copy()
    s_b = G.stats()
    assert st_deep == st_b
    assert s_deep["deep_sources"] == len(src) and s_b["deep_sources"] == 0
    assert np.array_equal(deep.view(np.uint64), batched.view(np.uint64))
    assert s_deep["max_levels"] == s_b["max_levels"]
    assert s_deep["dag_arcs"] == s_b["dag_arcs"] and s_deep["reached"] == s_b["reached"]
    return deep, st_deep


@pytest.mark.parametrize("g", [bcgen.grid(64, 64, 0.05, 3), bcgen.random_tree(3000, 2),
                               bcgen.disjoint_union(bcgen.path(300), bcgen.empty_graph(5), bcgen.cycle(401),
                                                    bcgen.grid(20, 30, 0.1, 4)),
                               bcgen.rmat(12, 8, 1)], ids=lambda g: g.name)
def test_deep_form_equals_batched_and_oracle(bc, g):
    src = bcgen.sample_sources(g, 150, 7)
    src = np.concatenate([src, src[:5]])  # repeated sources count once per occurrence
    G = bc.Graph(g.off, g.adj)
    got, st = both_forms(bc, G, src)
    if g.name.startswith("grid64"):  # corner-to-corner counts near C(126, 63) ~ 2^122
        assert st == bc.BC_W_SIGMA_INEXACT
        close(got, oracle.bc_ld(g.off, g.adj, src).astype(np.float64))
    else:
        assert st == bc.BC_OK
        close(got, oracle.bc(g.off, g.adj, src))


def test_deep_form_blocks_reused_across_sources(bc):
    """One block per SM: every block runs several sources in turn on the same slices."""
    g = bcgen.grid(40, 50, 0.05, 9)
    src = np.arange(g.n, dtype=np.int32)
    G = bc.Graph(g.off, g.adj)
    got, st = both_forms(bc, G, src, blocks_per_sm=1)
    assert G.stats()["grid_blocks"] < len(src)
    close(got, oracle.bc_ld(g.off, g.adj, src).astype(np.float64))


def test_deep_form_extended_range(bc):
    """Path counts up to C(238,119) ~ 2^233 on a full grid: the extended form, in both forms."""
    g = bcgen.grid(120, 120, 0.0)
    src = np.array([0, 121, 120 * 60 + 60, g.n - 1], np.int32)
    G = bc.Graph(g.off, g.adj)
    got, st = both_forms(bc, G, src)
    assert st == bc.BC_W_SIGMA_INEXACT
    close(got, oracle.bc_ld(g.off, g.adj, src).astype(np.float64))


def test_deep_form_heavy_rows(bc):
    """Rows above 1024 arcs: chunked sums in the same chunk order as the batched form."""
    g = bcgen.rmat(14, 32, 2)
    assert int(np.diff(g.off).max()) > 2 * 1024
    src = bcgen.sample_sources(g, 70, 3)
    G = bc.Graph(g.off, g.adj)
    got, st = both_forms(bc, G, src)
    close(got, oracle.bc(g.off, g.adj, src))


def test_deep_form_directed(bc):
    g = bcgen.orient(bcgen.rmat(13, 48, 3), 2, 0.5)  # heavy out-rows and in-rows
    assert int(np.diff(g.off).max()) > 1024
    src = bcgen.sample_sources(g, 80, 4)
    G = bc.Graph(g.off, g.adj, directed=True)
    got, st = both_forms(bc, G, src)
    close(got, oracle.bc(g.off, g.adj, src))
    n = 500
    dpath = bcgen.directed_csr(n, np.arange(n - 1), np.arange(1, n))
    D = bc.Graph(dpath.off, dpath.adj, directed=True)
    got, _ = both_forms(bc, D, np.arange(n, dtype=np.int32))
    close(got, np.array([i * (n - 1 - i) for i in range(n)], np.float64), rel=1e-12)


def test_deep_form_closed_forms_and_limit(bc):
    n = 65000  # depth 64999 from an end: inside the 65534-level limit
    g = bcgen.path(n)
    G = bc.Graph(g.off, g.adj)
    out, st = G.compute(np.array([0], np.int32), deep_form=2)
    assert st == bc.BC_OK and G.stats()["max_levels"] == n
    want = np.array([0.0] + [float(n - 1 - v) for v in range(1, n - 1)] + [0.0])
    assert np.array_equal(out.cpu().numpy(), want)
    deep = bcgen.path(70000)
    D = bc.Graph(deep.off, deep.adj)
    with pytest.raises(bc.BCError) as ei:
        D.compute(np.array([0], np.int32), deep_form=2)
    assert ei.value.status == bc.BC_E_LIMIT
    s0, nd = 35000, deep.n
    mid, st = D.compute(np.array([s0], np.int32), deep_form=2)
    v = np.arange(nd, dtype=np.float64)
    want_mid = np.where(v < s0, v, nd - 1 - v)
    want_mid[s0] = 0.0
    assert st == bc.BC_OK and np.array_equal(mid.cpu().numpy(), want_mid)
    with pytest.raises(bc.BCError) as ei:
        G.compute(np.array([0, n], np.int32), deep_form=2)
    assert ei.value.status == bc.BC_E_SOURCE
    with pytest.raises(bc.BCError):
        G.compute(np.array([0], np.int32), deep_form=3)


def test_automatic_form_choice(bc):
    """Auto: a sparse graph whose probe finds 48+ narrow levels runs per source; shallow ones stay batched."""
    g = bcgen.grid(300, 300, 0.05, 5)  # about 600 levels from the probe's vertex
    src = bcgen.sample_sources(g, 128, 2)
    G = bc.Graph(g.off, g.adj)
    out, st = G.compute(src)
    auto = out.cpu().numpy().copy()
    s = G.stats()
    assert s["deep_sources"] == len(src) and s["max_levels"] >= 300
    out, _ = G.compute(src, deep_form=1)
    assert np.array_equal(auto.view(np.uint64), out.cpu().numpy().view(np.uint64))
    out, _ = G.compute(src, batch_width=64)  # a width given by the caller keeps the batched form
    assert G.stats()["deep_sources"] == 0
    tree = bcgen.random_tree(20000, 3)  # hundreds of levels of a few dozen vertices
    T = bc.Graph(tree.off, tree.adj)
    T.compute(bcgen.sample_sources(tree, 100, 2))
    assert T.stats()["deep_sources"] == 100
    rng = np.random.default_rng(4)  # sparse random graph: about 20 levels
    sparse = bcgen.edges_to_csr(20000, rng.integers(0, 20000, 30000), rng.integers(0, 20000, 30000))
    S = bc.Graph(sparse.off, sparse.adj)
    S.compute(bcgen.sample_sources(sparse, 128, 2))
    assert S.stats()["deep_sources"] == 0 and S.stats()["max_levels"] < 48
    r = bcgen.rmat(12, 8, 1)  # dense enough that no probe runs
    R = bc.Graph(r.off, r.adj)
    R.compute(bcgen.sample_sources(r, 128, 2))
    assert R.stats()["deep_sources"] == 0


def test_bfs_on_deep_graphs_runs_per_source(bc):
    """bc_bfs on a deep graph takes the per-source form (forward only): the batched form's bits."""
    g = bcgen.grid(100, 100, 0.05, 6)
    src = bcgen.sample_sources(g, 80, 3)
    G = bc.Graph(g.off, g.adj)
    lev, mant, ex, st = G.bfs(src, exponent=True)
    assert st == bc.BC_W_SIGMA_INEXACT  # corner-to-corner counts near C(198, 99)
    assert G.stats()["deep_sources"] == len(src)
    lev, mant, ex = lev.cpu().numpy(), mant.cpu().numpy(), ex.cpu().numpy()
    for i in range(0, len(src), 8):
        olev, omant, oex, _ = oracle.source_sigma_split(g.off, g.adj, int(src[i]))
        assert np.array_equal(lev[i], olev)
        reached = olev >= 0
        assert np.all(mant[i][~reached] == 0) and np.all(ex[i][~reached] == 0)
        rel = np.abs(mant[i][reached] * np.ldexp(1.0, ex[i][reached] - oex[reached]) - omant[reached]) / omant[reached]
        assert rel.max() <= 1e-12
    # fewer than 64 sources on a graph of unknown depth: the batched form, the same bits
    B = bc.Graph(g.off, g.adj)
    blev, bmant, bex, bst = B.bfs(src[:40], exponent=True)
    assert B.stats()["deep_sources"] == 0 and bst == st
    assert np.array_equal(blev.cpu().numpy(), lev[:40])
    assert np.array_equal(bmant.cpu().numpy().view(np.uint64), mant[:40].view(np.uint64))
    assert np.array_equal(bex.cpu().numpy(), ex[:40])
    _, sig, _, _ = G.bfs(src, exponent=False)
    C = bc.Graph(g.off, g.adj)
    _, bsig, _, _ = C.bfs(src[:40], exponent=False)
    assert np.array_equal(bsig.cpu().numpy().view(np.uint64), sig.cpu().numpy()[:40].view(np.uint64))


def test_deep_form_rounds_and_epoch_wrap(bc):
    """More than 2^15 sources per block: two rounds, and the 16-bit epochs wrap (records cleared)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 5
    g = bcgen.path(n)
    reps = (sms * 65536 + 1000 + n - 1) // n
    src = np.tile(np.arange(n, dtype=np.int32), reps)  # every vertex `reps` times
    G = bc.Graph(g.off, g.adj)
    out, st = G.compute(src, deep_form=2, blocks_per_sm=1)
    s = G.stats()
    assert st == bc.BC_OK and s["deep_sources"] == len(src) and s["grid_blocks"] == sms
    assert s["kernel_launches"] >= 7  # mapping, two rounds of (traversal, row sum), the records' clearing
    want = np.array([2.0 * i * (n - 1 - i) * reps for i in range(n)])  # ordered pairs with i strictly between
    assert np.array_equal(out.cpu().numpy(), want)


def test_deep_form_allocation_failure_then_recovers(bc):
    """The per-source form's buffers come from the allocator hook: a refusal is BC_E_NOMEM, and the graph
    stays usable (the next call, with the default allocator, gives the batched form's bits)."""
    import ctypes
    lib = bc.load()
    g = bcgen.grid(30, 30, 0.05, 8)
    src = bcgen.sample_sources(g, 70, 5)
    G = bc.Graph(g.off, g.adj)
    ref, st = G.compute(src, deep_form=1)  # the call's own buffers exist from here on
    ref = ref.cpu().numpy().copy()
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    asked, freed = [], []
    hooks = (ALLOC(lambda nbytes, stream, ctx: asked.append(int(nbytes))),  # returns None: no memory
             FREE(lambda ptr, stream, ctx: freed.append(ptr)))
    assert lib.bc_set_allocator(ctypes.cast(hooks[0], ctypes.c_void_p), ctypes.cast(hooks[1], ctypes.c_void_p),
                                None) == bc.BC_OK
    try:
        with pytest.raises(bc.BCError) as ei:
            G.compute(src, deep_form=2)
        assert ei.value.status == bc.BC_E_NOMEM
        assert asked and not freed
    finally:
        assert lib.bc_set_allocator(None, None, None) == bc.BC_OK
    out, st2 = G.compute(src, deep_form=2)
    assert st2 == st and G.stats()["deep_sources"] == len(src)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), ref.view(np.uint64))


def test_plan_runs_deep_items_per_source(bc):
    """A many-graph plan with a deep item: that item runs in the per-source form at each replay,
    the others from the recorded graph; every output equals the direct call bit for bit."""
    import torch
    graphs = [bcgen.rmat(11, 8, 3), bcgen.grid(200, 200, 0.05, 7), bcgen.random_tree(5000, 4)]
    items, refs = [], []
    for i, g in enumerate(graphs):
        src = bcgen.sample_sources(g, 100, 11 + i)
        out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        items.append((bc.Graph(g.off, g.adj), src, out))
        R = bc.Graph(g.off, g.adj)
        ref, _ = R.compute(src)
        refs.append((ref.cpu().numpy().copy(), R.stats()["deep_sources"]))
    assert refs[0][1] == 0 and refs[1][1] == 100 and refs[2][1] == 100  # R-MAT batched, grid and tree per source
    plan = bc.ManyPlan(items)
    for _ in range(2):
        st = plan.run()
        assert all(int(x) in (bc.BC_OK, bc.BC_W_SIGMA_INEXACT) for x in st)
        for (G, src, out), (ref, _) in zip(items, refs):
            assert np.array_equal(out.cpu().numpy().view(np.uint64), ref.view(np.uint64))
    close(items[2][2].cpu().numpy(), oracle.bc(graphs[2].off, graphs[2].adj, items[2][1]))


def test_serving_deep_graph_jobs_equal_direct_calls(bc):
    """Jobs served on a graph known to be deep run through the direct call (per-source form):
    each result equals the direct call bit for bit, alone or with other jobs in the queue."""
    import torch
    g = bcgen.grid(150, 150, 0.05, 12)
    G = bc.Graph(g.off, g.adj)
    G.compute(bcgen.sample_sources(g, 80, 1))  # learns the depth (a probe, then the per-source form)
    assert G.stats()["deep_sources"] == 80
    lists = [bcgen.sample_sources(g, k, 20 + k) for k in (5, 70, 130, 33)]
    refs = []
    for src in lists:
        ref, _ = G.compute(src)
        refs.append(ref.cpu().numpy().copy())
    outs = [torch.empty(g.n, dtype=torch.float64, device="cuda") for _ in lists]
    jobs = [G.submit(src, out) for src, out in zip(lists, outs)]
    for job, out, ref in zip(jobs, outs, refs):
        st, lat = job.wait(60000)
        assert st in (bc.BC_OK, bc.BC_W_SIGMA_INEXACT) and lat >= 0
        assert np.array_equal(out.cpu().numpy().view(np.uint64), ref.view(np.uint64))
    close(outs[0].cpu().numpy(), oracle.bc_ld(g.off, g.adj, lists[0]).astype(np.float64))


@pytest.mark.parametrize("g", [bcgen.empty_graph(1), bcgen.path(2), bcgen.path(3), bcgen.star(6),
                               bcgen.disjoint_union(bcgen.empty_graph(3), bcgen.path(2))], ids=lambda g: g.name)
def test_deep_form_tiny_graphs(bc, g):
    src = np.arange(g.n, dtype=np.int32)
    G = bc.Graph(g.off, g.adj)
    got, st = both_forms(bc, G, src)
    assert st == bc.BC_OK
    assert np.array_equal(got, oracle.bc(g.off, g.adj, src))
