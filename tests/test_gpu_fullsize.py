"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark times, on outputs the oracle can compute in bounded time.

* 1024x1024 grid with 5% of edges removed: all 256 sampled sources at the
  benchmark's tuned batch width (extended form: counts reach ~2^2040), against
  the long-double oracle; the plain per-source form must agree bit for bit.
* R-MAT scale 22, edge factor 16: the benchmark's first 128-source batch
  (K = 128, the width the benchmark runs; the first 128 of its 4096 sources
  once grouped by hub distances, as bc_compute groups them) against the oracle
  on the host cores; three of its batches (the first two and the last of
  the grouped order) in one call on two teams, as the benchmark runs its 32;
  and the benchmark's whole 4096-source call by its BC sum (against the
  oracle's breadth-first path-length sums) and its exact zeros.
* The 2000-graph pool of uneven R-MAT graphs: sampled items (the smallest
  graph, the largest all-sources graph, the largest graph) recorded into one
  plan as the benchmark records the pool, each against the oracle.
* Serving over the R-MAT scale 14-22 pool: a second of Poisson requests at
  50 req/s, every request checked for success, sampled requests against the
  oracle.

Same tolerance as tests/test_gpu_parity.py: 1e-9 relative per vertex, exact
zeros exact.
"""
import os

import numpy as np
import pytest

import bcgen
import oracle

pytestmark = pytest.mark.gpu

REL = 1e-9
THREADS = max(1, min(os.cpu_count() or 1, 64))


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


def test_grid_1024_all_256_sources(bc):
    g = bcgen.grid(1024, 1024, 0.05, 1)
    src = bcgen.sample_sources(g, 256, 1)
    G = bc.Graph(g.off, g.adj)
    out, st = G.compute(src)  # the benchmark's call: the library picks its per-source form here
    assert st == bc.BC_W_SIGMA_INEXACT
    assert G.stats()["deep_sources"] == 256
    got = out.cpu().numpy().copy()
    assert_bc_close(got, oracle.bc_ld(g.off, g.adj, src).astype(np.float64))
    for kw in (dict(batch_width=32), dict(batch_width=1)):  # the batched and plain forms: the same bits
        other, st2 = G.compute(src, **kw)
        assert st2 == st and G.stats()["deep_sources"] == 0
        assert np.array_equal(other.cpu().numpy().view(np.uint64), got.view(np.uint64)), kw


def test_rmat22_first_benchmark_batch(bc):
    from grouping import grouped_order
    g = bcgen.rmat(22, 16, 1)
    G = bc.Graph(g.off, g.adj)
    allsrc = bcgen.sample_sources(g, 4096, 1)
    src = allsrc[grouped_order(g, G.export()[0], allsrc, threads=THREADS)][:128]  # the benchmark groups its sources
    out, st = G.compute(src, batch_width=128)
    assert st == bc.BC_OK
    assert G.stats()["batches"] == 1
    assert_bc_close(out.cpu().numpy(), oracle.bc(g.off, g.adj, src, threads=THREADS))


def test_rmat22_batches_on_two_teams_with_the_last_grouped_batch(bc):
    # the benchmark's call runs its 32 batches on 2 teams, batches adding into BC
    # in batch order through a turn counter: here 3 batches on 2 teams, the
    # first two of the grouped order and its last one
    from grouping import grouped_order
    g = bcgen.rmat(22, 16, 1)
    G = bc.Graph(g.off, g.adj)
    allsrc = bcgen.sample_sources(g, 4096, 1)
    order = grouped_order(g, G.export()[0], allsrc, threads=THREADS)
    src = np.concatenate([allsrc[order[:256]], allsrc[order[-128:]]])
    out, st = G.compute(src, batch_width=128, teams=2)  # 384 sources: grouped again, the same relative order
    assert st == bc.BC_OK
    s = G.stats()
    assert s["batches"] == 3 and s["teams"] == 2
    assert_bc_close(out.cpu().numpy(), oracle.bc(g.off, g.adj, src, threads=THREADS))


def test_rmat22_benchmark_call_sums_and_zeros(bc):
    # the benchmark's whole call (4096 grouped sources, 32 batches of 128 on two
    # teams) checked by properties that hold at any size: the raw BC summed over
    # all vertices is the sum over sources of (d(s,t) - 1) over reached t (the
    # oracle's breadth-first distances), and a vertex of degree at most 1 lies
    # inside no shortest path
    g = bcgen.rmat(22, 16, 1)
    G = bc.Graph(g.off, g.adj)
    src = bcgen.sample_sources(g, 4096, 1)
    out, st = G.compute(src)
    assert st == bc.BC_OK
    s = G.stats()
    assert s["batches"] == 32 and s["batch_width"] == 128 and s["teams"] == 2
    got = out.cpu().numpy()
    want = float(oracle.sum_dm1_bits(g.off, g.adj, src, threads=THREADS).sum())
    assert abs(got.sum() - want) <= 1e-9 * want
    assert np.all(got >= 0)
    assert np.all(got[np.diff(g.off) <= 1] == 0)


def test_pool_of_2000_sampled_items_in_one_plan(bc):
    import torch
    pool = bcgen.rmat_sizes_pool(2000, seed=1)
    ns = np.array([n for n, _, _ in pool])
    small = int(np.argmin(ns))
    all_src = int(np.argmax(np.where(ns <= 16384, ns, -1)))
    large = int(np.argmax(ns))
    items, want = [], []
    for i in (small, all_src, large):
        n, ef, sd = pool[i]
        g = bcgen.rmat_n(n, ef, sd)
        src = np.arange(g.n, dtype=np.int32) if g.n <= 16384 else bcgen.sample_sources(g, 256, sd)
        out = torch.empty(max(g.n, 1), dtype=torch.float64, device="cuda")
        items.append((bc.Graph(g.off, g.adj), src, out))
        want.append(oracle.bc(g.off, g.adj, src, threads=THREADS))
    plan = bc.ManyPlan(items)
    st = plan.run()
    assert all(int(s) in (bc.BC_OK, bc.BC_W_SIGMA_INEXACT) for s in st)
    for (G, _, out), w in zip(items, want):
        assert_bc_close(out.cpu().numpy()[: G.n], w)
    plan.close()


def test_serving_pool_14_to_22_sampled_requests(bc):
    import torch
    pool = [bcgen.rmat(s, 16, 1) for s in range(14, 23)]
    Gs = [bc.Graph(g.off, g.adj) for g in pool]
    reqs = bcgen.poisson_requests(50.0, 1.0, len(pool), seed=1)
    srcs = [bcgen.sample_sources(pool[gi], k, 100 + i) for i, (_, gi, k) in enumerate(reqs)]
    outs = [torch.empty(pool[gi].n, dtype=torch.float64, device="cuda") for _, gi, _ in reqs]
    jobs = [Gs[gi].submit(s, o) for (_, gi, _), s, o in zip(reqs, srcs, outs)]
    for j in jobs:
        assert j.wait(600000) is not None
    # sampled: requests the oracle finishes quickly (by source-arcs), one on the largest graph
    work = np.array([len(s) * pool[gi].m for s, (_, gi, _) in zip(srcs, reqs)], dtype=np.float64)
    picks = [int(i) for i in np.argsort(work)[:6]]
    biggest = [i for i, (_, gi, _) in enumerate(reqs) if gi == len(pool) - 1]
    if biggest:
        picks.append(min(biggest, key=lambda i: len(srcs[i])))
    for i in picks:
        _, gi, _ = reqs[i]
        g = pool[gi]
        assert_bc_close(outs[i].cpu().numpy(), oracle.bc(g.off, g.adj, srcs[i], threads=THREADS))
