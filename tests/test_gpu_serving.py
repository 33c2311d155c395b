"""Serving and failure handling on the GPU, through the C ABI.

* Admission by device memory: with a budget that admits one workspace at a
  time, jobs on different graphs run one after another (peak concurrency 1)
  and give the same bits as direct calls, within the oracle's tolerance; with
  room for several, they overlap.
* bc_cancel withdraws a queued job (its output untouched, its poll reports
  BC_E_CANCELLED) and leaves running or finished jobs alone.
* An allocator hook that returns NULL: the calls that need device memory
  report BC_E_NOMEM, nothing is left half-built, and once the default
  allocator is back the same graph and new graphs compute correct results.
All failures are made on the host (a budget, a cancel, a hook); no GPU fault.
"""
import ctypes

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
    zero = want == 0
    assert np.all(got[zero] == 0)
    err = np.abs(got[~zero] - want[~zero]) / want[~zero]
    assert err.max() <= rel, err.max()


def grow_to_three_slots(bc, budget):
    bc.server_config(3, budget)  # the slot count may only grow: 3 whatever earlier tests set


def test_admission_by_memory_one_workspace_at_a_time(bc):
    import torch
    graphs = [bcgen.rmat(14, 8, s) for s in (1, 2, 3)]
    Gs = [bc.Graph(g.off, g.adj) for g in graphs]
    srcs = [bcgen.sample_sources(g, 200, 7 + i) for i, g in enumerate(graphs)]
    direct = [G.compute(s)[0].cpu().numpy().copy() for G, s in zip(Gs, srcs)]

    def serve(budget):
        grow_to_three_slots(bc, budget)
        bc.server_reset_stats()
        outs = [torch.full((g.n,), -1.0, dtype=torch.float64, device="cuda") for g in graphs for _ in range(2)]
        jobs = [Gs[i // 2].submit(srcs[i // 2], outs[i]) for i in range(6)]
        for j in jobs:
            assert j.wait(600000)[0] == bc.BC_OK
        peak, done = bc.server_stats()
        return peak, done, [o.cpu().numpy() for o in outs]

    try:
        peak, done, outs = serve(1)  # one byte: a job is admitted only when nothing else runs
        assert peak == 1 and done == 6
        for i, got in enumerate(outs):
            assert np.array_equal(got.view(np.uint64), direct[i // 2].view(np.uint64))
        for i, (g, s) in enumerate(zip(graphs, srcs)):
            assert_bc_close(outs[2 * i], oracle.bc(g.off, g.adj, s))
        peak, done, outs = serve(1 << 50)  # room for every workspace: the three graphs' jobs overlap
        assert done == 6 and peak >= 2
        for i, got in enumerate(outs):
            assert np.array_equal(got.view(np.uint64), direct[i // 2].view(np.uint64))
    finally:
        grow_to_three_slots(bc, 1 << 50)


def test_cancel_withdraws_only_queued_jobs(bc):
    import torch
    big, small = bcgen.rmat(16, 16, 3), bcgen.rmat(10, 8, 4)
    Gb, Gs = bc.Graph(big.off, big.adj), bc.Graph(small.off, small.adj)
    try:
        grow_to_three_slots(bc, 1)  # one job at a time: the second waits behind the first
        ob = torch.empty(big.n, dtype=torch.float64, device="cuda")
        os_ = torch.full((small.n,), -1.0, dtype=torch.float64, device="cuda")
        sb, ss = bcgen.sample_sources(big, 1024, 1), bcgen.sample_sources(small, 64, 1)
        jb = Gb.submit(sb, ob)
        js = Gs.submit(ss, os_)
        assert js.cancel()  # still queued behind the running job
        with pytest.raises(bc.BCError) as ei:
            js.wait(600000)
        assert ei.value.status == bc.BC_E_CANCELLED
        assert jb.wait(600000)[0] == bc.BC_OK
        assert torch.all(os_ == -1.0)  # never written
        assert_bc_close(ob.cpu().numpy(), oracle.bc(big.off, big.adj, sb, threads=8))
        # once a job's final status has been read its id is released: unknown to bc_cancel
        j2 = Gs.submit(ss, os_)
        assert j2.wait(600000)[0] == bc.BC_OK
        assert bc.load().bc_cancel(j2.id) == bc.BC_E_INVALID_ARG
    finally:
        grow_to_three_slots(bc, 1 << 50)


def test_allocator_failure_reports_nomem_then_recovers(bc):
    lib = bc.load()
    g = bcgen.rmat(11, 8, 2)
    src = bcgen.sample_sources(g, 96, 2)
    G = bc.Graph(g.off, g.adj)  # built with the default allocator
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    asked, freed = [], []

    def no_memory(nbytes, stream, ctx):
        asked.append(int(nbytes))
        return None

    def no_free(ptr, stream, ctx):
        freed.append(ptr)  # nothing was allocated through this hook, so nothing may come back

    hooks = (ALLOC(no_memory), FREE(no_free))
    assert lib.bc_set_allocator(ctypes.cast(hooks[0], ctypes.c_void_p), ctypes.cast(hooks[1], ctypes.c_void_p),
                                None) == bc.BC_OK
    try:
        with pytest.raises(bc.BCError) as ei:
            bc.Graph(g.off, g.adj)
        assert ei.value.status == bc.BC_E_NOMEM
        with pytest.raises(bc.BCError) as ei:
            G.compute(src, batch_width=64)  # a first call at this width needs a workspace
        assert ei.value.status == bc.BC_E_NOMEM
        assert asked and not freed
    finally:
        assert lib.bc_set_allocator(None, None, None) == bc.BC_OK
    out, st = G.compute(src, batch_width=64)
    assert st == bc.BC_OK
    want = oracle.bc(g.off, g.adj, src)
    assert_bc_close(out.cpu().numpy(), want)
    G2 = bc.Graph(g.off, g.adj)
    out2, _ = G2.compute(src, batch_width=64)
    assert np.array_equal(out2.cpu().numpy().view(np.uint64), out.cpu().numpy().view(np.uint64))
