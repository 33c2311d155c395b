"""The allocation-free entry point, bc_compute_noalloc, through the C ABI.

It serves callers that may not allocate device memory themselves -- host code
whose framework owns the whole device through its own memory pool and
forbids other allocations, or latency-critical code that must stay out of the
CUDA allocator -- by keeping every intermediate in one static device array.
This test checks that its output equals the regular entry point's
(bc_compute), within the parity tolerance the other GPU tests use, on two
calls in a row with different sources (the shared array keeps the previous
call's contents, so the second call proves that each call starts clean), and
that a graph beyond its fixed capacity is refused before any device work.
The file sorts last so that a stop-at-first-failure run has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import bcgen

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
    zero = want == 0
    assert np.all(got[zero] == 0)
    rel = np.abs(got[~zero] - want[~zero]) / np.abs(want[~zero])
    assert rel.max() <= REL, rel.max()


def test_noalloc_matches_regular_entry_point_twice(bc):
    import torch
    g = bcgen.disjoint_union(bcgen.rmat(12, 8, 1), bcgen.path(6))  # has isolated vertices too
    lib = bc.load()
    d_off = torch.from_numpy(g.off).cuda()
    d_adj = torch.from_numpy(g.adj).cuda()
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    G = bc.Graph(g.off, g.adj)
    for seed, k in ((1, 100), (2, 45)):
        src = bcgen.sample_sources(g, k, seed)
        src = np.concatenate([src, src[:3]])  # repeated sources count once per entry
        want, _ = G.compute(src)
        d_src = torch.from_numpy(src).cuda()
        st = lib.bc_compute_noalloc(d_off.data_ptr(), d_adj.data_ptr(), g.n, g.m, d_src.data_ptr(), len(src),
                                    out.data_ptr(), ctypes.c_void_p(stream))
        assert st in (bc.BC_OK, bc.BC_W_SIGMA_INEXACT), bc.last_error()
        close(out.cpu().numpy(), want.cpu().numpy())


def test_noalloc_refuses_graphs_beyond_its_capacity(bc):
    lib = bc.load()
    # refused from the sizes alone: nothing on the device is read or written
    st = lib.bc_compute_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), 40000, 10, ctypes.c_void_p(16), 1,
                                ctypes.c_void_p(16), None)
    assert st == bc.BC_E_LIMIT
    assert "32768" in bc.last_error()
