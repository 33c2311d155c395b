"""Host logic of the multi-GPU form (one rank per GPU, sources sharded by rank,
no data-path collective): per-rank source lists and the max-over-ranks timing
of bench.py, run as two gloo ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    import bcgen
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = bcgen.rmat(10, 8, 1)
        src = bench.shard_sources(g, 64, rank, world)
        ms = 100.0 + 25.0 * rank  # this rank's own (fake) timed region
        slowest = bench.max_over_ranks(ms, dist, "cpu")
        rate = bench.aggregate_rate(world, len(src), g.m, slowest)
        np.savez(os.path.join(outdir, f"r{rank}.npz"), src=src, slowest=slowest, rate=rate, m=g.m)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_sources_and_take_the_slowest_time(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"r{i}.npz") for i in range(world)]
    import bcgen
    g = bcgen.rmat(10, 8, 1)
    # every rank has its own list of the same size, drawn as the generator defines
    assert len(r[0]["src"]) == len(r[1]["src"]) == 64
    assert not np.array_equal(r[0]["src"], r[1]["src"])
    assert np.array_equal(r[0]["src"], bcgen.sample_sources(g, 64, 1))
    assert np.array_equal(r[1]["src"], bcgen.sample_sources(g, 64, 2))
    # both ranks agree on the slowest time and report the whole-job rate
    assert float(r[0]["slowest"]) == float(r[1]["slowest"]) == 125.0
    want = world * 64 * int(r[0]["m"]) / 0.125
    assert float(r[0]["rate"]) == pytest.approx(want)


def test_one_rank_keeps_the_single_gpu_workload():
    import bcgen
    import bench
    g = bcgen.rmat(10, 8, 1)
    assert np.array_equal(bench.shard_sources(g, 32, 0, 1), bcgen.sample_sources(g, 32, 1))
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
