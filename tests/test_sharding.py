"""Host logic of the multi-GPU form, run as gloo ranks on the CPU.

One job's sources are split round-robin by batch over the ranks
(paper_2305_03317_b300.sharded), every rank computes a partial BC over its
batches, the ranks exchange statuses, all-gather the partials and sum them in
rank order.  Here the oracle stands in for the device step (each rank's
partial BC) and a left-to-right numpy sum for bc_reduce_ranks (whose kernel is
checked against that sum on the GPU in test_gpu_parity.py); the split, the
status exchange and the gather are the library's own code.  Also the
benchmark's max-over-ranks timing.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

REL = 1e-9
K = 32


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _job():
    import bcgen
    g = bcgen.rmat(10, 8, 1)
    return g, bcgen.sample_sources(g, 300, 1)  # 10 batches of 32, the last ragged


def rank_sum(rows):
    """The reduction's definition: rows added left to right in rank order."""
    acc = rows[0].copy()
    for r in rows[1:]:
        acc = acc + r
    return acc


def _split_main(rank, world, port, outdir):
    import torch
    import oracle
    from paper_2305_03317_b300 import sharded
    dist = _init(rank, world, port)
    try:
        g, src = _job()
        mine = sharded.shard_of(src, K, rank, world)
        part = oracle.bc(g.off, g.adj, mine)  # stand-in for this rank's bc_compute_ex
        st = sharded.exchange_statuses(0 if rank else 2, device="cpu")  # rank 0 reports a warning
        parts = sharded.gather_partials(torch.from_numpy(part)).numpy()
        np.savez(os.path.join(outdir, f"r{rank}.npz"), mine=mine, parts=parts, total=rank_sum(list(parts)),
                 status=st)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_split_one_job_and_sum_in_rank_order(tmp_path, world):
    mp = pytest.importorskip("torch.multiprocessing")
    import oracle
    from paper_2305_03317_b300 import sharded
    mp.spawn(_split_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"r{i}.npz") for i in range(world)]
    g, src = _job()
    # every batch of the job on exactly one rank, round-robin, whole batches in order
    nb = (len(src) + K - 1) // K
    for i in range(world):
        want = np.concatenate([src[b * K:(b + 1) * K] for b in range(i, nb, world)])
        assert np.array_equal(r[i]["mine"], want)
    assert sorted(np.concatenate([x["mine"] for x in r]).tolist()) == sorted(src.tolist())
    # the gathered rows are the ranks' partials, in rank order, on every rank
    for i in range(world):
        assert np.array_equal(r[i]["parts"], r[0]["parts"])
        assert np.array_equal(r[0]["parts"][i], oracle.bc(g.off, g.adj, r[i]["mine"]))
    # every rank holds the same bits, the rank-order sum of one process's emulation
    emul = rank_sum([oracle.bc(g.off, g.adj, sharded.shard_of(src, K, i, world)) for i in range(world)])
    for i in range(world):
        assert np.array_equal(r[i]["total"].view(np.uint64), emul.view(np.uint64))
        assert int(r[i]["status"]) == 2
    # and the job's BC within the parity tolerance
    want = oracle.bc(g.off, g.adj, src)
    zero = want == 0
    assert np.all(emul[zero] == 0)
    assert np.max(np.abs(emul[~zero] - want[~zero]) / want[~zero]) <= REL


def _fail_main(rank, world, port, outdir):
    from paper_2305_03317_b300 import sharded
    dist = _init(rank, world, port)
    try:
        st = sharded.exchange_statuses(-3 if rank == 1 else 0, device="cpu")  # rank 1's call failed
        np.save(os.path.join(outdir, f"s{rank}.npy"), np.array([st]))
    finally:
        dist.destroy_process_group()


def test_a_failed_rank_is_seen_by_every_rank_before_the_gather(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_fail_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    assert [int(np.load(tmp_path / f"s{i}.npy")[0]) for i in range(2)] == [-3, -3]


def test_shard_edge_cases():
    from paper_2305_03317_b300 import sharded
    order = np.arange(70, dtype=np.int32)
    assert sharded.shard_of(order, 32, 0, 4).tolist() == list(range(32))
    assert sharded.shard_of(order, 32, 2, 4).tolist() == list(range(64, 70))
    assert len(sharded.shard_of(order, 32, 3, 4)) == 0  # more ranks than batches: an empty share
    assert sharded.worst_status([0, 2, 0]) == 2
    assert sharded.worst_status([2, -5, -3]) == -5


def _timing_main(rank, world, port, outdir):
    import bench
    dist = _init(rank, world, port)
    try:
        ms = 100.0 + 25.0 * rank  # this rank's own (fake) timed region
        slowest = bench.max_over_ranks(ms, dist, "cpu")
        np.save(os.path.join(outdir, f"t{rank}.npy"), np.array([slowest]))
    finally:
        dist.destroy_process_group()


def test_benchmark_takes_the_slowest_rank(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_timing_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    assert [float(np.load(tmp_path / f"t{i}.npy")[0]) for i in range(2)] == [125.0, 125.0]
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
