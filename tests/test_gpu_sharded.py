"""The multi-GPU job split on a real GPU, through NCCL, with one rank.

Every box here has one GPU, so the split runs as a one-rank NCCL process
group: the job's batch order from bc_source_batches, the device status
exchange, the NCCL all-gather of the partial BC and bc_reduce_ranks all run
as they do on N GPUs.  With one rank the share is the whole job in the order
a direct call uses, so the result equals bc_compute bit for bit (and the
oracle within the parity tolerance).  Runs in a child process so that the
process group never outlives the test.
"""
import os
import socket
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import torch
import torch.distributed as dist
import bcgen, oracle
import paper_2305_03317_b300 as bc
from paper_2305_03317_b300 import sharded
dist.init_process_group("nccl", rank=0, world_size=1)
torch.cuda.set_device(0)
try:
    g = bcgen.rmat(12, 8, 1)
    G = bc.Graph(g.off, g.adj)
    src = bcgen.sample_sources(g, 700, 9)
    direct, _ = G.compute(src)
    direct = direct.cpu().numpy().copy()
    out, st = sharded.compute(G, src)
    got = out.cpu().numpy()
    assert st == bc.BC_OK, st
    assert np.array_equal(got.view(np.uint64), direct.view(np.uint64))
    want = oracle.bc(g.off, g.adj, src)
    zero = want == 0
    assert np.all(got[zero] == 0)
    assert np.max(np.abs(got[~zero] - want[~zero]) / want[~zero]) <= 1e-9
    # a failing share (a source outside the graph) reaches the caller as the library's error
    try:
        sharded.compute(G, np.array([0, g.n], np.int32))
        raise AssertionError("expected BCError")
    except bc.BCError as e:
        assert e.status == bc.BC_E_SOURCE, e.status
    print("SHARDED_OK")
finally:
    dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_one_rank_nccl_split_equals_direct_call():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()), NCCL_NVLS_ENABLE="0")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "SHARDED_OK" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
