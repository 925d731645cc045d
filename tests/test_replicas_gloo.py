"""World-size-2 gloo tests (CPU) of the multi-GPU path.

The hot path shards without any data-path collective: replicas each run a
whole layer, and a layer's output channels are independent (output ct
o = m*B + b needs only the weights of channel m).  These tests check, with two
CPU ranks: (1) the timing aggregation used by bench.py (barrier, max over
ranks, whole-job throughput); (2) that sharding a layer's output channels
across ranks and concatenating reproduces the unsharded result (computed with
the oracle on each rank, so no GPU is needed)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    from oracle import conv
    from paper_2506_11586_gb300 import replicas
    from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, Stream, uniform_residues

    r, w, _ = replicas.init(backend="gloo")
    assert (r, w) == (rank, world)
    replicas.barrier()
    mx = replicas.reduce_max(1.5 + rank)
    thr = replicas.whole_job_throughput(100.0, w, mx)

    # output-channel sharding of a small layer, oracle on each rank
    C_, H, W, M, N = 5, 7, 7, 4, 4096
    moduli = CANONICAL_PRIMES[:2]
    s = Stream(3, 0)
    K = s.int8(M * C_ * 9).astype(np.int64).reshape(M, C_, 3, 3)
    p = conv.canonical_partition(C_, H, W, M, 3, 3, 1, N)
    ct = uniform_residues(Stream(4, 0), moduli, (p.I, 2), N)
    Kp = conv.pack_weights(K, p)
    ks = np.arange(0, N, 97, dtype=np.uint32)
    mine = [o for o in range(p.O) if (o // p.B) % w == r]   # channel m -> rank m % world
    part = conv.conv_ct_pt(ct, Kp, p, moduli, ks=ks, outputs=mine)
    gathered = [None] * w
    dist.all_gather_object(gathered, (mine, part))
    if r == 0:
        full = conv.conv_ct_pt(ct, Kp, p, moduli, ks=ks)
        merged = np.zeros_like(full)
        for outs, arr in gathered:
            merged[outs] = arr
        q.put(("ok", mx, thr, bool(np.array_equal(merged, full))))
    replicas.barrier()
    replicas.shutdown()


def test_two_rank_aggregation_and_sharding():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    status, mx, thr, equal = q.get(timeout=10)
    assert status == "ok"
    assert mx == pytest.approx(2.5)
    assert thr == pytest.approx(100.0 * 2 / 2.5)
    assert equal
