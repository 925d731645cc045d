"""World-size-2 gloo tests (CPU) of the multi-GPU path.

Replicas each run whole layers (no data-path collective); a sharded layer
splits its output channels, which are independent (output ct o = m*B + b
needs only the weights of channel m), with one broadcast of the inputs.  These tests check, with two
CPU ranks: (1) the timing aggregation used by bench.py (barrier, max over
ranks, whole-job throughput); (2) the sharded layer's host logic: contiguous
channel ranges that tile the layer (replicas.channel_shard), the broadcast of
the input ciphertexts from one rank (replicas.broadcast_inputs), and that the
ranks' output ranges concatenate to the unsharded result (computed with the
oracle on each rank, so no GPU is needed; the library's shards,
hc_weights_preprocess_range, are checked on the GPU in test_gpu_shard.py)."""
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

    # output-channel shards of a small layer: rank 0 holds the input ciphertexts and
    # broadcasts them (the sharded layer's one exchange), each rank computes its own
    # contiguous channel range [m0, m1) = output ciphertexts [m0*B, m1*B) (oracle on
    # each rank, so no GPU is needed), and the gathered ranges tile the whole output
    C_, H, W, M, N = 5, 7, 7, 5, 4096
    moduli = CANONICAL_PRIMES[:2]
    s = Stream(3, 0)
    K = s.int8(M * C_ * 9).astype(np.int64).reshape(M, C_, 3, 3)
    p = conv.canonical_partition(C_, H, W, M, 3, 3, 1, N)
    import torch
    ct_t = torch.zeros((p.I, 2, len(moduli), N), dtype=torch.int64)
    if r == 0:
        ct_t.copy_(torch.from_numpy(uniform_residues(Stream(4, 0), moduli, (p.I, 2), N).view(np.int64)))
    replicas.broadcast_inputs(ct_t, src=0)
    ct = ct_t.numpy().view(np.uint64)
    Kp = conv.pack_weights(K, p)
    ks = np.arange(0, N, 97, dtype=np.uint32)
    m0, m1 = replicas.channel_shard(M, w, r)
    mine = list(range(m0 * p.B, m1 * p.B))
    part = conv.conv_ct_pt(ct, Kp, p, moduli, ks=ks, outputs=mine)
    gathered = [None] * w
    dist.all_gather_object(gathered, ((m0, m1), mine, part))
    if r == 0:
        full = conv.conv_ct_pt(uniform_residues(Stream(4, 0), moduli, (p.I, 2), N), Kp, p, moduli, ks=ks)
        merged = np.zeros_like(full)
        ranges = sorted(g[0] for g in gathered)
        tiles = ranges[0][0] == 0 and ranges[-1][1] == M and all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        for _, outs, arr in gathered:
            merged[outs] = arr
        q.put(("ok", mx, thr, bool(np.array_equal(merged, full)) and tiles))
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


def test_channel_shards_tile_the_layer():
    from paper_2506_11586_gb300 import replicas
    for M in range(1, 40):
        for world in range(1, 9):
            ranges = [replicas.channel_shard(M, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == M
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
