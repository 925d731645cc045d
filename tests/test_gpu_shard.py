"""Output-channel shards of a layer through the library (hc_weights_preprocess_range):
the metric 56x56x64 -> 64 layer (N = 8192, L = 3) run as two shards one after
the other on one GPU, and a strided layer as three uneven shards, must
concatenate, output ciphertext for output ciphertext, to the unsharded layer's
output bit for bit (the sharded multi-GPU form: each GPU holds its channels'
weights and a copy of the inputs, and writes its own outputs)."""
import numpy as np
import pytest

from paper_2506_11586_gb300.inputs import (CANONICAL_PRIMES, CONV_56x56x64, T_PLAIN, Stream, conv_tensors,
                                           uniform_residues)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_11586_gb300 import _lib
    from paper_2506_11586_gb300.build import build
    build()
    return _lib


def _sharded_equals_whole(L, ctx, desc, K, nl, N, world, seed):
    from paper_2506_11586_gb300 import replicas
    w = L.hc_weights_preprocess(ctx, desc, K)
    ct = uniform_residues(Stream(seed, 0), CANONICAL_PRIMES[:nl], (w.I, 2), N)
    d_in = torch.from_numpy(ct.view(np.int64)).cuda()
    whole = torch.empty(w.O * 2 * nl * N, dtype=torch.int64, device="cuda")
    L.hc_conv_ct_pt(ctx, w, d_in, whole)
    B = w.O // desc.M
    parts = []
    for r in range(world):
        m0, m1 = replicas.channel_shard(desc.M, world, r)
        ws = L.hc_weights_preprocess_range(ctx, desc, K, m0, m1)
        assert ws.I == w.I and ws.O == (m1 - m0) * B           # same inputs, its own outputs
        out = torch.full((ws.O * 2 * nl * N,), -1, dtype=torch.int64, device="cuda")
        L.hc_conv_ct_pt(ctx, ws, d_in, out)
        parts.append(out)
    torch.cuda.synchronize()
    return bool(torch.equal(torch.cat(parts), whole))


def test_metric_layer_as_two_shards(L):
    sh, N, nl = CONV_56x56x64, 8192, 3
    _, K = conv_tensors(sh, seed=2)
    ctx = L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    desc = L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad)
    assert _sharded_equals_whole(L, ctx, desc, K, nl, N, 2, 500)


def test_strided_layer_as_three_uneven_shards(L):
    N, nl = 4096, 2
    ctx = L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    desc = L.make_desc(6, 15, 13, 7, 3, 3, pad=1, stride=2)
    K = Stream(501, 1).int8(7 * 6 * 9).reshape(7, 6, 3, 3)
    assert _sharded_equals_whole(L, ctx, desc, K, nl, N, 3, 502)


def test_bad_ranges_are_rejected(L):
    ctx = L.hc_ctx_create(4096, CANONICAL_PRIMES[:2], T_PLAIN)
    desc = L.make_desc(4, 6, 6, 5, 3, 3, pad=1)
    K = np.zeros((5, 4, 3, 3), dtype=np.int8)
    for m0, m1 in ((3, 3), (4, 2), (0, 6)):
        with pytest.raises(L.HcError) as e:
            L.hc_weights_preprocess_range(ctx, desc, K, m0, m1)
        assert e.value.status == L.HC_ERR_INVALID_ARG
