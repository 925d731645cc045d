"""GPU tests of the request loop (hc_server_*): continuous batching of conv
requests over resident weights with admission by a device-memory budget.
Every request's result equals, bit for bit, the same layer run alone on the
same input (hc_conv_ct_pt_host), whatever else was in flight; one result is
also checked against the oracle's schoolbook convolution (Sec. 6.2)."""
import threading

import numpy as np
import pytest

from gpu_util import sample_indices
from oracle import conv
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream, uniform_residues

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (C, H, W, M, kh, kw, pad, N, L)
SHAPES = [
    (8, 12, 12, 6, 3, 3, 1, 8192, 3),
    (16, 9, 9, 12, 1, 1, 0, 8192, 3),
    (5, 20, 20, 4, 3, 3, 1, 16384, 4),
    (24, 7, 7, 40, 1, 1, 0, 16384, 4),
]


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_11586_gb300 import _lib
    from paper_2506_11586_gb300.build import build
    build()
    return _lib


@pytest.fixture(scope="module")
def layers(L):
    ctxs = {(N, nl): L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN) for N, nl in ((8192, 3), (16384, 4))}
    out = []
    for i, (C_, H, W, M, kh, kw, pad, N, nl) in enumerate(SHAPES):
        ctx = ctxs[(N, nl)]
        K = Stream(60 + i, 1).int8(M * C_ * kh * kw).astype(np.int64).reshape(M, C_, kh, kw)
        w = L.hc_weights_preprocess(ctx, L.make_desc(C_, H, W, M, kh, kw, pad=pad), K.astype(np.int8))
        p = conv.canonical_partition(C_, H, W, M, kh, kw, pad, N)
        out.append(dict(ctx=ctx, w=w, K=K, p=p, nl=nl, N=N))
    return out


def _input(ly, seed):
    return uniform_residues(Stream(seed, 9), CANONICAL_PRIMES[:ly["nl"]], (ly["w"].I, 2), ly["N"])


def _alone(L, ly, ct):
    out = np.zeros((ly["w"].O, 2, ly["nl"], ly["N"]), dtype=np.uint64)
    L.hc_conv_ct_pt_host(ly["ctx"], ly["w"], np.ascontiguousarray(ct), out)
    return out


# stream slots, and whether smaller ring degrees run at higher stream priority
@pytest.mark.parametrize("inflight,flags", [(2, 0), (4, 0), (4, 1)])
def test_mixed_requests_equal_alone(L, layers, inflight, flags):
    srv = L.hc_server_create(budget_bytes=2 << 30, max_batch=16, max_inflight=inflight, flags=flags)
    ids = [L.hc_server_add_layer(srv, ly["ctx"], ly["w"]) for ly in layers]
    order = Stream(5, 77).below(len(layers), 48)
    reqs = []
    for j, li in enumerate(order):
        ly = layers[int(li)]
        ct = _input(ly, 1000 + j)
        h_out = np.zeros((ly["w"].O, 2, ly["nl"], ly["N"]), dtype=np.uint64) if j % 2 == 0 else None
        reqs.append((int(li), ct, h_out))
    tickets = [None] * len(reqs)

    def submit(part):                      # two submitting threads interleave
        for j in part:
            li, ct, h_out = reqs[j]
            tickets[j] = L.hc_server_submit(srv, ids[li], ct, h_out)

    th = [threading.Thread(target=submit, args=(range(k, len(reqs), 2),)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for j, (li, ct, h_out) in enumerate(reqs):
        info = L.hc_server_wait(srv, tickets[j], 60.0)
        assert info["status"] == L.HC_OK and info["latency_ms"] >= info["queue_ms"] >= 0.0
        got = h_out
        if got is None:
            got = np.zeros((layers[li]["w"].O, 2, layers[li]["nl"], layers[li]["N"]), dtype=np.uint64)
            L.hc_server_fetch(srv, tickets[j], got)
            assert L.hc_server_result(srv, tickets[j]) != 0
        assert np.array_equal(got, _alone(L, layers[li], ct)), j
        L.hc_server_release(srv, tickets[j])
    st = L.hc_server_stats_get(srv)
    assert st["submitted"] == st["completed"] == len(reqs)
    assert st["max_batch_seen"] > 1 and st["batches"] < len(reqs)       # requests were batched
    assert st["bytes_in_use"] == 0 and st["peak_bytes_in_use"] <= st["pool_bytes"]
    assert st["products"] == sum(layers[li]["p"].products for li, _, _ in reqs)
    # one result against the oracle's schoolbook convolution
    ly = layers[0]
    ct = _input(ly, 4242)
    t = L.hc_server_submit(srv, ids[0], ct)
    L.hc_server_wait(srv, t)
    got = np.zeros((ly["w"].O, 2, ly["nl"], ly["N"]), dtype=np.uint64)
    L.hc_server_fetch(srv, t, got)
    ks = sample_indices(ly["N"], 16, 8)
    want = conv.conv_ct_pt(ct, conv.pack_weights(ly["K"], ly["p"]), ly["p"], CANONICAL_PRIMES[:ly["nl"]], ks)
    assert np.array_equal(got[..., ks], want)
    L.hc_server_release(srv, t)
    L.hc_server_shutdown(srv)


def test_budget_admission(L, layers):
    ly = layers[3]                          # 16384 / 4 limbs: 1 MiB per ciphertext
    need = (2 * ly["w"].I + ly["w"].O) * 2 * 4 * 16384 * 8
    srv = L.hc_server_create(budget_bytes=2 * need + 4096, max_batch=8, max_inflight=2)
    lid = L.hc_server_add_layer(srv, ly["ctx"], ly["w"])
    cts = [_input(ly, 2000 + j) for j in range(10)]
    outs = [np.zeros((ly["w"].O, 2, 4, 16384), dtype=np.uint64) for _ in cts]
    tickets = [L.hc_server_submit(srv, lid, c, o) for c, o in zip(cts, outs)]
    for t in tickets:
        assert L.hc_server_wait(srv, t, 60.0)["status"] == L.HC_OK
        L.hc_server_release(srv, t)
    st = L.hc_server_stats_get(srv)
    assert st["peak_bytes_in_use"] <= 2 * need + 4096 and st["completed"] == 10
    for c, o in zip(cts, outs):
        assert np.array_equal(o, _alone(L, ly, c))
    # a request that alone exceeds the pool is refused at submission
    small = L.hc_server_create(budget_bytes=need // 2, max_batch=4, max_inflight=1)
    lid2 = L.hc_server_add_layer(small, ly["ctx"], ly["w"])
    with pytest.raises(L.HcError) as e:
        L.hc_server_submit(small, lid2, cts[0])
    assert e.value.status == L.HC_ERR_BUDGET
    assert L.hc_server_stats_get(small)["refused"] == 1
    L.hc_free(small)
    L.hc_free(srv)


def test_results_held_until_release(L, layers):
    """Pool-resident results keep their memory until released; queued requests
    wait for it, then run."""
    ly = layers[2]
    need = (2 * ly["w"].I + ly["w"].O) * 2 * 4 * 16384 * 8
    srv = L.hc_server_create(budget_bytes=need + 1024, max_batch=4, max_inflight=1)
    lid = L.hc_server_add_layer(srv, ly["ctx"], ly["w"])
    a, b = _input(ly, 1), _input(ly, 2)
    ta = L.hc_server_submit(srv, lid, a)
    L.hc_server_wait(srv, ta)
    tb = L.hc_server_submit(srv, lid, b)
    with pytest.raises(L.HcError) as e:      # b cannot be admitted while a's result holds the pool
        L.hc_server_wait(srv, tb, 0.5)
    assert e.value.status == L.HC_ERR_TIMEOUT
    got_a = np.zeros((ly["w"].O, 2, 4, 16384), dtype=np.uint64)
    L.hc_server_fetch(srv, ta, got_a)
    L.hc_server_release(srv, ta)
    L.hc_server_wait(srv, tb, 60.0)
    got_b = np.zeros_like(got_a)
    L.hc_server_fetch(srv, tb, got_b)
    L.hc_server_release(srv, tb)
    assert np.array_equal(got_a, _alone(L, ly, a)) and np.array_equal(got_b, _alone(L, ly, b))
    with pytest.raises(L.HcError):
        L.hc_server_release(srv, tb)         # released once only
    L.hc_free(srv)


def test_batch_timeout_reported_per_request(L, layers):
    """A bounded device wait that runs out inside a batch (the server's self-test
    wait, which nothing completes) makes every request of that batch complete
    with HC_ERR_TIMEOUT and uncounted products; the error goes to the batch's
    own slot word, so the contexts' flags stay clean, and a server without the
    self-test on the same layers still returns exact results."""
    bad = L.hc_server_create(budget_bytes=1 << 30, max_batch=8, max_inflight=2, selftest_wait_limit=64)
    ids = [L.hc_server_add_layer(bad, ly["ctx"], ly["w"]) for ly in layers[:2]]
    tickets = [L.hc_server_submit(bad, ids[j % 2], _input(layers[j % 2], 3000 + j)) for j in range(4)]
    for t in tickets:
        assert L.hc_server_wait(bad, t, 60.0)["status"] == L.HC_ERR_TIMEOUT
        L.hc_server_release(bad, t)
    st = L.hc_server_stats_get(bad)
    assert st["completed"] == 4 and st["products"] == 0
    L.hc_free(bad)
    for ly in layers[:2]:
        L.hc_ctx_device_status(ly["ctx"])           # the contexts' own flags were never touched
    good = L.hc_server_create(budget_bytes=1 << 30, max_batch=8, max_inflight=2)
    lid = L.hc_server_add_layer(good, layers[0]["ctx"], layers[0]["w"])
    ct = _input(layers[0], 3100)
    out = np.zeros((layers[0]["w"].O, 2, layers[0]["nl"], layers[0]["N"]), dtype=np.uint64)
    t = L.hc_server_submit(good, lid, ct, out)
    assert L.hc_server_wait(good, t, 60.0)["status"] == L.HC_OK
    L.hc_server_release(good, t)
    assert np.array_equal(out, _alone(L, layers[0], ct))
    L.hc_free(good)
