"""GPU parity of the server's step around the convolution (hc_conv_server_step:
share add, convolution, output mask, slot extraction; Sec. 7 and Sec. 6.2)
against the oracle, bit-exact, and end to end through BFV: the client's
decryption of every returned slot is conv(x_c + x_s) - r mod t."""
import numpy as np
import pytest

from gpu_util import sample_indices, to_dev, to_host
from oracle import bfv, conv
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, CONV_56x56x64, T_PLAIN, Stream, conv_tensors

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


def _case(C_, H, W, M, kh, kw, pad, N, nl, seed, part=None, x_c=None, K=None):
    s = Stream(seed, 41)
    p = conv.Partition(C_, H, W, M, kh, kw, pad, N, *part) if part else \
        conv.canonical_partition(C_, H, W, M, kh, kw, pad, N)
    params = bfv.Params(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    sk = s.ternary(N)
    if x_c is None:
        x_c = s.below(T_PLAIN, C_ * H * W).astype(np.int64).reshape(C_, H, W)
        K = s.int8(M * C_ * kh * kw).astype(np.int64).reshape(M, C_, kh, kw)
    x_s = s.below(T_PLAIN, C_ * H * W).astype(np.int64).reshape(C_, H, W)
    r = s.below(T_PLAIN, M * p.Ho * p.Wo).astype(np.int64).reshape(M, p.Ho, p.Wo)
    packed = conv.pack_input(x_c, p)
    ct = np.zeros((p.I, 2, nl, N), dtype=np.uint64)
    for i in range(p.I):
        a = np.stack([s.below(q, N) for q in params.moduli])
        ct[i] = bfv.encrypt(params, sk, packed[i], a, s.rounded_gaussian(N))
    return p, params, sk, x_c, x_s, np.asarray(K, dtype=np.int64), r, ct


def _run(L, p, params, K, ct, x_s, r):
    nl = len(params.moduli)
    ctx = L.hc_ctx_create(p.N, params.moduli, T_PLAIN)
    w = L.hc_weights_preprocess(ctx, L.make_desc(p.C, p.H, p.W, p.M, p.kh, p.kw, pad=p.pad, Cw=p.Cw, Hw=p.Hw,
                                                  Ww=p.Ww), K.astype(np.int8))
    S = L.slot_count(w)
    assert S == conv.slot_count(p)
    out = torch.empty(p.O * 2 * nl * p.N, dtype=torch.int64, device="cuda")
    slots = torch.empty(p.O * nl * S, dtype=torch.int64, device="cuda")
    L.hc_conv_server_step(ctx, w, to_dev(ct), to_dev(x_s.astype(np.uint64)), to_dev(r.astype(np.uint64)), out, slots)
    L.hc_ctx_device_status(ctx)
    torch.cuda.synchronize()
    return to_host(out).reshape(p.O, 2, nl, p.N), to_host(slots).reshape(p.O, nl, S)


def test_server_step_small_layer_full_parity_and_decryption(L):
    p, params, sk, x_c, x_s, K, r, ct = _case(5, 7, 6, 3, 3, 3, 1, 4096, 2, 1, part=(3, 6, 5))
    got_out, got_slots = _run(L, p, params, K, ct, x_s, r)
    ct1 = conv.share_add(ct, x_s, p, params.moduli, T_PLAIN)
    want_out = conv.conv_ct_pt(ct1, conv.pack_weights(K, p), p, params.moduli)
    assert np.array_equal(got_out, want_out)
    assert np.array_equal(got_slots, conv.extract_masked(want_out, r, p, params.moduli, T_PLAIN))
    y = conv.conv2d_mod_t((x_c + x_s) % T_PLAIN, K, p.pad, T_PLAIN)
    for o in range(p.O):
        _check_output(p, params, sk, got_out, got_slots, y, r, o)


def _check_output(p, params, sk, got_out, got_slots, y, r, o):
    """Decrypt every returned slot of output o (c0 slot + full c1) and compare with y - r mod t."""
    m, b = divmod(o, p.B)
    sl = conv.output_slots(p, b)
    c = got_out[o].copy()
    for k, _, _ in sl:
        rel = k - p.offset
        c[0, :, k] = got_slots[o, :, (rel // p.Ww) * p.ow + rel % p.Ww]
    got = bfv.decrypt_at(params, sk, c, [k for k, _, _ in sl])
    want = [(int(y[m, row, col]) - int(r[m, row, col])) % T_PLAIN for _, row, col in sl]
    assert [int(v) for v in got] == want, o


def test_server_step_56x56x64_sampled(L):
    sh = CONV_56x56x64
    x_c, K = conv_tensors(sh, seed=2)
    p, params, sk, x_c, x_s, K, r, ct = _case(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, sh.pad, 8192, 3, 2, x_c=x_c, K=K)
    got_out, got_slots = _run(L, p, params, K, ct, x_s, r)
    ct1 = conv.share_add(ct, x_s, p, params.moduli, T_PLAIN)
    outs = [0, 1, p.O // 2, p.O - 1]
    ks = sample_indices(p.N, 8, 6)
    want = conv.conv_ct_pt(ct1, conv.pack_weights(K, p), p, params.moduli, ks, outputs=outs)
    assert np.array_equal(got_out[outs][..., ks], want)
    y = conv.conv2d_mod_t((x_c + x_s) % T_PLAIN, K, p.pad, T_PLAIN)
    for o in outs:                                   # every slot of these outputs decrypts to y - r
        _check_output(p, params, sk, got_out, got_slots, y, r, o)


def _sparse_vs_full(L, ctx, w, ct, share, mask):
    """hc_conv_server_step_sparse against hc_conv_server_step on the same inputs:
    c1 of every output and every slot, bit for bit."""
    nl, N = ctx.L, ctx.N
    S = L.slot_count(w)
    out = torch.empty(w.O * 2 * nl * N, dtype=torch.int64, device="cuda")
    slots = torch.empty(w.O * nl * S, dtype=torch.int64, device="cuda")
    c1 = torch.full((w.O * nl * N,), -1, dtype=torch.int64, device="cuda")
    slots2 = torch.full_like(slots, -1)
    d_in = to_dev(ct)
    d_share = to_dev(share.astype(np.uint64)) if share is not None else None
    d_mask = to_dev(mask.astype(np.uint64)) if mask is not None else None
    L.hc_conv_server_step(ctx, w, d_in, d_share, d_mask, out, slots)
    L.hc_conv_server_step_sparse(ctx, w, d_in, d_share, d_mask, c1, slots2)
    L.hc_ctx_device_status(ctx)
    torch.cuda.synchronize()
    assert torch.equal(slots2, slots)
    assert torch.equal(c1.view(w.O, nl * N), out.view(w.O, 2, nl * N)[:, 1])
    return to_host(c1).reshape(w.O, nl, N), to_host(slots2).reshape(w.O, nl, S)


def test_sparse_server_step_matches_full_step_and_oracle(L):
    p, params, sk, x_c, x_s, K, r, ct = _case(5, 7, 6, 3, 3, 3, 1, 4096, 2, 3, part=(3, 6, 5))
    ctx = L.hc_ctx_create(p.N, params.moduli, T_PLAIN)
    d = L.make_desc(p.C, p.H, p.W, p.M, p.kh, p.kw, pad=p.pad, Cw=p.Cw, Hw=p.Hw, Ww=p.Ww)
    ct1 = conv.share_add(ct, x_s, p, params.moduli, T_PLAIN)
    want_out = conv.conv_ct_pt(ct1, conv.pack_weights(K, p), p, params.moduli)
    want_slots = conv.extract_masked(want_out, r, p, params.moduli, T_PLAIN)
    for mode in range(3):
        w = L.hc_weights_preprocess_ex(ctx, d, K.astype(np.int8), mode)
        c1, slots = _sparse_vs_full(L, ctx, w, ct, x_s, r)
        assert np.array_equal(c1, want_out[:, 1]) and np.array_equal(slots, want_slots), mode
        _sparse_vs_full(L, ctx, w, ct, None, None)          # no share, no mask
        w.close()
    # the client decrypts every returned slot from (slot, c1) alone
    y = conv.conv2d_mod_t((x_c + x_s) % T_PLAIN, K, p.pad, T_PLAIN)
    for o in range(p.O):
        c = np.zeros((2, len(params.moduli), p.N), dtype=np.uint64)
        c[1] = c1[o]
        _check_output(p, params, sk, np.stack([c] * p.O), slots, y, r, o)


def test_sparse_server_step_56x56x64(L):
    sh = CONV_56x56x64
    x_c, K = conv_tensors(sh, seed=2)
    p, params, sk, x_c, x_s, K, r, ct = _case(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, sh.pad, 8192, 3, 4, x_c=x_c, K=K)
    ctx = L.hc_ctx_create(8192, params.moduli, T_PLAIN)
    w = L.hc_weights_preprocess(ctx, L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad), K.astype(np.int8))
    for form in (0, 2):                                     # three launches; per-limb chains on side streams
        L.hc_ctx_set_variant(ctx, L.KIND_CONV_FORM, form)
        for v in range(3):                                  # every launch shape of the inverse transform
            L.hc_ctx_set_variant(ctx, L.KIND_NTT_INV_CT, v)
            _sparse_vs_full(L, ctx, w, ct, x_s, r)
            _sparse_vs_full(L, ctx, w, ct, None, None)
