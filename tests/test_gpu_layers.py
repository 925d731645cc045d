"""GPU parity of the linear layers beyond stride-1 convolutions (Sec. 8.1's
networks, Sec. 6.1 coefficient encoding): stride-2 convolutions (SqueezeNet-1.1
conv1, ResNet-50 conv1 7x7 and its downsampling layers) through the polyphase
split, and fully connected layers (ResNet-50's classifier) through
matrix-vector packing.  Every output uint64 must equal the oracle's schoolbook
result on the same inputs (sampled coefficients at full size, everything on
small layers); all preprocessing modes, plans, the server step and saved
weights must give the same bits; end to end through BFV the client decrypts
layer(x_c + x_s) - r mod t."""
import numpy as np
import pytest

from gpu_util import sample_indices, to_dev, to_host
from oracle import bfv, conv, layers
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream, uniform_residues

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


_CTX = {}


def _ctx(L, N, nl):
    if (N, nl) not in _CTX:
        _CTX[(N, nl)] = L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    return _CTX[(N, nl)]


def _run(L, ctx, w, ct):
    out = torch.empty(w.O * 2 * ctx.L * ctx.N, dtype=torch.int64, device="cuda")
    out.fill_(-1)
    L.hc_conv_ct_pt(ctx, w, to_dev(ct), out)
    L.hc_ctx_device_status(ctx)
    torch.cuda.synchronize()
    return out


# (C, H, W, M, kh, kw, stride, pad, N, L): full-size layers of the networks, sampled
STRIDED_FULL = [
    (3, 224, 224, 64, 3, 3, 2, 0, 8192, 3),       # SqueezeNet-1.1 conv1
    (3, 224, 224, 64, 7, 7, 2, 3, 16384, 4),      # ResNet-50 conv1
    (128, 56, 56, 128, 3, 3, 2, 1, 16384, 4),     # ResNet-50 layer2.0 conv2
    (1024, 14, 14, 2048, 1, 1, 2, 0, 16384, 4),   # ResNet-50 layer4.0 projection
]


@pytest.mark.parametrize("shape", STRIDED_FULL)
def test_strided_full_size_sampled(L, shape):
    C_, H, W, M, kh, kw, st, pad, N, nl = shape
    ctx = _ctx(L, N, nl)
    s = Stream(61, sum(shape))
    K = s.int8(M * C_ * kh * kw).astype(np.int64).reshape(M, C_, kh, kw)
    w = L.hc_weights_preprocess(ctx, L.make_desc(C_, H, W, M, kh, kw, pad=pad, stride=st), K.astype(np.int8))
    ph, p = layers.strided_partition(C_, H, W, M, kh, kw, st, pad, N)
    assert (w.computed.C, w.computed.kh, w.computed.Cw, w.computed.Hw, w.computed.Ww) == (ph.C1, ph.kh1, p.Cw, p.Hw, p.Ww)
    assert (w.I, w.O, w.products) == (p.I, p.O, p.products)
    ct = uniform_residues(s, CANONICAL_PRIMES[:nl], (p.I, 2), N)
    got = to_host(_run(L, ctx, w, ct)).reshape(p.O, 2, nl, N)
    outs = sorted({0, p.O // 3, p.O - 1})
    ks = sample_indices(N, 10, 62)
    Kp = conv.pack_weights(layers.polyphase_kernel(K, ph), p)
    want = conv.conv_ct_pt(ct, Kp, p, CANONICAL_PRIMES[:nl], ks, outputs=outs)
    assert np.array_equal(got[outs][..., ks], want)


def _sparse_matches(L, ctx, w, ct, share, mask, full_out, full_slots):
    """hc_conv_server_step_sparse returns c1 of the full step's outputs and the same slots."""
    c1 = torch.full((w.O * ctx.L * ctx.N,), -1, dtype=torch.int64, device="cuda")
    slots = torch.full((w.O * ctx.L * L.slot_count(w),), -1, dtype=torch.int64, device="cuda")
    L.hc_conv_server_step_sparse(ctx, w, to_dev(ct), to_dev(share.astype(np.uint64)), to_dev(mask.astype(np.uint64)),
                                 c1, slots)
    L.hc_ctx_device_status(ctx)
    assert np.array_equal(to_host(c1).reshape(w.O, ctx.L, ctx.N), full_out[:, 1])
    assert np.array_equal(to_host(slots).reshape(full_slots.shape), full_slots)


SMALL_STRIDED = [
    (4, 9, 9, 3, 3, 3, 2, 1, 4096, 2),
    (3, 11, 10, 4, 7, 7, 2, 3, 4096, 2),
    (5, 8, 8, 2, 1, 1, 2, 0, 4096, 2),
    (2, 13, 11, 3, 4, 2, 3, 1, 8192, 3),
]


def _bfv_inputs(s, params, sk, packed):
    ct = np.zeros((packed.shape[0], 2, len(params.moduli), params.N), dtype=np.uint64)
    for i in range(packed.shape[0]):
        a = np.stack([s.below(q, params.N) for q in params.moduli])
        ct[i] = bfv.encrypt(params, sk, packed[i], a, s.rounded_gaussian(params.N))
    return ct


@pytest.mark.parametrize("shape", SMALL_STRIDED)
def test_strided_server_step_full_parity_modes_and_decryption(L, shape):
    C_, H, W, M, kh, kw, st, pad, N, nl = shape
    ctx = _ctx(L, N, nl)
    s = Stream(63, sum(shape))
    params = bfv.Params(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    sk = s.ternary(N)
    x_c = s.below(T_PLAIN, C_ * H * W).astype(np.int64).reshape(C_, H, W)
    x_s = s.below(T_PLAIN, C_ * H * W).astype(np.int64).reshape(C_, H, W)
    K = s.int8(M * C_ * kh * kw).astype(np.int64).reshape(M, C_, kh, kw)
    ph, p = layers.strided_partition(C_, H, W, M, kh, kw, st, pad, N)
    r = s.below(T_PLAIN, M * p.Ho * p.Wo).astype(np.int64).reshape(M, p.Ho, p.Wo)
    ct = _bfv_inputs(s, params, sk, conv.pack_input(layers.polyphase_input(x_c, ph), p))
    d = L.make_desc(C_, H, W, M, kh, kw, pad=pad, stride=st)
    ws = [L.hc_weights_preprocess_ex(ctx, d, K.astype(np.int8), mode) for mode in range(3)]
    ref = _run(L, ctx, ws[0], ct)
    for w in ws[1:]:
        assert torch.equal(_run(L, ctx, w, ct), ref)
    # oracle: whole layer, every coefficient
    Kp = conv.pack_weights(layers.polyphase_kernel(K, ph), p)
    assert np.array_equal(to_host(ref).reshape(p.O, 2, nl, N), conv.conv_ct_pt(ct, Kp, p, params.moduli))
    # the server step: share through the phase split, mask, slots
    S = L.slot_count(ws[0])
    assert S == conv.slot_count(p)
    ct1 = layers.strided_share_add(ct, x_s, ph, p, params.moduli, T_PLAIN)
    want_out = conv.conv_ct_pt(ct1, Kp, p, params.moduli)
    want_slots = conv.extract_masked(want_out, r, p, params.moduli, T_PLAIN)
    y = layers.conv2d_strided_mod_t((x_c + x_s) % T_PLAIN, K, st, pad, T_PLAIN)
    for w in ws:
        out = torch.empty(p.O * 2 * nl * N, dtype=torch.int64, device="cuda")
        slots = torch.empty(p.O * nl * S, dtype=torch.int64, device="cuda")
        L.hc_conv_server_step(ctx, w, to_dev(ct), to_dev(x_s.astype(np.uint64)), to_dev(r.astype(np.uint64)),
                              out, slots)
        L.hc_ctx_device_status(ctx)
        got_out = to_host(out).reshape(p.O, 2, nl, N)
        got_slots = to_host(slots).reshape(p.O, nl, S)
        assert np.array_equal(got_out, want_out) and np.array_equal(got_slots, want_slots)
        _sparse_matches(L, ctx, w, ct, x_s, r, got_out, got_slots)
    # the client decrypts layer(x_c + x_s) - r at every output
    n = 0
    for m in range(M):
        for b in range(p.B):
            o = m * p.B + b
            for k, row, col in conv.output_slots(p, b):
                rel = k - p.offset
                c = got_out[o].copy()
                c[0, :, k] = got_slots[o, :, (rel // p.Ww) * p.ow + rel % p.Ww]
                assert int(bfv.decrypt_at(params, sk, c, [k])[0]) == (int(y[m, row, col]) - int(r[m, row, col])) % T_PLAIN
                n += 1
    assert n == M * ph.Ho * ph.Wo


def test_fc_resnet50_classifier_sampled(L):
    C_, M, N, nl = 2048, 1000, 16384, 4
    ctx = _ctx(L, N, nl)
    s = Stream(64, 0)
    Wm = s.int8(M * C_).astype(np.int64).reshape(M, C_)
    w = L.hc_weights_preprocess_fc(ctx, L.make_fc_desc(C_, M), Wm.astype(np.int8))
    fp = layers.canonical_fc_partition(C_, M, N)
    assert (w.kind, w.No, w.I, w.O, w.products, L.slot_count(w)) == (1, fp.No, fp.I, fp.O, fp.P, fp.No)
    ct = uniform_residues(s, CANONICAL_PRIMES[:nl], (fp.I, 2), N)
    got = to_host(_run(L, ctx, w, ct)).reshape(fp.O, 2, nl, N)
    ks = np.array(sorted(set(sample_indices(N, 10, 65)) |
                         {layers.fc_output_coeff(fp, m)[1] for m in (0, fp.No - 1, 5 * fp.No + 3)}), dtype=np.uint32)
    outs = [0, fp.O - 1]
    want = conv.conv_ct_pt(ct, layers.pack_fc_weights(Wm, fp), fp, CANONICAL_PRIMES[:nl], ks, outputs=outs)
    assert np.array_equal(got[outs][..., ks], want)


@pytest.mark.parametrize("C_,M,N,nl,Cw,No", [(45, 23, 4096, 2, 20, 9), (300, 70, 8192, 3, 0, 0),
                                             (17, 5, 16384, 4, 17, 1)])
def test_fc_server_step_full_parity_modes_and_decryption(L, C_, M, N, nl, Cw, No):
    ctx = _ctx(L, N, nl)
    s = Stream(66, C_ * M)
    params = bfv.Params(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    sk = s.ternary(N)
    res, *_ = L.hc_fc_partition(L.make_fc_desc(C_, M, Cw, No), N)
    fp = layers.FcPartition(C_, M, N, res.Cw, res.No)
    if not Cw:
        assert fp == layers.canonical_fc_partition(C_, M, N)
    x_c = s.below(T_PLAIN, C_).astype(np.int64)
    x_s = s.below(T_PLAIN, C_).astype(np.int64)
    Wm = s.int8(M * C_).astype(np.int64).reshape(M, C_)
    r = s.below(T_PLAIN, M).astype(np.int64)
    ct = _bfv_inputs(s, params, sk, layers.pack_fc_input(x_c, fp))
    ws = [L.hc_weights_preprocess_fc(ctx, L.make_fc_desc(C_, M, Cw, No), Wm.astype(np.int8), mode) for mode in range(3)]
    Wp = layers.pack_fc_weights(Wm, fp)
    want_plain = conv.conv_ct_pt(ct, Wp, fp, params.moduli)
    ct1 = layers.fc_share_add(ct, x_s, fp, params.moduli, T_PLAIN)
    want_out = conv.conv_ct_pt(ct1, Wp, fp, params.moduli)
    want_slots = layers.fc_extract_masked(want_out, r, fp, params.moduli, T_PLAIN)
    for w in ws:
        assert np.array_equal(to_host(_run(L, ctx, w, ct)).reshape(fp.O, 2, nl, N), want_plain)
        out = torch.empty(fp.O * 2 * nl * N, dtype=torch.int64, device="cuda")
        slots = torch.empty(fp.O * nl * fp.No, dtype=torch.int64, device="cuda")
        L.hc_conv_server_step(ctx, w, to_dev(ct), to_dev(x_s.astype(np.uint64)), to_dev(r.astype(np.uint64)),
                              out, slots)
        L.hc_ctx_device_status(ctx)
        got_out, got_slots = to_host(out).reshape(fp.O, 2, nl, N), to_host(slots).reshape(fp.O, nl, fp.No)
        assert np.array_equal(got_out, want_out) and np.array_equal(got_slots, want_slots)
        _sparse_matches(L, ctx, w, ct, x_s, r, got_out, got_slots)
    y = layers.fc_mod_t((x_c + x_s) % T_PLAIN, Wm, T_PLAIN)
    for m in range(M):
        mp, k = layers.fc_output_coeff(fp, m)
        c = got_out[mp].copy()
        c[0, :, k] = got_slots[mp, :, m - mp * fp.No]
        assert int(bfv.decrypt_at(params, sk, c, [k])[0]) == (int(y[m]) - int(r[m])) % T_PLAIN, m


def test_strided_and_fc_in_plans_and_saved_weights(L, tmp_path):
    """One plan over a strided layer, an FC layer and a stride-1 layer of mixed
    degrees: bit-equal to each layer alone, direct and replayed; saved and
    loaded weights of both kinds compute the same bits."""
    s = Stream(67, 0)
    items = []
    specs = [("conv", (3, 30, 30, 8, 7, 7, 2, 3), (16384, 4)), ("fc", (300, 70), (8192, 3)),
             ("conv", (6, 12, 12, 5, 3, 3, 1, 1), (8192, 3)), ("conv", (16, 20, 20, 12, 3, 3, 2, 1), (4096, 2))]
    for kind, sh, (N, nl) in specs:
        ctx = _ctx(L, N, nl)
        if kind == "conv":
            C_, H, W, M, kh, kw, st, pad = sh
            K = s.int8(M * C_ * kh * kw).reshape(M, C_, kh, kw)
            w = L.hc_weights_preprocess(ctx, L.make_desc(C_, H, W, M, kh, kw, pad=pad, stride=st), K)
        else:
            C_, M = sh
            w = L.hc_weights_preprocess_fc(ctx, L.make_fc_desc(C_, M), s.int8(M * C_).reshape(M, C_))
        ct = uniform_residues(s, CANONICAL_PRIMES[:nl], (w.I, 2), N)
        d_in = to_dev(ct)
        ref = _run(L, ctx, w, ct)
        items.append(dict(ctx=ctx, w=w, d_in=d_in, ref=ref, out=torch.empty_like(ref)))
        path = tmp_path / ("w%d.bin" % len(items))
        L.hc_weights_save(w, path)
        w2 = L.hc_weights_load(ctx, path)
        assert (w2.I, w2.O, w2.kind, w2.No, w2.n_slots) == (w.I, w.O, w.kind, w.No, w.n_slots)
        assert torch.equal(_run(L, ctx, w2, ct), ref)
    plan = L.hc_plan_create([L.work_conv(it["ctx"], it["w"], it["d_in"], it["out"]) for it in items])
    assert L.hc_plan_info(plan)[0] == sum(it["w"].products for it in items)
    for rnd in range(3):                                     # direct, capture, replay
        for it in items:
            it["out"].fill_(-1)
        L.hc_plan_run(plan)
        torch.cuda.synchronize()
        for it in items:
            assert torch.equal(it["out"], it["ref"]), rnd
