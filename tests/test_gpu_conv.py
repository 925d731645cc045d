"""GPU parity of the convolution path: hc_weights_preprocess (offline NTT of
packed weights, Sec. 6.2 / Sec. 8.1) and hc_conv_ct_pt (online NTT -> MAC ->
INTT, Sec. 6.2) against the oracle's schoolbook convolution, bit-exact, and
end to end through BFV: encrypt -> GPU conv -> decrypt == plaintext conv mod t."""
import numpy as np
import pytest

from gpu_util import sample_indices, to_dev, to_host
from oracle import bfv, conv, core
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


def _encrypted_layer(C_, H, W, M, kh, kw, pad, N, nl, seed, x=None, K=None):
    s = Stream(seed, 3)
    if x is None:
        x = s.below(T_PLAIN, C_ * H * W).astype(np.int64).reshape(C_, H, W)
        K = s.int8(M * C_ * kh * kw).astype(np.int64).reshape(M, C_, kh, kw)
    p = conv.canonical_partition(C_, H, W, M, kh, kw, pad, N)
    params = bfv.Params(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    sk = s.ternary(N)
    xin = conv.pack_input(x, p)
    ct = np.zeros((p.I, 2, nl, N), dtype=np.uint64)
    for i in range(p.I):
        a = np.stack([s.below(q, N) for q in params.moduli])
        ct[i] = bfv.encrypt(params, sk, xin[i], a, s.rounded_gaussian(N))
    return x, np.asarray(K, dtype=np.int64), p, params, sk, ct


def _gpu_layer(L, p, params, K):
    ctx = L.hc_ctx_create(p.N, params.moduli, T_PLAIN)
    d = L.make_desc(p.C, p.H, p.W, p.M, p.kh, p.kw, pad=p.pad)
    w = L.hc_weights_preprocess(ctx, d, K.astype(np.int8))
    assert (w.desc.Cw, w.desc.Hw, w.desc.Ww, w.I, w.O) == (p.Cw, p.Hw, p.Ww, p.I, p.O)
    return ctx, w


def _check_decrypt(p, params, sk, out, y, ms):
    for m in ms:
        for b in range(p.B):
            slots = conv.output_slots(p, b)
            ks = [k for k, _, _ in slots]
            got = bfv.decrypt_at(params, sk, out[m * p.B + b], ks)
            want = np.array([y[m, r, c] for _, r, c in slots])
            assert np.array_equal(got, want), (m, b)


@pytest.mark.parametrize("shape", [
    (5, 7, 6, 3, 3, 3, 1, 4096, 2),     # ragged channel group, edge blocks
    (12, 9, 9, 4, 1, 1, 0, 8192, 3),    # 1x1 convolution
    (6, 20, 20, 3, 3, 3, 1, 16384, 4),  # N = 16384, four limbs
])
def test_small_layer_full_parity(L, shape):
    x, K, p, params, sk, ct = _encrypted_layer(*shape, seed=sum(shape))
    ctx, w = _gpu_layer(L, p, params, K)
    d_in = to_dev(ct)
    d_out = torch.empty(p.O * 2 * len(params.moduli) * p.N, dtype=torch.int64, device="cuda")
    L.hc_conv_ct_pt(ctx, w, d_in, d_out)
    torch.cuda.synchronize()
    got = to_host(d_out).reshape(p.O, 2, len(params.moduli), p.N)
    Kp = conv.pack_weights(K, p)
    want = conv.conv_ct_pt(ct, Kp, p, params.moduli)
    assert np.array_equal(got, want)
    assert np.array_equal(to_host(d_in).reshape(ct.shape), ct)        # input untouched
    y = conv.conv2d_mod_t(x, K, p.pad, T_PLAIN)
    _check_decrypt(p, params, sk, got, y, range(p.M))
    # the plain one-launch-per-product path gives the same bits
    d_plain = torch.empty_like(d_out)
    L.hc_conv_ct_pt_plain(ctx, w, d_in, d_plain)
    torch.cuda.synchronize()
    assert torch.equal(d_plain, d_out)
    # host-buffer entry point
    h_out = np.zeros((p.O, 2, len(params.moduli), p.N), dtype=np.uint64)
    L.hc_conv_ct_pt_host(ctx, w, np.ascontiguousarray(ct), h_out)
    assert np.array_equal(h_out, got)


def test_preprocessed_weights_are_ntt_of_packing(L):
    C_, H, W, M = 6, 10, 10, 4
    s = Stream(44, 0)
    K = s.int8(M * C_ * 9).astype(np.int64).reshape(M, C_, 3, 3)
    N, moduli = 8192, CANONICAL_PRIMES[:3]
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    w = L.hc_weights_preprocess(ctx, L.make_desc(C_, H, W, M, 3, 3, pad=1), K.astype(np.int8))
    p = conv.canonical_partition(C_, H, W, M, 3, 3, 1, N)
    _, n_pt = L.hc_weights_data(w)
    assert n_pt == p.P
    buf = torch.empty(p.P * 3 * N, dtype=torch.int64, device="cuda")
    L.hc_weights_export(w, buf)
    torch.cuda.synchronize()
    got = to_host(buf).reshape(p.P, 3, N)
    Kp = conv.pack_weights(K, p)
    ks = sample_indices(N, 48, 3)
    for pi in range(p.P):
        for li, q in enumerate(moduli):
            want = core.ntt(core.lift_small(Kp[pi], q), q, core.min_psi(q, N), ks)
            assert np.array_equal(got[pi, li][ks], want), (pi, li)


@pytest.fixture(scope="module")
def layer_56x56x64():
    """The 56x56x64 -> 64, 3x3 layer at N = 8192 with three primes, encrypted."""
    sh = CONV_56x56x64
    x, K = conv_tensors(sh, seed=2)
    return _encrypted_layer(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, sh.pad, 8192, 3, seed=2, x=x, K=K)


def test_layer_56x56x64_parity(L, layer_56x56x64):
    x, K, p, params, sk, ct = layer_56x56x64
    assert (p.I, p.P, p.O, p.products) == (32, 512, 256, 2048)
    ctx, w = _gpu_layer(L, p, params, K)
    d_in = to_dev(ct)
    d_out = torch.empty(p.O * 2 * 3 * p.N, dtype=torch.int64, device="cuda")
    L.hc_conv_ct_pt(ctx, w, d_in, d_out)
    L.hc_ctx_device_status(ctx)          # no bounded device wait ran out
    torch.cuda.synchronize()
    got = to_host(d_out).reshape(p.O, 2, 3, p.N)
    # sampled coefficients of every output polynomial vs the schoolbook conv
    ks = sample_indices(p.N, 40, 11)
    want = conv.conv_ct_pt(ct, conv.pack_weights(K, p), p, params.moduli, ks)
    assert np.array_equal(got[..., ks], want)
    # decrypt every output slot of a spread of output channels
    y = conv.conv2d_mod_t(x, K, p.pad, T_PLAIN)
    _check_decrypt(p, params, sk, got, y, [0, 1, 31, 63])
    # repeat run is deterministic; plain path agrees bit for bit
    d_out2 = torch.empty_like(d_out)
    L.hc_conv_ct_pt(ctx, w, d_in, d_out2)
    torch.cuda.synchronize()
    assert torch.equal(d_out2, d_out)
    d_plain = torch.empty_like(d_out)
    L.hc_conv_ct_pt_plain(ctx, w, d_in, d_plain)
    torch.cuda.synchronize()
    assert torch.equal(d_plain, d_out)


def test_layer_56x56x64_every_coefficient(L, layer_56x56x64):
    """Every residue of the metric layer's output (256 ciphertexts x 2
    components x 3 limbs x 8192 coefficients) equals the oracle's sparse
    schoolbook convolution, under the tuned launch form of the bench (the
    limbs' chains on parallel streams) and under one launch per phase."""
    x, K, p, params, sk, ct = layer_56x56x64
    ctx, w = _gpu_layer(L, p, params, K)
    want = conv.conv_ct_pt(ct, conv.pack_weights(K, p), p, params.moduli)
    d_in = to_dev(ct)
    for form in (2, 0):
        L.hc_ctx_set_variant(ctx, L.KIND_CONV_FORM, form)
        d_out = torch.full((p.O * 2 * 3 * p.N,), -1, dtype=torch.int64, device="cuda")
        L.hc_conv_ct_pt(ctx, w, d_in, d_out)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(d_out).reshape(p.O, 2, 3, p.N), want), form


def test_conv_argument_errors(L):
    N, moduli = 4096, CANONICAL_PRIMES[:2]
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    other = L.hc_ctx_create(N, moduli, T_PLAIN)
    K = np.zeros((2, 3, 3, 3), dtype=np.int8)
    w = L.hc_weights_preprocess(ctx, L.make_desc(3, 5, 5, 2, 3, 3, pad=1), K)
    buf = torch.zeros(w.I * 2 * 2 * N, dtype=torch.int64, device="cuda")
    out = torch.zeros(w.O * 2 * 2 * N, dtype=torch.int64, device="cuda")
    with pytest.raises(L.HcError) as e:
        L.hc_conv_ct_pt(other, w, buf, out)           # weights of another context
    assert e.value.status == L.HC_ERR_INVALID_ARG
    with pytest.raises(L.HcError) as e:
        L.hc_weights_preprocess(ctx, L.make_desc(3, 5, 5, 2, 3, 3, pad=1, stride=0), K)
    assert e.value.status == L.HC_ERR_INVALID_ARG
    with pytest.raises(L.HcError) as e:
        L.hc_weights_preprocess(ctx, L.make_desc(3, 1, 1, 2, 3, 3, pad=0, stride=2), K)
    assert e.value.status == L.HC_ERR_INVALID_ARG      # kernel larger than the input
    L.hc_conv_ct_pt(ctx, w, buf, out)                 # all-zero input -> all-zero output
    torch.cuda.synchronize()
    assert int(out.abs().sum()) == 0


@pytest.mark.parametrize("moduli_kind", ["far_from_2^50", "canonical_G_over_16"])
def test_generic_reduction_paths(L, moduli_kind):
    """The MAC's reduction has a special form for q = 2^50 - c with small c (the
    canonical primes) and a generic one; this covers the generic one twice:
    primes far below 2^50, and canonical primes with more than 16 channel groups
    (where the special form's input bound does not hold)."""
    N = 8192
    if moduli_kind == "far_from_2^50":
        moduli = tuple(core.ntt_primes(47, 15, 3))
        shape, part = (9, 11, 11, 5, 3, 3, 1), None
    else:
        moduli = CANONICAL_PRIMES[:3]
        shape, part = (34, 6, 6, 3, 1, 1, 0), (2, 6, 6)    # Cw = 2 -> G = 17
    C_, H, W, M, kh, kw, pad = shape
    assert all(2 ** 32 < q < 2 ** 50 and q % (2 * N) == 1 for q in moduli)
    s = Stream(77, len(moduli))
    K = s.int8(M * C_ * kh * kw).astype(np.int64).reshape(M, C_, kh, kw)
    p = conv.Partition(C_, H, W, M, kh, kw, pad, N, *part) if part else \
        conv.canonical_partition(C_, H, W, M, kh, kw, pad, N)
    if part:
        assert p.G == 17
    else:
        assert all((1 << 50) - q >= (1 << 22) for q in moduli)
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    w = L.hc_weights_preprocess(ctx, L.make_desc(C_, H, W, M, kh, kw, pad=pad, Cw=p.Cw, Hw=p.Hw, Ww=p.Ww),
                                K.astype(np.int8))
    ct = uniform_residues(s, moduli, (p.I, 2), N)
    out = torch.empty(p.O * 2 * len(moduli) * N, dtype=torch.int64, device="cuda")
    L.hc_conv_ct_pt(ctx, w, to_dev(ct), out)
    torch.cuda.synchronize()
    ks = sample_indices(N, 24, 9)
    want = conv.conv_ct_pt(ct, conv.pack_weights(K, p), p, moduli, ks)
    assert np.array_equal(to_host(out).reshape(p.O, 2, len(moduli), N)[..., ks], want)


@pytest.mark.parametrize("M", [1, 2, 7, 13, 64])
def test_host_entry_point_blocks_of_output_channels(L, M):
    """hc_conv_ct_pt_host runs offline-weight layers in up to eight blocks of output
    channels, copying each block back while the next is computed: pinned and
    pageable host buffers, block counts that do not divide M, every bit equal to
    the device entry point."""
    N, nl = 8192, 3
    ctx = L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    s = Stream(48, M)
    C_, H, W = 12, 20, 20
    K = s.int8(M * C_ * 9).reshape(M, C_, 3, 3)
    w = L.hc_weights_preprocess(ctx, L.make_desc(C_, H, W, M, 3, 3, pad=1), K)
    ct = uniform_residues(s, CANONICAL_PRIMES[:nl], (w.I, 2), N)
    d_out = torch.empty(w.O * 2 * nl * N, dtype=torch.int64, device="cuda")
    L.hc_conv_ct_pt(ctx, w, to_dev(ct), d_out)
    torch.cuda.synchronize()
    want = to_host(d_out)
    h_in = torch.from_numpy(ct.reshape(-1).view(np.int64)).pin_memory()
    h_out = torch.full((w.O * 2 * nl * N,), -1, dtype=torch.int64).pin_memory()
    for _ in range(2):
        L.hc_conv_ct_pt_host(ctx, w, h_in, h_out)
        assert np.array_equal(h_out.numpy().view(np.uint64), want)
        h_out.fill_(-1)
    pageable = np.zeros(w.O * 2 * nl * N, dtype=np.uint64)
    L.hc_conv_ct_pt_host(ctx, w, np.ascontiguousarray(ct), pageable)
    assert np.array_equal(pageable, want)


@pytest.mark.parametrize("G, B_blocks", [(2, 1), (3, 9), (4, 9), (5, 1), (8, 4), (15, 9), (16, 1)])
def test_mac_channel_group_sweep(L, G, B_blocks, tmp_path):
    """The blocked MAC sums G channel groups per output row in pairs of
    accumulator chains, with channel x row tiles when a channel has several
    rows (several spatial blocks) and a few-rows path otherwise (one block:
    two rows per channel), and the last of an odd number of output channels
    alone. Every output residue must equal the oracle's schoolbook sum for even
    and odd G up to the special-form reduction's limit of 16 terms, with
    offline weights, online weights and weights after a save / load round trip."""
    N, nl = 4096, 2
    moduli = CANONICAL_PRIMES[:nl]
    Cw = 2
    C_, M = G * Cw, 5
    H = W = 8 if B_blocks == 4 else 6
    Hw = Ww = {1: 8, 4: 6, 9: 4}[B_blocks]
    p = conv.Partition(C_, H, W, M, 3, 3, 1, N, Cw, Hw, Ww)
    assert p.G == G and p.B == B_blocks, (p.G, p.B)
    s = Stream(91, G)
    K = s.int8(M * C_ * 9).astype(np.int64).reshape(M, C_, 3, 3)
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    desc = L.make_desc(C_, H, W, M, 3, 3, pad=1, Cw=Cw, Hw=Hw, Ww=Ww)
    ct = uniform_residues(s, moduli, (p.I, 2), N)
    want = conv.conv_ct_pt(ct, conv.pack_weights(K, p), p, moduli)
    d_in = to_dev(ct)
    offline = L.hc_weights_preprocess_ex(ctx, desc, K.astype(np.int8), L.HC_WEIGHTS_NTT_OFFLINE)
    online = L.hc_weights_preprocess_ex(ctx, desc, K.astype(np.int8), L.HC_WEIGHTS_NTT_ONLINE)
    L.hc_weights_save(offline, tmp_path / "w.bin")
    loaded = L.hc_weights_load(ctx, tmp_path / "w.bin")
    for name, w in (("offline", offline), ("online", online), ("loaded", loaded)):
        out = torch.empty(p.O * 2 * nl * N, dtype=torch.int64, device="cuda")
        L.hc_conv_ct_pt(ctx, w, d_in, out)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(out).reshape(p.O, 2, nl, N), want), name
