"""GPU parity of the tensor-core convolution MAC (MAC variant 3: residues split
into 8-bit limbs, exact f16 products summed in fp32 by tcgen05 MMAs, recombined
and reduced mod q; the NTT-domain MAC of Sec. 6.2).  Every output residue must
equal the oracle's schoolbook convolution and the integer MAC's, for every
channel-group count and row count the kernel takes, ragged and multi-block
output channels, the special-form and the generic reduction, all-maximal
limbs, and every launch form; shapes it does not take fall back to the
integer MAC."""
import numpy as np
import pytest

from gpu_util import sample_indices, to_dev, to_host
from oracle import conv, core
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, CONV_56x56x64, T_PLAIN, Stream, conv_tensors, \
    uniform_residues

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TC = 3  # the tensor-core MAC variant of the blocked convolution MAC


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_11586_gb300 import _lib
    from paper_2506_11586_gb300.build import build
    build()
    return _lib


def _layer(L, moduli, N, C_, H, W, M, Cw, Hw, Ww, seed):
    p = conv.Partition(C_, H, W, M, 3, 3, 1, N, Cw, Hw, Ww)
    s = Stream(seed, M)
    K = s.int8(M * C_ * 9).astype(np.int64).reshape(M, C_, 3, 3)
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    w = L.hc_weights_preprocess(ctx, L.make_desc(C_, H, W, M, 3, 3, pad=1, Cw=Cw, Hw=Hw, Ww=Ww),
                                K.astype(np.int8))
    return p, K, ctx, w, s


def _run(L, ctx, w, d_in, variant, form=0):
    L.hc_ctx_set_variant(ctx, L.KIND_MAC_CONV, variant)
    L.hc_ctx_set_variant(ctx, L.KIND_CONV_FORM, form)
    out = torch.full((w.O * 2 * ctx.L * ctx.N,), -1, dtype=torch.int64, device="cuda")
    L.hc_conv_ct_pt(ctx, w, d_in, out)
    L.hc_ctx_device_status(ctx)
    return to_host(out).reshape(w.O, 2, ctx.L, ctx.N)


@pytest.mark.parametrize("G, B_blocks, M", [(1, 1, 3), (2, 4, 5), (3, 1, 64), (5, 4, 7), (8, 4, 5), (8, 1, 70),
                                            (4, 2, 130), (6, 3, 9)])
def test_tc_mac_matches_oracle(L, G, B_blocks, M):
    """G = 1..8 channel groups, 2, 4, 6 or 8 rows per group, one ragged or several
    blocks of 64 output channels: every residue equals the oracle's (all slots for
    small layers, sampled slots for M > 64) and the integer MAC's."""
    N, nl = 4096, 2
    moduli = CANONICAL_PRIMES[:nl]
    Cw = 2
    H = W = 6
    Hw, Ww = {1: (8, 8), 2: (6, 8), 3: (4, 8), 4: (6, 6)}[B_blocks]
    p, K, ctx, w, s = _layer(L, moduli, N, G * Cw, H, W, M, Cw, Hw, Ww, 200 + G)
    assert (p.G, p.B) == (G, B_blocks)
    ct = uniform_residues(s, moduli, (p.I, 2), N)
    d_in = to_dev(ct)
    got = _run(L, ctx, w, d_in, TC)
    ks = None if M <= 8 else sample_indices(N, 24, G)
    want = conv.conv_ct_pt(ct, conv.pack_weights(K, p), p, moduli, ks)
    assert np.array_equal(got if ks is None else got[..., ks], want)
    assert np.array_equal(got, _run(L, ctx, w, d_in, 1))


def test_tc_mac_ring_degree_16384(L):
    """N = 16384 with four limbs (the ResNet-50 configuration), three blocks of 64
    channels (the last ragged), 4 channel groups and 2 spatial blocks: sampled slots
    equal the oracle, every residue the integer MAC's, in launch forms 0 and 2."""
    N, nl = 16384, 4
    moduli = CANONICAL_PRIMES[:nl]
    p, K, ctx, w, s = _layer(L, moduli, N, 8, 6, 6, 150, 2, 6, 8, 260)
    assert (p.G, p.B) == (4, 2)
    ct = uniform_residues(s, moduli, (p.I, 2), N)
    d_in = to_dev(ct)
    got = _run(L, ctx, w, d_in, TC)
    ks = sample_indices(N, 16, 7)
    assert np.array_equal(got[..., ks], conv.conv_ct_pt(ct, conv.pack_weights(K, p), p, moduli, ks))
    assert np.array_equal(got, _run(L, ctx, w, d_in, 1))
    assert np.array_equal(got, _run(L, ctx, w, d_in, TC, 2))


def test_tc_mac_maximal_limbs_and_generic_reduction(L):
    """Inputs all q - 1 (every 8-bit limb 255 but the top one) with eight channel
    groups, the largest sums the fp32 accumulation must hold exactly; primes far
    below 2^50 (the generic reduction) as well as the canonical ones."""
    N = 4096
    for moduli in (CANONICAL_PRIMES[:2], tuple(core.ntt_primes(47, 13, 2))):
        p, K, ctx, w, s = _layer(L, moduli, N, 16, 6, 6, 6, 2, 6, 6, 230)
        assert (p.G, p.B) == (8, 4)
        ct = np.stack([np.full((p.I, 2, N), q - 1, dtype=np.uint64) for q in moduli], axis=2)
        d_in = to_dev(ct)
        got = _run(L, ctx, w, d_in, TC)
        ks = sample_indices(N, 16, 5)
        want = conv.conv_ct_pt(ct, conv.pack_weights(K, p), p, moduli, ks)
        assert np.array_equal(got[..., ks], want)
        assert np.array_equal(got, _run(L, ctx, w, d_in, 1))


def test_tc_mac_metric_layer_every_form(L):
    """The 56x56x64 -> 64 layer at N = 8192, three limbs (G = 8, four spatial
    blocks): the tensor-core MAC in launch forms 0 and 2 equals the integer MAC
    bit for bit, and sampled slots equal the oracle."""
    sh, N, moduli = CONV_56x56x64, 8192, CANONICAL_PRIMES[:3]
    _, K = conv_tensors(sh, seed=2)
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    w = L.hc_weights_preprocess(ctx, L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad), K)
    ct = uniform_residues(Stream(2, 5), moduli, (w.I, 2), N)
    d_in = to_dev(ct)
    want = _run(L, ctx, w, d_in, 1, 0)
    for form in (0, 2):
        assert np.array_equal(_run(L, ctx, w, d_in, TC, form), want), form
    p = conv.canonical_partition(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, sh.pad, N)
    ks = sample_indices(N, 8, 3)
    assert np.array_equal(want[..., ks], conv.conv_ct_pt(ct, conv.pack_weights(K.astype(np.int64), p), p,
                                                         moduli, ks))


def test_tc_mac_falls_back_outside_its_shapes(L):
    """G = 9 channel groups and 2B = 12 rows are outside the tensor-core MAC; with
    variant 3 set the layer runs on the integer MAC and stays exact."""
    N, nl = 4096, 2
    moduli = CANONICAL_PRIMES[:nl]
    for (G, Hw, Ww) in ((9, 8, 8), (2, 4, 6)):
        p, K, ctx, w, s = _layer(L, moduli, N, 2 * G, 6, 6, 3, 2, Hw, Ww, 240 + G)
        assert p.G > 8 or 2 * p.B > 8
        ct = uniform_residues(s, moduli, (p.I, 2), N)
        got = _run(L, ctx, w, to_dev(ct), TC)
        assert np.array_equal(got, conv.conv_ct_pt(ct, conv.pack_weights(K, p), p, moduli))


def test_tc_variant_range(L):
    ctx = L.hc_ctx_create(4096, CANONICAL_PRIMES[:2], T_PLAIN)
    L.hc_ctx_set_variant(ctx, L.KIND_MAC_CONV, TC)
    assert L.hc_ctx_get_variant(ctx, L.KIND_MAC_CONV) == TC
    for kind, v in ((L.KIND_MAC_CONV, 4), (L.KIND_NTT_INV_CT, 3)):
        with pytest.raises(L.HcError) as e:
            L.hc_ctx_set_variant(ctx, kind, v)
        assert e.value.status == L.HC_ERR_INVALID_ARG
