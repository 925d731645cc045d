"""Every launch-shape variant of every kernel family computes the same bits as
the oracle: forward / inverse NTT (App. C.1), the fused NTT-domain MAC +
inverse NTT of a convolution (Sec. 6.2), and the fused standalone product."""
import numpy as np
import pytest

from gpu_util import sample_indices, to_dev, to_host
from oracle import conv, core
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream, uniform_residues

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SIZES = [(4096, 2), (8192, 3), (16384, 4)]


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_11586_gb300 import _lib
    from paper_2506_11586_gb300.build import build
    build()
    return _lib


@pytest.mark.parametrize("N,nl", SIZES)
def test_transform_variants(L, N, nl):
    moduli = CANONICAL_PRIMES[:nl]
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    a = uniform_residues(Stream(7, N), moduli, (3,), N)
    ks = sample_indices(N, 24, N + 1)
    psis = [core.min_psi(q, N) for q in moduli]
    want = [[core.ntt(a[p, li], q, psis[li], ks) for li, q in enumerate(moduli)] for p in range(3)]
    for v in range(L.N_VARIANTS):
        L.hc_ctx_set_variant(ctx, L.KIND_NTT_FWD, v)
        L.hc_ctx_set_variant(ctx, L.KIND_NTT_INV, v)
        assert L.hc_ctx_get_variant(ctx, L.KIND_NTT_FWD) == v
        d = to_dev(a)
        L.hc_ntt_fwd(ctx, d)
        torch.cuda.synchronize()
        A = to_host(d).reshape(a.shape)
        for p in range(3):
            for li in range(nl):
                assert np.array_equal(A[p, li][ks], want[p][li]), (v, p, li)
        L.hc_ntt_inv(ctx, d)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(d).reshape(a.shape), a), v


@pytest.mark.parametrize("N,nl", SIZES)
def test_conv_and_product_variants(L, N, nl):
    moduli = CANONICAL_PRIMES[:nl]
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    C_, H, W, M = 7, 9, 9, 3
    s = Stream(8, N)
    K = s.int8(M * C_ * 9).astype(np.int64).reshape(M, C_, 3, 3)
    p = conv.canonical_partition(C_, H, W, M, 3, 3, 1, N)
    ct = uniform_residues(s, moduli, (p.I, 2), N)
    w = L.hc_weights_preprocess(ctx, L.make_desc(C_, H, W, M, 3, 3, pad=1), K.astype(np.int8))
    ks = sample_indices(N, 24, 3)
    want = conv.conv_ct_pt(ct, conv.pack_weights(K, p), p, moduli, ks)
    d_in = to_dev(ct)
    out = torch.empty(p.O * 2 * nl * N, dtype=torch.int64, device="cuda")
    for vm in range(L.N_VARIANTS):
        for vf in range(L.N_VARIANTS):
            L.hc_ctx_set_variant(ctx, L.KIND_MAC_CONV, vm)
            L.hc_ctx_set_variant(ctx, L.KIND_NTT_FWD_CT, vf)
            L.hc_ctx_set_variant(ctx, L.KIND_NTT_INV_CT, vf)
            out.fill_(-1)
            L.hc_conv_ct_pt(ctx, w, d_in, out)
            torch.cuda.synchronize()
            got = to_host(out).reshape(p.O, 2, nl, N)
            assert np.array_equal(got[..., ks], want), (vm, vf)
    # fused MAC + inverse NTT (general slot lists): every output slot sums two products
    slots = np.arange(p.I) // 2
    n_out = int(slots.max()) + 1
    pt_c = uniform_residues(Stream(11, N), moduli, (p.I,), N)
    ptn = to_dev(pt_c)
    L.hc_ntt_fwd(ctx, ptn)
    want_m = np.zeros((n_out, 2, nl, len(ks)), dtype=object)
    for j in range(p.I):
        for c in range(2):
            for li, q in enumerate(moduli):
                want_m[slots[j], c, li] += core.negacyclic(ct[j, c, li], pt_c[j, li], q, ks).astype(object)
    for li, q in enumerate(moduli):
        want_m[:, :, li] %= q
    mo = torch.empty(n_out * 2 * nl * N, dtype=torch.int64, device="cuda")
    for vm in range(L.N_VARIANTS):
        L.hc_ctx_set_variant(ctx, L.KIND_MAC_INTT, vm)
        mo.fill_(-1)
        L.hc_ctpt_mac(ctx, d_in, ptn, slots, mo)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(mo).reshape(n_out, 2, nl, N)[..., ks], want_m.astype(np.uint64)), vm
    # standalone fused products: out[j] = ct[j] * pt[j]
    n = 5
    pc = uniform_residues(Stream(9, N), moduli, (n, 2), N)
    pt = uniform_residues(Stream(10, N), moduli, (n,), N)
    want_p = np.zeros((n, 2, nl, len(ks)), dtype=np.uint64)
    for j in range(n):
        for c in range(2):
            for li, q in enumerate(moduli):
                want_p[j, c, li] = core.negacyclic(pc[j, c, li], pt[j, li], q, ks)
    ptn = to_dev(pt)
    L.hc_ntt_fwd(ctx, ptn)
    po = torch.empty(n * 2 * nl * N, dtype=torch.int64, device="cuda")
    for v in range(L.N_VARIANTS):
        L.hc_ctx_set_variant(ctx, L.KIND_PRODUCT, v)
        po.fill_(-1)
        L.hc_ctpt_mac(ctx, to_dev(pc), ptn, np.arange(n), po)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(po).reshape(n, 2, nl, N)[..., ks], want_p), v


def test_blocked_mac_stage_ring_wraps(L):
    """A 1x1 layer with many output channels at N = 16384, L = 4: every CTA
    streams more weight stages than the ring holds, under every stage-size
    variant; sampled coefficients of a spread of outputs vs the oracle."""
    N, nl, C_, H, W, M = 16384, 4, 64, 16, 16, 300
    moduli = CANONICAL_PRIMES[:nl]
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    s = Stream(12, N)
    K = s.int8(M * C_).astype(np.int64).reshape(M, C_, 1, 1)
    p = conv.canonical_partition(C_, H, W, M, 1, 1, 0, N)
    ct = uniform_residues(s, moduli, (p.I, 2), N)
    w = L.hc_weights_preprocess(ctx, L.make_desc(C_, H, W, M, 1, 1), K.astype(np.int8))
    ks = sample_indices(N, 8, 4)
    outs = [0, 1, 37, 150, p.O - 2, p.O - 1]
    want = conv.conv_ct_pt(ct, conv.pack_weights(K, p), p, moduli, ks, outputs=outs)
    d_in = to_dev(ct)
    out = torch.empty(p.O * 2 * nl * N, dtype=torch.int64, device="cuda")
    ref = None
    for vm in range(L.N_VARIANTS):
        L.hc_ctx_set_variant(ctx, L.KIND_MAC_CONV, vm)
        out.fill_(-1)
        L.hc_conv_ct_pt(ctx, w, d_in, out)
        L.hc_ctx_device_status(ctx)
        torch.cuda.synchronize()
        got = to_host(out).reshape(p.O, 2, nl, N)
        assert np.array_equal(got[outs][..., ks], want), vm
        if ref is None:
            ref = out.clone()
        assert torch.equal(out, ref), vm


def test_variant_argument_errors(L):
    ctx = L.hc_ctx_create(4096, CANONICAL_PRIMES[:1], T_PLAIN)
    with pytest.raises(L.HcError):
        L.hc_ctx_set_variant(ctx, 99, 0)
    with pytest.raises(L.HcError):
        L.hc_ctx_set_variant(ctx, L.KIND_MAC_INTT, L.N_VARIANTS)


@pytest.mark.parametrize("N,nl,n", [(4096, 2, 700), (8192, 3, 400), (16384, 4, 120)])
def test_persistent_inverse_many_units(L, N, nl, n):
    """Variant 2 of the inverse transforms is a persistent kernel whose resident
    CTAs walk more polynomial limbs than there are CTAs: each loads the next
    limb while it finishes the current one. With n*L limbs well above the
    resident count (two or one CTAs per SM), every limb must match variant 0
    bit for bit, as a plain inverse NTT and as the inverse NTT of ciphertexts
    (two components per ciphertext), and the round trip must give the input."""
    moduli = CANONICAL_PRIMES[:nl]
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    a = uniform_residues(Stream(12, N), moduli, (n,), N)
    d0 = to_dev(a)
    L.hc_ntt_fwd(ctx, d0)
    outs = []
    for v in (0, 2):
        L.hc_ctx_set_variant(ctx, L.KIND_NTT_INV, v)
        d = d0.clone()
        L.hc_ntt_inv(ctx, d)
        torch.cuda.synchronize()
        outs.append(to_host(d))
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[1].reshape(a.shape), a)
    # ciphertext form (KIND_NTT_INV_CT): a 1x1 layer with O*2*L output limbs
    C_, H, W, M = 8, 12, 12, 160
    st = Stream(13, N)
    K = st.int8(M * C_).astype(np.int64).reshape(M, C_, 1, 1)
    p = conv.canonical_partition(C_, H, W, M, 1, 1, 0, N)
    assert p.O * 2 * nl > 600
    ct = uniform_residues(st, moduli, (p.I, 2), N)
    w = L.hc_weights_preprocess(ctx, L.make_desc(C_, H, W, M, 1, 1, pad=0), K.astype(np.int8))
    d_in = to_dev(ct)
    got = []
    for v in (0, 2):
        L.hc_ctx_set_variant(ctx, L.KIND_NTT_INV_CT, v)
        out = torch.full((p.O * 2 * nl * N,), -1, dtype=torch.int64, device="cuda")
        L.hc_conv_ct_pt(ctx, w, d_in, out)
        torch.cuda.synchronize()
        got.append(to_host(out).reshape(p.O, 2, nl, N))
    assert np.array_equal(got[0], got[1])
    ks = sample_indices(N, 8, M)
    want = conv.conv_ct_pt(ct, conv.pack_weights(K, p), p, moduli, ks)
    assert np.array_equal(got[1][..., ks], want)


def test_default_launch_shapes(L):
    """A new context starts with the measured-best transforms at N >= 8192 (the
    two-CTA cluster forward and the persistent / cluster inverse, variant 2) and
    variant 0 for everything else; a forward-inverse round trip under the defaults
    at every degree, with few and with many limbs, returns the input."""
    for N, nl in SIZES:
        ctx = L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN)
        want = 2 if N >= 8192 else 0
        for kind in (L.KIND_NTT_FWD, L.KIND_NTT_INV, L.KIND_NTT_FWD_CT, L.KIND_NTT_INV_CT):
            assert L.hc_ctx_get_variant(ctx, kind) == want, (N, kind)
        for kind in (L.KIND_MAC_INTT, L.KIND_PRODUCT, L.KIND_MAC_CONV, L.KIND_CONV_FORM):
            assert L.hc_ctx_get_variant(ctx, kind) == 0, (N, kind)
        for n in (1, 400 if N < 16384 else 160):
            a = uniform_residues(Stream(14, n), CANONICAL_PRIMES[:nl], (n,), N)
            d = to_dev(a)
            L.hc_ntt_fwd(ctx, d)
            L.hc_ntt_inv(ctx, d)
            torch.cuda.synchronize()
            assert np.array_equal(to_host(d).reshape(a.shape), a), (N, n)
