"""The three NTT-preprocessing modes of a convolution's weights (the paper's
linear layers with offline, online or no NTT preprocessing, Sec. 9; Sec. 6.2):
offline (NTT'd once, resident), online (NTT'd by every call) and no NTT (a
direct negacyclic product sum in the coefficient domain) give the same bits,
equal to the oracle's schoolbook convolution, for every ring degree; the
server step runs in every mode; modes the plain form and plans do not take
are refused."""
import numpy as np
import pytest

from gpu_util import sample_indices, to_dev, to_host
from oracle import conv
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


@pytest.mark.parametrize("shape", [
    (5, 7, 6, 3, 3, 3, 1, 4096, 2),
    (12, 9, 9, 4, 1, 1, 0, 8192, 3),
    (6, 20, 20, 3, 3, 3, 1, 16384, 4),
])
def test_modes_agree_with_each_other_and_the_oracle(L, shape):
    C_, H, W, M, kh, kw, pad, N, nl = shape
    moduli = CANONICAL_PRIMES[:nl]
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    s = Stream(70, N)
    K = s.int8(M * C_ * kh * kw).astype(np.int64).reshape(M, C_, kh, kw)
    d = L.make_desc(C_, H, W, M, kh, kw, pad=pad)
    ws = [L.hc_weights_preprocess_ex(ctx, d, K.astype(np.int8), mode) for mode in range(3)]
    p = conv.canonical_partition(C_, H, W, M, kh, kw, pad, N)
    ct = uniform_residues(s, moduli, (p.I, 2), N)
    d_in = to_dev(ct)
    outs = []
    for w in ws:
        out = torch.empty(p.O * 2 * nl * N, dtype=torch.int64, device="cuda")
        out.fill_(-1)
        L.hc_conv_ct_pt(ctx, w, d_in, out)
        torch.cuda.synchronize()
        outs.append(out)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    ks = sample_indices(N, 16, 3)
    want = conv.conv_ct_pt(ct, conv.pack_weights(K, p), p, moduli, ks)
    assert np.array_equal(to_host(outs[2]).reshape(p.O, 2, nl, N)[..., ks], want)
    # the server step in every mode
    S = L.slot_count(ws[0])
    slots = [torch.empty(p.O * nl * S, dtype=torch.int64, device="cuda") for _ in ws]
    share = to_dev(s.below(T_PLAIN, C_ * H * W))
    mask = to_dev(s.below(T_PLAIN, M * p.Ho * p.Wo))
    for w, sl in zip(ws, slots):
        full = torch.empty(p.O * 2 * nl * N, dtype=torch.int64, device="cuda")
        L.hc_conv_server_step(ctx, w, d_in, share, mask, full, sl)
    torch.cuda.synchronize()
    assert torch.equal(slots[0], slots[1]) and torch.equal(slots[0], slots[2])
    # the no-NTT mode also runs without any allocation
    out = torch.empty_like(outs[0])
    L.hc_conv_ct_pt_noalloc(ctx, ws[2], d_in, out)
    torch.cuda.synchronize()
    assert torch.equal(out, outs[0])
    # refusals
    for w in ws[1:]:
        with pytest.raises(L.HcError) as e:
            L.hc_conv_ct_pt_plain(ctx, w, d_in, out)
        assert e.value.status == L.HC_ERR_UNSUPPORTED
        with pytest.raises(L.HcError):
            L.hc_plan_create([L.work_conv(ctx, w, d_in, out)])
    with pytest.raises(L.HcError):
        L.hc_weights_data(ws[2])
    L.hc_ctx_device_status(ctx)
