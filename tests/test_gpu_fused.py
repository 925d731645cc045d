"""GPU parity of the alternative launch forms of the convolution (Sec. 6.2:
NTT of the inputs, NTT-domain MAC, INTT of the outputs): form 1, one fused
persistent launch whose CTAs take tasks in order and wait on per-limb
completion counters; form 2, one forward -> MAC -> inverse chain per limb on
parallel streams.  Every output must equal, bit for bit, the three-launch
form (0) and the oracle's schoolbook convolution, for single layers of every
degree, many layers of one degree, and mixed degrees; repeated runs (counters
reset) and graph replays too."""
import numpy as np
import pytest

from gpu_util import sample_indices, to_dev, to_host
from oracle import conv
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream, uniform_residues

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (C, H, W, M, kh, kw, pad, N, L)
LAYERS = [
    (5, 7, 6, 3, 3, 3, 1, 4096, 2),
    (12, 9, 9, 4, 1, 1, 0, 8192, 3),
    (16, 13, 13, 40, 3, 3, 1, 8192, 3),
    (40, 7, 7, 70, 1, 1, 0, 8192, 3),
    (6, 20, 20, 3, 3, 3, 1, 16384, 4),
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
def ctxs(L):
    return {(N, nl): L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN) for N, nl in ((4096, 2), (8192, 3), (16384, 4))}


def _item(L, ctxs, shape, seed):
    C_, H, W, M, kh, kw, pad, N, nl = shape
    ctx = ctxs[(N, nl)]
    s = Stream(seed, 21)
    K = s.int8(M * C_ * kh * kw).astype(np.int64).reshape(M, C_, kh, kw)
    w = L.hc_weights_preprocess(ctx, L.make_desc(C_, H, W, M, kh, kw, pad=pad), K.astype(np.int8))
    ct = uniform_residues(s, CANONICAL_PRIMES[:nl], (w.I, 2), N)
    p = conv.canonical_partition(C_, H, W, M, kh, kw, pad, N)
    out = torch.empty(w.O * 2 * nl * N, dtype=torch.int64, device="cuda")
    return dict(ctx=ctx, w=w, K=K, p=p, ct=ct, nl=nl, d_in=to_dev(ct), d_out=out)


def _form(L, ctxs, v):
    for c in ctxs.values():
        L.hc_ctx_set_variant(c, L.KIND_CONV_FORM, v)


@pytest.mark.parametrize("form", [1, 2])
def test_fused_single_layers_match_three_launch_form_and_oracle(L, ctxs, form):
    for i, sh in enumerate(LAYERS):
        it = _item(L, ctxs, sh, 900 + i)
        _form(L, ctxs, 0)
        ref = torch.empty_like(it["d_out"])
        L.hc_conv_ct_pt(it["ctx"], it["w"], it["d_in"], ref)
        _form(L, ctxs, form)
        for _ in range(2):                         # counters are reset by every launch
            it["d_out"].fill_(-1)
            L.hc_conv_ct_pt(it["ctx"], it["w"], it["d_in"], it["d_out"])
            L.hc_ctx_device_status(it["ctx"])
            torch.cuda.synchronize()
            assert torch.equal(it["d_out"], ref), sh
        p, nl = it["p"], it["nl"]
        ks = sample_indices(p.N, 12, 40 + i)
        outs = sorted({0, p.O // 2, p.O - 1})
        got = to_host(it["d_out"]).reshape(p.O, 2, nl, p.N)
        want = conv.conv_ct_pt(it["ct"], conv.pack_weights(it["K"], p), p, CANONICAL_PRIMES[:nl], ks, outputs=outs)
        assert np.array_equal(got[outs][..., ks], want), sh
    _form(L, ctxs, 0)


@pytest.mark.parametrize("form", [1, 2])
def test_fused_plan_many_layers_and_degrees(L, ctxs, form):
    items = [_item(L, ctxs, sh, 950 + i) for i, sh in enumerate(LAYERS + LAYERS[1:4])]
    _form(L, ctxs, 0)
    refs = []
    for it in items:
        r = torch.empty_like(it["d_out"])
        L.hc_conv_ct_pt(it["ctx"], it["w"], it["d_in"], r)
        refs.append(r)
    _form(L, ctxs, form)
    plan = L.hc_plan_create([L.work_conv(it["ctx"], it["w"], it["d_in"], it["d_out"]) for it in items])
    # form 1: one fused launch per ring degree; form 2: three launches per limb and degree
    assert L.hc_plan_info(plan)[2] == (3 if form == 1 else 3 * (2 + 3 + 4))
    for rnd in range(4):                           # direct, capture, replays
        for it in items:
            it["d_out"].fill_(-1)
        L.hc_plan_run(plan)
        torch.cuda.synchronize()
        for it, r in zip(items, refs):
            assert torch.equal(it["d_out"], r), (rnd, it["p"])
    for c in ctxs.values():
        L.hc_ctx_device_status(c)
    _form(L, ctxs, 0)
