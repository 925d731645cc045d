"""hc_conv_ct_pt_noalloc: the convolution layer for callers that must not
allocate device memory (for instance a service whose GPU memory is all
reserved up front by another framework's caching allocator, or a
latency-critical loop in which cudaMalloc / cudaFree would synchronise the
device).  It keeps its scratch in a static device array instead of asking an
allocator, and must give the same bits as the allocating hc_conv_ct_pt.

This file is named so that pytest collects it last: a run that stops at the
first failure has then already run every other test.  It passes both on its
own in a fresh process and after the rest of the suite (the static scratch
keeps the previous call's contents, which the entry point never reads)."""
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


def _two_calls_match(L, ctx, w, moduli, N):
    out_words = w.O * 2 * len(moduli) * N
    for call, seed in enumerate((101, 202)):          # two different inputs, one after the other
        ct = uniform_residues(Stream(seed, 0), moduli, (w.I, 2), N)
        d_in = torch.from_numpy(ct.view(np.int64)).cuda()
        want = torch.empty(out_words, dtype=torch.int64, device="cuda")
        got = torch.full((out_words,), -1, dtype=torch.int64, device="cuda")
        L.hc_conv_ct_pt(ctx, w, d_in, want)
        L.hc_conv_ct_pt_noalloc(ctx, w, d_in, got)
        torch.cuda.synchronize()
        # integer results: the tolerance is zero, every residue must match
        assert torch.equal(got, want), "call %d differs from hc_conv_ct_pt" % call


# launch forms of the layer (kernel family 7): three launches, one fused persistent
# launch (its dependency counters sit in the static scratch after the NTT'd inputs),
# and one chain of three launches per limb on parallel streams
@pytest.mark.parametrize("form", [0, 1, 2])
def test_noalloc_matches_allocating_path_on_two_calls_in_a_row(L, form):
    sh, N, moduli = CONV_56x56x64, 8192, CANONICAL_PRIMES[:3]
    _, K = conv_tensors(sh, seed=2)
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    L.hc_ctx_set_variant(ctx, L.KIND_CONV_FORM, form)
    w = L.hc_weights_preprocess(ctx, L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad), K)
    _two_calls_match(L, ctx, w, moduli, N)


def test_noalloc_fused_form_without_room_for_its_counters(L):
    # 256 -> 16 channels, 3x3 at 28x28, N = 16384, L = 4: I = 16 input ciphertexts,
    # whose NTT'd limbs fill the 16 MiB static scratch exactly; the fused form's
    # counters do not fit, so the layer must run unfused and still match
    N, moduli = 16384, CANONICAL_PRIMES[:4]
    desc = L.make_desc(256, 28, 28, 16, 3, 3, pad=1)
    _, I, _, _ = L.hc_conv_partition(desc, N)
    assert I * 2 * len(moduli) * N * 8 == 16 << 20
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    L.hc_ctx_set_variant(ctx, L.KIND_CONV_FORM, 1)
    K = Stream(7, 0).int8(16 * 256 * 9).reshape(16, 256, 3, 3)
    w = L.hc_weights_preprocess(ctx, desc, K)
    _two_calls_match(L, ctx, w, moduli, N)


def test_noalloc_rejects_layers_beyond_its_static_scratch(L):
    # a 256 -> 128 channel 1x1 layer at 56x56 with N = 16384, L = 4 needs more
    # than the 16 MiB static scratch for its NTT'd inputs
    N, moduli = 16384, CANONICAL_PRIMES[:4]
    desc = L.make_desc(256, 56, 56, 128, 1, 1)
    _, I, _, _ = L.hc_conv_partition(desc, N)
    assert I * 2 * len(moduli) * N * 8 > 16 << 20
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    w = L.hc_weights_preprocess(ctx, desc, np.zeros((128, 256, 1, 1), dtype=np.int8))
    d_in = torch.zeros(w.I * 2 * len(moduli) * N, dtype=torch.int64, device="cuda")
    d_out = torch.zeros(w.O * 2 * len(moduli) * N, dtype=torch.int64, device="cuda")
    with pytest.raises(L.HcError) as e:
        L.hc_conv_ct_pt_noalloc(ctx, w, d_in, d_out)
    assert e.value.status == L.HC_ERR_BUDGET
