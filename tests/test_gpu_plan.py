"""GPU parity of plans (batching across layers, products and ring degrees,
Sec. 6.2): a plan's batched run (first run direct, later runs replay a CUDA
graph), its plain one-launch-per-product run and every item run alone through
hc_conv_ct_pt / hc_ctpt_mac give the same bits; standalone products of mixed
ring degree match the oracle's schoolbook products (App. C.1) on sampled
coefficients; conv items match the oracle's schoolbook convolution."""
import numpy as np
import pytest

from gpu_util import sample_indices, to_dev, to_host
from oracle import conv, core
from paper_2506_11586_gb300.inputs import (CANONICAL_PRIMES, SQUEEZENET_1_1, T_PLAIN, UNEVEN_CLASSES, Stream,
                                           conv_tensors, uneven_mix, uniform_residues)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (C, H, W, M, kh, kw, pad, N, L): ragged groups, 1x1 and 3x3, three ring degrees
LAYERS = [
    (5, 7, 6, 3, 3, 3, 1, 4096, 2),
    (12, 9, 9, 4, 1, 1, 0, 8192, 3),
    (16, 13, 13, 8, 3, 3, 1, 8192, 3),
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


def _empty(n_words):
    return torch.empty(n_words, dtype=torch.int64, device="cuda")


def _conv_item(L, ctxs, shape, seed):
    C_, H, W, M, kh, kw, pad, N, nl = shape
    ctx = ctxs[(N, nl)]
    s = Stream(seed, 5)
    K = s.int8(M * C_ * kh * kw).astype(np.int64).reshape(M, C_, kh, kw)
    w = L.hc_weights_preprocess(ctx, L.make_desc(C_, H, W, M, kh, kw, pad=pad), K.astype(np.int8))
    ct = uniform_residues(s, CANONICAL_PRIMES[:nl], (w.I, 2), N)
    p = conv.canonical_partition(C_, H, W, M, kh, kw, pad, N)
    return dict(ctx=ctx, w=w, K=K, p=p, ct=ct, d_in=to_dev(ct), d_out=_empty(w.O * 2 * nl * N))


def _single(L, it):
    ref = torch.empty_like(it["d_out"])
    L.hc_conv_ct_pt(it["ctx"], it["w"], it["d_in"], ref)
    return ref


def test_plan_convs_match_single_layers_and_oracle(L, ctxs):
    items = [_conv_item(L, ctxs, sh, 100 + i) for i, sh in enumerate(LAYERS)]
    plan = L.hc_plan_create([L.work_conv(it["ctx"], it["w"], it["d_in"], it["d_out"]) for it in items])
    n_prod, nbytes, launches = L.hc_plan_info(plan)
    assert n_prod == sum(it["p"].products for it in items)
    assert launches == 3 + 1 + 3   # forward and inverse per ring degree, one MAC launch
    for rnd in range(3):           # run 0 direct, run 1 captures + replays, run 2 replays
        if rnd == 2:               # new input values in the same buffers: the graph reads them at replay
            for i, it in enumerate(items):
                nl = len(it["ctx"].moduli)
                it["ct"] = uniform_residues(Stream(200 + i, 5), CANONICAL_PRIMES[:nl], (it["w"].I, 2), it["p"].N)
                it["d_in"].copy_(to_dev(it["ct"]))
            torch.cuda.synchronize()
        for it in items:
            it["d_out"].fill_(-1)
        L.hc_plan_run(plan)
        torch.cuda.synchronize()
        for it in items:
            assert torch.equal(it["d_out"], _single(L, it)), (rnd, it["p"])
    # oracle: every output of the ragged N = 4096 layer in full, sampled coefficients of the others
    for j, it in enumerate(items):
        p, nl = it["p"], len(it["ctx"].moduli)
        got = to_host(it["d_out"]).reshape(p.O, 2, nl, p.N)
        ks = None if j == 0 else sample_indices(p.N, 16, 30 + j)
        want = conv.conv_ct_pt(it["ct"], conv.pack_weights(it["K"], p), p, CANONICAL_PRIMES[:nl], ks,
                               outputs=None if j == 0 else [0, p.O - 1])
        if j == 0:
            assert np.array_equal(got, want)
        else:
            assert np.array_equal(got[[0, p.O - 1]][..., ks], want)
    # plain one-launch-per-product form: same bits
    keep = [it["d_out"].clone() for it in items]
    L.hc_plan_run_plain(plan)
    torch.cuda.synchronize()
    for it, k in zip(items, keep):
        assert torch.equal(it["d_out"], k)
    for it in items:
        L.hc_ctx_device_status(it["ctx"])


def _product_item(L, ctxs, N, nl, n, seed):
    ctx = ctxs[(N, nl)]
    s = Stream(seed, 6)
    ct = uniform_residues(s, CANONICAL_PRIMES[:nl], (n, 2), N)
    pt = uniform_residues(s, CANONICAL_PRIMES[:nl], (n,), N)
    d_pt = to_dev(pt)
    L.hc_ntt_fwd(ctx, d_pt)
    return dict(ctx=ctx, N=N, nl=nl, n=n, ct=ct, pt=pt, d_ct=to_dev(ct), d_pt=d_pt, d_out=_empty(n * 2 * nl * N))


def _check_products_oracle(it, which, nks, seed):
    N, nl = it["N"], it["nl"]
    got = to_host(it["d_out"]).reshape(it["n"], 2, nl, N)
    ks = sample_indices(N, nks, seed)
    for j in which:
        for c in range(2):
            for li, q in enumerate(CANONICAL_PRIMES[:nl]):
                want = core.negacyclic(it["ct"][j, c, li], it["pt"][j, li], q, ks)
                assert np.array_equal(got[j, c, li][ks], want), (N, j, c, li)


def test_plan_mixed_degree_products_and_conv(L, ctxs):
    prods = [_product_item(L, ctxs, N, nl, n, 300 + n) for (N, nl, n) in ((4096, 2, 5), (8192, 3, 4), (16384, 4, 3))]
    cv = _conv_item(L, ctxs, LAYERS[2], 400)
    items = [L.work_products(it["ctx"], it["d_ct"], it["d_pt"], it["d_out"]) for it in prods]
    items.append(L.work_conv(cv["ctx"], cv["w"], cv["d_in"], cv["d_out"]))
    plan = L.hc_plan_create(items)
    assert L.hc_plan_info(plan)[0] == 12 + cv["p"].products
    for _ in range(3):
        L.hc_plan_run(plan)
    torch.cuda.synchronize()
    for it in prods:
        _check_products_oracle(it, range(it["n"]), 24, it["N"])
        ref = torch.empty_like(it["d_out"])      # per-degree fused product launch: same bits
        L.hc_ctpt_mac(it["ctx"], it["d_ct"], it["d_pt"], np.arange(it["n"]), ref)
        torch.cuda.synchronize()
        assert torch.equal(ref, it["d_out"])
    assert torch.equal(cv["d_out"], _single(L, cv))
    keep = [it["d_out"].clone() for it in prods]
    L.hc_plan_run_plain(plan)
    torch.cuda.synchronize()
    for it, k in zip(prods, keep):
        assert torch.equal(it["d_out"], k)


def test_plan_products_in_place(L, ctxs):
    it = _product_item(L, ctxs, 8192, 3, 3, 77)
    ref = torch.empty_like(it["d_ct"])
    L.hc_ctpt_mac(it["ctx"], it["d_ct"], it["d_pt"], np.arange(3), ref)
    plan = L.hc_plan_create([L.work_products(it["ctx"], it["d_ct"], it["d_pt"], it["d_ct"])])
    L.hc_plan_run(plan)
    torch.cuda.synchronize()
    assert torch.equal(it["d_ct"], ref)


def test_plan_rejects_overlapping_items(L, ctxs):
    a = _product_item(L, ctxs, 4096, 2, 2, 1)
    b = _product_item(L, ctxs, 4096, 2, 2, 2)
    with pytest.raises(L.HcError) as e:     # two items write the same output
        L.hc_plan_create([L.work_products(a["ctx"], a["d_ct"], a["d_pt"], a["d_out"]),
                          L.work_products(b["ctx"], b["d_ct"], b["d_pt"], a["d_out"])])
    assert e.value.status == L.HC_ERR_INVALID_ARG
    with pytest.raises(L.HcError) as e:     # output shifted against its own input
        big = _empty(3 * 2 * 2 * 4096)
        L.hc_plan_create([L.work_products(a["ctx"], big[: 2 * 2 * 2 * 4096], a["d_pt"], big[2 * 2 * 4096:])])
    assert e.value.status == L.HC_ERR_INVALID_ARG
    with pytest.raises(L.HcError):          # one item's output is another's input
        L.hc_plan_create([L.work_products(a["ctx"], a["d_ct"], a["d_pt"], a["d_out"]),
                          L.work_products(b["ctx"], a["d_out"], b["d_pt"], b["d_out"])])
    # shared read-only inputs are fine
    plan = L.hc_plan_create([L.work_products(a["ctx"], a["d_ct"], a["d_pt"], a["d_out"]),
                             L.work_products(b["ctx"], a["d_ct"], a["d_pt"], b["d_out"])])
    L.hc_plan_run(plan)
    torch.cuda.synchronize()
    assert torch.equal(a["d_out"], b["d_out"])


def test_plan_autotune_keeps_bits_and_caches(L, ctxs, tmp_path):
    items = [_conv_item(L, ctxs, sh, 500 + i) for i, sh in enumerate(LAYERS[:3])]
    plan = L.hc_plan_create([L.work_conv(it["ctx"], it["w"], it["d_in"], it["d_out"]) for it in items])
    L.hc_plan_run(plan)
    torch.cuda.synchronize()
    before = [it["d_out"].clone() for it in items]
    cache = str(tmp_path / "tune.txt")
    L.hc_plan_autotune(plan, cache)
    lines = open(cache).read().split("\n")
    lines = [x for x in lines if x]
    assert len(lines) == 2 * 4        # fwd_ct, blocked MAC, inv_ct and launch form for each of the two contexts
    chosen = {k: L.hc_ctx_get_variant(ctxs[(4096, 2)], k)
              for k in (L.KIND_NTT_FWD_CT, L.KIND_MAC_CONV, L.KIND_NTT_INV_CT, L.KIND_CONV_FORM)}
    for _ in range(2):                 # direct run, then graph captured with the tuned variants
        L.hc_plan_run(plan)
    torch.cuda.synchronize()
    for it, b in zip(items, before):
        assert torch.equal(it["d_out"], b)
    # a second autotune reads the cache and changes nothing
    for k in chosen:
        L.hc_ctx_set_variant(ctxs[(4096, 2)], k, (chosen[k] + 1) % L.N_VARIANTS)
    L.hc_plan_autotune(plan, cache)
    assert len([x for x in open(cache).read().split("\n") if x]) == 8
    assert {k: L.hc_ctx_get_variant(ctxs[(4096, 2)], k) for k in chosen} == chosen


def test_uneven_batch_2000_products(L, ctxs):
    """2000 standalone products, 40/40/20 over (4096, 2), (8192, 3), (16384, 4),
    in one persistent launch: sampled coefficients of a spread of products vs
    the oracle; every product vs the plain one-launch-per-product run."""
    labels = uneven_mix(2000, seed=4)
    prods = []
    for cls, (N, nl, _) in enumerate(UNEVEN_CLASSES):
        prods.append(_product_item(L, ctxs, N, nl, int((labels == cls).sum()), 4000 + cls))
    assert [it["n"] for it in prods] == [800, 800, 400]
    plan = L.hc_plan_create([L.work_products(it["ctx"], it["d_ct"], it["d_pt"], it["d_out"]) for it in prods])
    assert L.hc_plan_info(plan)[:1] == (2000,)
    assert L.hc_plan_info(plan)[2] == 1
    L.hc_plan_run(plan)
    L.hc_plan_run(plan)
    torch.cuda.synchronize()
    for it in prods:
        _check_products_oracle(it, [0, it["n"] // 2, it["n"] - 1], 12, 7 * it["N"])
    batched = [it["d_out"].clone() for it in prods]
    for it in prods:
        it["d_out"].fill_(0)
    L.hc_plan_run_plain(plan)
    torch.cuda.synchronize()
    for it, b in zip(prods, batched):
        assert torch.equal(it["d_out"], b)


def test_squeezenet_plan_matches_layers(L, ctxs):
    """Every stride-1 SqueezeNet-1.1 layer at N = 8192, L = 3 in one plan:
    each layer's outputs equal the single-layer call's, bit for bit; two
    layers are spot-checked against the oracle's schoolbook convolution."""
    ctx = ctxs[(8192, 3)]
    items = []
    for i, sh in enumerate(SQUEEZENET_1_1):
        x, K = conv_tensors(sh, seed=3)
        w = L.hc_weights_preprocess(ctx, L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad),
                                    K.astype(np.int8))
        ct = uniform_residues(Stream(3, 100 + i), CANONICAL_PRIMES[:3], (w.I, 2), 8192)
        items.append(dict(ctx=ctx, w=w, K=K, sh=sh, ct=ct, d_in=to_dev(ct), d_out=_empty(w.O * 2 * 3 * 8192)))
    assert len(items) == 25
    plan = L.hc_plan_create([L.work_conv(ctx, it["w"], it["d_in"], it["d_out"]) for it in items])
    n_prod = L.hc_plan_info(plan)[0]
    assert n_prod == sum(it["w"].desc.M * it["w"].I for it in items) == 23568
    L.hc_plan_run(plan)
    L.hc_plan_run(plan)
    torch.cuda.synchronize()
    for it in items:
        assert torch.equal(it["d_out"], _single(L, it)), it["sh"].name
    ks = sample_indices(8192, 8, 5)
    for it in (items[0], items[-1]):
        sh = it["sh"]
        p = conv.canonical_partition(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, sh.pad, 8192)
        got = to_host(it["d_out"]).reshape(p.O, 2, 3, 8192)
        outs = [0, p.O // 2, p.O - 1]
        want = conv.conv_ct_pt(it["ct"], conv.pack_weights(it["K"], p), p, CANONICAL_PRIMES[:3], ks, outputs=outs)
        assert np.array_equal(got[outs][..., ks], want), sh.name
    L.hc_ctx_device_status(ctx)
