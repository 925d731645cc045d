"""GPU parity of hc_ctpt_mac (NTT-domain multiply-accumulate, Sec. 6.2) on the
plain ct x pt batch: N = 4096, two 50-bit primes = 1 mod 8192, 16 products
with coefficients uniform in [0, q_i), checked against the oracle's dense
schoolbook products, every coefficient, bit-exact."""
import numpy as np
import pytest

from gpu_util import to_dev, to_host
from oracle import core
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream, uniform_residues

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N, NL, NPROD = 4096, 2, 16
MODULI = CANONICAL_PRIMES[:NL]


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_11586_gb300 import _lib
    from paper_2506_11586_gb300.build import build
    build()
    return _lib


@pytest.fixture(scope="module")
def batch():
    s = Stream(1, 0)
    ct = uniform_residues(s, MODULI, (NPROD, 2), N)        # [16][2][2][N]
    pt = uniform_residues(s, MODULI, (NPROD,), N)          # [16][2][N] coefficient domain
    # oracle: every product, dense schoolbook per (product, component, limb)
    b = np.broadcast_to(pt[:, None], ct.shape)
    prods = core.negacyclic_batch(ct, b, MODULI)           # [16][2][2][N]
    return ct, pt, prods


def _sum_mod(prods, idx):
    out = np.zeros(prods.shape[1:], dtype=object)
    for j in idx:
        out = out + prods[j].astype(object)
    for li, q in enumerate(MODULI):
        out[:, li] = out[:, li] % q
    return out.astype(np.uint64)


def _pt_ntt(L, ctx, pt):
    d = to_dev(pt)
    L.hc_ntt_fwd(ctx, d)
    return d


def test_independent_products(L, batch):
    ct, pt, prods = batch
    ctx = L.hc_ctx_create(N, MODULI, T_PLAIN)
    ptn = _pt_ntt(L, ctx, pt)
    out = torch.empty(NPROD * 2 * NL * N, dtype=torch.int64, device="cuda")
    L.hc_ctpt_mac(ctx, to_dev(ct), ptn, np.arange(NPROD), out)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(out).reshape(prods.shape), prods)


def test_accumulated_into_one_slot(L, batch):
    ct, pt, prods = batch
    ctx = L.hc_ctx_create(N, MODULI, T_PLAIN)
    ptn = _pt_ntt(L, ctx, pt)
    out = torch.empty(2 * NL * N, dtype=torch.int64, device="cuda")
    L.hc_ctpt_mac(ctx, to_dev(ct), ptn, np.zeros(NPROD), out)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(out).reshape(2, NL, N), _sum_mod(prods, range(NPROD)))


def test_mixed_slots_with_empty_slots(L, batch):
    ct, pt, prods = batch
    ctx = L.hc_ctx_create(N, MODULI, T_PLAIN)
    ptn = _pt_ntt(L, ctx, pt)
    slots = np.array([0, 0, 2, 2, 2, 5, 6, 6, 6, 6, 0, 2, 5, 5, 9, 0], dtype=np.uint32)
    n_out = 11
    out = torch.full((n_out * 2 * NL * N,), 12345, dtype=torch.int64, device="cuda")
    L.hc_ctpt_mac(ctx, to_dev(ct), ptn, slots, out)
    torch.cuda.synchronize()
    got = to_host(out).reshape(n_out, 2, NL, N)
    for s_ in range(n_out):
        idx = np.nonzero(slots == s_)[0]
        want = _sum_mod(prods, idx) if idx.size else np.zeros((2, NL, N), dtype=np.uint64)
        assert np.array_equal(got[s_], want), s_


def test_single_and_empty_batches(L, batch):
    ct, pt, prods = batch
    ctx = L.hc_ctx_create(N, MODULI, T_PLAIN)
    ptn = _pt_ntt(L, ctx, pt[:1])
    out = torch.empty(3 * 2 * NL * N, dtype=torch.int64, device="cuda")
    L.hc_ctpt_mac(ctx, to_dev(ct[:1]), ptn, np.array([1]), out)   # one product, slots 0 and 2 empty
    torch.cuda.synchronize()
    got = to_host(out).reshape(3, 2, NL, N)
    assert np.all(got[0] == 0) and np.all(got[2] == 0)
    assert np.array_equal(got[1], prods[0])
    empty = torch.empty(0, dtype=torch.int64, device="cuda")
    L.hc_ctpt_mac(ctx, empty, empty, np.zeros(0), out)             # n = 0: all slots zero
    torch.cuda.synchronize()
    assert np.all(to_host(out) == 0)
    with pytest.raises(L.HcError) as e:
        L.hc_ctpt_mac(ctx, to_dev(ct[:1]), ptn, np.array([3]), out)  # slot >= n_out
    assert e.value.status == L.HC_ERR_INVALID_ARG
