"""GPU parity of hc_ntt_fwd / hc_ntt_inv (App. C.1) against the oracle's
O(N^2) definition, bit-exact, through the C ABI."""
import numpy as np
import pytest

from gpu_util import sample_indices, to_dev, to_host
from oracle import core
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


@pytest.mark.parametrize("N,nl", [(4096, 2), (8192, 3), (16384, 4)])
def test_ntt_fwd_inv_vs_oracle(L, N, nl):
    moduli = CANONICAL_PRIMES[:nl]
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    info = L.hc_ctx_info(ctx)
    psis = [core.min_psi(q, N) for q in moduli]
    assert info["psi"] == psis and info["moduli"] == list(moduli)
    n = 3  # several polys: a ragged count of CTAs per limb
    a = uniform_residues(Stream(1, N), moduli, (n,), N)
    d = to_dev(a)
    L.hc_ntt_fwd(ctx, d)
    torch.cuda.synchronize()
    A = to_host(d).reshape(n, nl, N)
    ks = sample_indices(N, 96, N)
    for p in range(n):
        for li, q in enumerate(moduli):
            if N == 4096 and p == 0:
                assert np.array_equal(A[p, li], core.ntt(a[p, li], q, psis[li])), (p, li)
            else:
                assert np.array_equal(A[p, li][ks], core.ntt(a[p, li], q, psis[li], ks)), (p, li)
    assert int(A.max()) < max(moduli)
    # inverse: back to the input, every coefficient
    L.hc_ntt_inv(ctx, d)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(d).reshape(n, nl, N), a)
    # inverse against the oracle on an independent NTT-domain input
    B = uniform_residues(Stream(2, N), moduli, (2,), N)
    d = to_dev(B)
    L.hc_ntt_inv(ctx, d)
    torch.cuda.synchronize()
    b = to_host(d).reshape(2, nl, N)
    for p in range(2):
        for li, q in enumerate(moduli):
            assert np.array_equal(b[p, li][ks], core.intt(B[p, li], q, psis[li], ks)), (p, li)


def test_ntt_edge_inputs(L):
    N, moduli = 8192, CANONICAL_PRIMES[:2]
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    a = np.zeros((4, 2, N), dtype=np.uint64)
    a[1, :, 0] = 1                                  # delta -> all ones
    for li, q in enumerate(moduli):
        a[2, li, :] = q - 1                         # all maximal residues
    a[3, :, 5] = 1                                  # monomial X^5
    d = to_dev(a)
    L.hc_ntt_fwd(ctx, d)
    torch.cuda.synchronize()
    A = to_host(d).reshape(4, 2, N)
    assert np.all(A[0] == 0)
    assert np.all(A[1] == 1)
    ks = sample_indices(N, 32, 5)
    for li, q in enumerate(moduli):
        psi = core.min_psi(q, N)
        assert np.array_equal(A[2, li][ks], core.ntt(a[2, li], q, psi, ks))
        assert np.array_equal(A[3, li][ks], core.ntt(a[3, li], q, psi, ks))
    L.hc_ntt_inv(ctx, d)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(d).reshape(4, 2, N), a)


def test_ntt_empty_and_errors(L):
    ctx = L.hc_ctx_create(4096, CANONICAL_PRIMES[:1], T_PLAIN)
    empty = torch.empty(0, dtype=torch.int64, device="cuda")
    L.hc_ntt_fwd(ctx, empty)            # n_polys == 0: no-op
    L.hc_ntt_inv(ctx, empty)
    with pytest.raises(L.HcError) as e:
        L.hc_ctx_create(4096, [CANONICAL_PRIMES[0], CANONICAL_PRIMES[0]], T_PLAIN)
    assert e.value.status == L.HC_ERR_BAD_MODULUS


def test_checked_mode_rejects_out_of_range(L):
    N, moduli = 4096, CANONICAL_PRIMES[:2]
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN, flags=L.HC_CTX_CHECKED)
    a = uniform_residues(Stream(9, 0), moduli, (2,), N)
    d = to_dev(a)
    L.hc_ntt_fwd(ctx, d)                # in range: fine
    L.hc_ntt_inv(ctx, d)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(d).reshape(2, 2, N), a)
    a[1, 1, 77] = moduli[1]             # == q: out of range
    d = to_dev(a)
    with pytest.raises(L.HcError) as e:
        L.hc_ntt_fwd(ctx, d)
    assert e.value.status == L.HC_ERR_RANGE
    torch.cuda.synchronize()
    assert np.array_equal(to_host(d).reshape(2, 2, N), a)   # untouched
