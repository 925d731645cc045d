"""GPU parity of the Z_P layer operations (SecONNds-P's HELiKs-style linear
layers, Sec. 6.1; rotations by key switching, Sec. 2.1): hc_ct_rotate and
hc_mac_rotate must equal, every uint64 of every output, the oracle's key-switched
rotation and multiply-accumulate-rotate iteration on the same BFV ciphertexts
and Galois keys, and decrypt to the rotated / accumulated slot vectors."""
import numpy as np
import pytest

from gpu_util import to_dev, to_host
from oracle import bfv, zp
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, Stream

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


def _setup(N, nl, pbits, seed, g=5):
    kp = zp.KsParams(N, tuple(CANONICAL_PRIMES[:nl]), CANONICAL_PRIMES[nl])
    P = zp.plaintext_prime(N, pbits)
    s = Stream(seed, 0)
    sk = s.ternary(N)
    a = np.stack([np.stack([s.below(q, N) for q in kp.qp]) for _ in range(nl)])
    e = np.stack([s.rounded_gaussian(N) for _ in range(nl)])
    gk = zp.galois_key(kp, sk, g, a, e)
    params = zp.bfv_params(N, kp.moduli, P)
    return kp, P, s, sk, gk, params


def _encrypt(s, params, sk, poly):
    a = np.stack([s.below(q, params.N) for q in params.moduli])
    return bfv.encrypt(params, sk, poly, a, s.rounded_gaussian(params.N))


def _slots(s, N, P):
    return s.below(P, N).astype(np.int64).reshape(2, N // 2)


@pytest.mark.parametrize("g", [5, None])   # None: the inverse element (right rotation)
def test_rotation_matches_oracle_and_decrypts(L, g):
    N, nl = 4096, 2
    g = g or pow(5, -1, 2 * N)
    kp, P, s, sk, gk, params = _setup(N, nl, 17, 81, g)
    ctx = L.hc_ctx_create(N, kp.moduli, P)
    key = L.hc_galois_key_create(ctx, kp.special, g, gk)
    ms = [_slots(s, N, P) for _ in range(3)]
    cts = np.stack([_encrypt(s, params, sk, zp.encode(m, N, P)) for m in ms])
    out = torch.full((3 * 2 * nl * N,), -1, dtype=torch.int64, device="cuda")
    L.hc_ct_rotate(ctx, key, to_dev(cts), out)
    L.hc_ctx_device_status(ctx)
    got = to_host(out).reshape(3, 2, nl, N)
    shift = -1 if g == 5 else 1
    for c in range(3):
        want = zp.rotate(cts[c], gk, g, kp)
        assert np.array_equal(got[c], want), c
        dec = bfv.decrypt_at(params, sk, got[c], list(range(N)))
        assert np.array_equal(zp.decode(dec.astype(np.uint64), N, P), np.roll(ms[c], shift, axis=1))


def test_rotation_full_size_sampled(L):
    """N = 8192, three 50-bit primes and a 37-bit plaintext prime (SqueezeNet's precision)."""
    N, nl = 8192, 3
    kp, P, s, sk, gk, params = _setup(N, nl, 37, 82)
    ctx = L.hc_ctx_create(N, kp.moduli, P)
    key = L.hc_galois_key_create(ctx, kp.special, 5, gk)
    m = _slots(s, N, P)
    ct = _encrypt(s, params, sk, zp.encode(m, N, P))
    out = torch.empty(2 * nl * N, dtype=torch.int64, device="cuda")
    L.hc_ct_rotate(ctx, key, to_dev(ct), out)
    L.hc_ctx_device_status(ctx)
    got = to_host(out).reshape(2, nl, N)
    assert np.array_equal(got, zp.rotate(ct, gk, 5, kp))
    dec = bfv.decrypt_at(params, sk, got, list(range(N)))
    assert np.array_equal(zp.decode(dec.astype(np.uint64), N, P), np.roll(m, -1, axis=1))


@pytest.mark.parametrize("n", [1, 2, 5])
def test_mac_rotate_matches_oracle_and_slot_formula(L, n):
    N, nl = 4096, 2
    kp, P, s, sk, gk, params = _setup(N, nl, 17, 83 + n)
    ctx = L.hc_ctx_create(N, kp.moduli, P)
    key = L.hc_galois_key_create(ctx, kp.special, 5, gk)
    m = _slots(s, N, P)
    ws = [_slots(s, N, P) for _ in range(n)]
    ct = _encrypt(s, params, sk, zp.encode(m, N, P))
    polys = np.stack([zp.encode(w, N, P) for w in ws])
    w_ntt = torch.empty(n * nl * N, dtype=torch.int64, device="cuda")
    L.hc_zp_plain_preprocess(ctx, P, polys, w_ntt)
    out = torch.full((2 * nl * N,), -1, dtype=torch.int64, device="cuda")
    L.hc_mac_rotate(ctx, key, to_dev(ct), w_ntt, out)
    L.hc_ctx_device_status(ctx)
    got = to_host(out).reshape(2, nl, N)
    lifts = [zp.lift_plain(p, P, kp.moduli) for p in polys]
    assert np.array_equal(got, zp.mac_rotate(ct, lifts, gk, 5, kp))
    dec = bfv.decrypt_at(params, sk, got, list(range(N)))
    assert np.array_equal(zp.decode(dec.astype(np.uint64), N, P), zp.slot_mac_rotate(m, ws, P))


def test_rotation_argument_errors(L):
    N, nl = 4096, 2
    kp, P, s, sk, gk, params = _setup(N, nl, 17, 90)
    ctx = L.hc_ctx_create(N, kp.moduli, P)
    for g, special, status in ((4, kp.special, L.HC_ERR_INVALID_ARG), (2 * N + 1, kp.special, L.HC_ERR_INVALID_ARG),
                               (5, kp.moduli[0], L.HC_ERR_BAD_MODULUS), (5, 97, L.HC_ERR_BAD_MODULUS)):
        with pytest.raises(L.HcError) as e:
            L.hc_galois_key_create(ctx, special, g, gk)
        assert e.value.status == status, (g, special)
    key = L.hc_galois_key_create(ctx, kp.special, 5, gk)
    buf = torch.zeros(2 * nl * N, dtype=torch.int64, device="cuda")
    with pytest.raises(L.HcError) as e:
        L.hc_ct_rotate(ctx, key, buf, buf)                   # in place
    assert e.value.status == L.HC_ERR_INVALID_ARG
    other = L.hc_ctx_create(N, kp.moduli, P)
    with pytest.raises(L.HcError) as e:
        L.hc_ct_rotate(other, key, buf, torch.zeros_like(buf))
    assert e.value.status == L.HC_ERR_INVALID_ARG
    with pytest.raises(L.HcError) as e:
        L.hc_zp_plain_preprocess(ctx, P, np.full(N, P, dtype=np.uint64), torch.empty(nl * N, dtype=torch.int64,
                                                                                     device="cuda"))
    assert e.value.status == L.HC_ERR_RANGE


def _plain_ctx(L, N, P):
    return L.hc_ctx_create(N, [P], P)


@pytest.mark.parametrize("N", [4096, 8192])
def test_simd_encode_decode_match_oracle(L, N):
    """hc_zp_encode / hc_zp_decode against the oracle's BFV batching (the slot
    layout of the rotations): every coefficient of every encoding equal, decode
    inverts encode, and the encodings multiply slot-wise (sigma_5 rotates them)."""
    P = zp.plaintext_prime(N, 37)
    ctx_p = _plain_ctx(L, N, P)
    s = Stream(95, N)
    ms = np.stack([_slots(s, N, P) for _ in range(3)])
    d_slots = to_dev(ms)
    d_poly = torch.full((3 * N,), -1, dtype=torch.int64, device="cuda")
    L.hc_zp_encode(ctx_p, d_slots, d_poly)
    torch.cuda.synchronize()
    got = to_host(d_poly).reshape(3, N)
    for i in range(3 if N == 4096 else 1):                    # the oracle's encoder is O(N^2)
        assert np.array_equal(got[i], zp.encode(ms[i], N, P)), i
    back = torch.full_like(d_slots, -1)
    L.hc_zp_decode(ctx_p, d_poly, back)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(back).reshape(ms.shape), ms)
    for i in range(3):
        assert np.array_equal(zp.decode(got[i], N, P), ms[i])


def test_matvec_layer_decrypts_to_the_matrix_product(L):
    """A HELiKs-style matrix-vector layer end to end on the GPU: the server's
    weights through hc_zp_matvec_preprocess (diagonals, SIMD encoding, lift, NTT),
    the client's periodic input vector encrypted, hc_mac_rotate with the Galois key
    for sigma_5; decryption gives W v mod P in the input's periodic format. The
    plaintexts equal the oracle's diagonal encodings, and a rectangular matrix is
    padded as the oracle pads it. N = 8192, three limbs, a 37-bit P."""
    N, nl = 8192, 3
    kp, P, s, sk, gk, params = _setup(N, nl, 37, 96)
    ctx = L.hc_ctx_create(N, kp.moduli, P)
    ctx_p = _plain_ctx(L, N, P)
    key = L.hc_galois_key_create(ctx, kp.special, 5, gk)
    n_out, n_in = 12, 16
    Wm = s.below(P, n_out * n_in).astype(np.uint64).reshape(n_out, n_in)
    v = s.below(P, n_in).astype(np.int64)
    n = zp.matvec_size(n_out, n_in)
    w_ntt = torch.empty(n * nl * N, dtype=torch.int64, device="cuda")
    assert L.hc_zp_matvec_preprocess(ctx, ctx_p, Wm, w_ntt) == n
    # the resident plaintexts are the NTT of the lifted oracle encodings of the diagonals
    diag = zp.matvec_diagonals(Wm.astype(np.int64), N, P)
    for i in (0, n - 1):
        lift = zp.lift_plain(zp.encode(diag[i], N, P), P, kp.moduli)
        chk = to_dev(lift)
        L.hc_ntt_fwd(ctx, chk)
        torch.cuda.synchronize()
        assert torch.equal(chk.reshape(-1), w_ntt.view(n, -1)[i]), i
    ct = _encrypt(s, params, sk, zp.encode(zp.periodic_slots(v, N), N, P))
    out = torch.empty(2 * nl * N, dtype=torch.int64, device="cuda")
    L.hc_mac_rotate(ctx, key, to_dev(ct), w_ntt, out)
    L.hc_ctx_device_status(ctx)
    dec = bfv.decrypt_at(params, sk, to_host(out).reshape(2, nl, N), list(range(N)))
    want = np.zeros(n, dtype=np.int64)
    want[:n_out] = (Wm.astype(object) @ v.astype(object)) % P
    assert np.array_equal(zp.decode(dec.astype(np.uint64), N, P), zp.periodic_slots(want, N))


def test_zp_encoding_argument_errors(L):
    N = 4096
    P = zp.plaintext_prime(N, 37)
    ctx_p = _plain_ctx(L, N, P)
    ctx2 = L.hc_ctx_create(N, CANONICAL_PRIMES[:2], P)
    buf = torch.zeros(N, dtype=torch.int64, device="cuda")
    with pytest.raises(L.HcError) as e:
        L.hc_zp_encode(ctx2, torch.zeros(2 * N, dtype=torch.int64, device="cuda"), buf)   # two moduli
    assert e.value.status == L.HC_ERR_INVALID_ARG
    with pytest.raises(L.HcError) as e:
        L.hc_zp_encode(ctx_p, buf, buf)                                                    # in place
    assert e.value.status == L.HC_ERR_INVALID_ARG
    with pytest.raises(L.HcError) as e:                                                   # too large for N/2
        L.hc_zp_matvec_preprocess(ctx2, ctx_p, np.zeros((N, 1), dtype=np.uint64), buf)
    assert e.value.status == L.HC_ERR_INVALID_ARG
    with pytest.raises(L.HcError) as e:                                                   # entry >= P
        L.hc_zp_matvec_preprocess(ctx2, ctx_p, np.full((2, 2), P, dtype=np.uint64),
                                  torch.zeros(2 * 2 * N, dtype=torch.int64, device="cuda"))
    assert e.value.status == L.HC_ERR_RANGE
    with pytest.raises(L.HcError) as e:                                                   # d_out too small
        L.hc_zp_matvec_preprocess(ctx2, ctx_p, np.zeros((4, 4), dtype=np.uint64), buf)
    assert e.value.status == L.HC_ERR_INVALID_ARG


@pytest.mark.parametrize("n", [1, 3])
def test_mac_rotate_many_equals_one_by_one(L, n):
    """m ciphertexts through the same n plaintexts in lockstep (hc_mac_rotate_many)
    give, ciphertext by ciphertext, the bits of hc_mac_rotate, and decrypt to the
    slot formula; m = 5 spans several products per plaintext and a batched key switch."""
    N, nl, m = 4096, 2, 5
    kp, P, s, sk, gk, params = _setup(N, nl, 17, 97 + n)
    ctx = L.hc_ctx_create(N, kp.moduli, P)
    key = L.hc_galois_key_create(ctx, kp.special, 5, gk)
    ms = [_slots(s, N, P) for _ in range(m)]
    ws = [_slots(s, N, P) for _ in range(n)]
    cts = np.stack([_encrypt(s, params, sk, zp.encode(x, N, P)) for x in ms])
    polys = np.stack([zp.encode(w, N, P) for w in ws])
    w_ntt = torch.empty(n * nl * N, dtype=torch.int64, device="cuda")
    L.hc_zp_plain_preprocess(ctx, P, polys, w_ntt)
    d_cts = to_dev(cts)
    out = torch.full((m * 2 * nl * N,), -1, dtype=torch.int64, device="cuda")
    L.hc_mac_rotate_many(ctx, key, d_cts, w_ntt, out)
    L.hc_ctx_device_status(ctx)
    got = to_host(out).reshape(m, 2, nl, N)
    one = torch.empty(2 * nl * N, dtype=torch.int64, device="cuda")
    for j in range(m):
        L.hc_mac_rotate(ctx, key, to_dev(cts[j]), w_ntt, one)
        torch.cuda.synchronize()
        assert np.array_equal(got[j], to_host(one).reshape(2, nl, N)), j
        dec = bfv.decrypt_at(params, sk, got[j], list(range(N)))
        assert np.array_equal(zp.decode(dec.astype(np.uint64), N, P), zp.slot_mac_rotate(ms[j], ws, P)), j
