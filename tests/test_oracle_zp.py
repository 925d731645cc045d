"""Pins of the oracle's Z_P SIMD layer (oracle/zp.py): slot encoding, Galois
automorphisms, key-switched slot rotations and the HELiKs-style
multiply-accumulate-rotate iteration used by SecONNds-P's linear layers
(Sec. 6.1, Sec. 2.3, Sec. 2.1).  Pins come from the algebra: slot products are
the ring product, sigma_5 rotates the slot rows, automorphisms compose and
multiply, rotated ciphertexts decrypt to rotated slot vectors with small
noise, the rounding division by the special prime is exact on multiples, and
the iteration decrypts to the slot-wise formula."""
import numpy as np
import pytest

from oracle import bfv, core, zp
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, Stream

N = 4096
L = 2
P = zp.plaintext_prime(N, 17)
KP = zp.KsParams(N, tuple(CANONICAL_PRIMES[:L]), CANONICAL_PRIMES[L])


def _slots(s):
    return s.below(P, N).astype(np.int64).reshape(2, N // 2)


def test_plaintext_prime():
    assert core.is_prime(P) and P % (2 * N) == 1 and P < (1 << 17)
    P37 = zp.plaintext_prime(8192, 37)
    assert core.is_prime(P37) and P37 % 16384 == 1 and (1 << 36) < P37 < (1 << 37)


def test_slot_exponents_cover_the_odd_residues():
    e = zp.slot_exponents(N)
    assert sorted(e.reshape(-1).tolist()) == list(range(1, 2 * N, 2))
    assert sorted(zp.slot_index(N).reshape(-1).tolist()) == list(range(N))


def test_encode_decode_roundtrip_and_slotwise_products():
    s = Stream(71, 0)
    m1, m2 = _slots(s), _slots(s)
    p1, p2 = zp.encode(m1, N, P), zp.encode(m2, N, P)
    assert np.array_equal(zp.decode(p1, N, P), m1)
    prod = core.negacyclic(p1, p2, P)                       # ring product mod (X^N + 1, P)
    assert np.array_equal(zp.decode(prod, N, P), (m1 * m2) % P)
    # the constant polynomial 1 has every slot equal to 1
    one = np.zeros(N, dtype=np.uint64)
    one[0] = 1
    assert np.all(zp.decode(one, N, P) == 1)


def test_automorphism_closed_form_and_homomorphism():
    q = KP.moduli[0]
    s = Stream(72, 0)
    for i in (0, 1, 5, N // 2 + 3, N - 1):
        for g in (5, 3, 2 * N - 1):
            x = np.zeros(N, dtype=np.uint64)
            x[i] = 1
            y = zp.automorphism(x, g, q)
            j = i * g % (2 * N)
            want = np.zeros(N, dtype=np.uint64)
            want[j % N] = 1 if j < N else q - 1              # X^(ig) with X^N = -1
            assert np.array_equal(y, want), (i, g)
    a, b = s.below(q, N), s.below(q, N)
    g, h = 5, 25
    assert np.array_equal(zp.automorphism(zp.automorphism(a, g, q), h, q), zp.automorphism(a, g * h % (2 * N), q))
    assert np.array_equal(zp.automorphism(core.negacyclic(a, b, q), g, q),
                          core.negacyclic(zp.automorphism(a, g, q), zp.automorphism(b, g, q), q))


def test_sigma5_rotates_both_slot_rows_left():
    m = _slots(Stream(73, 0))
    p = zp.encode(m, N, P)
    assert np.array_equal(zp.decode(zp.automorphism(p, 5, P), N, P), np.roll(m, -1, axis=1))
    g_inv = pow(5, -1, 2 * N)
    assert np.array_equal(zp.decode(zp.automorphism(p, g_inv, P), N, P), np.roll(m, 1, axis=1))


def test_mod_down_divides_multiples_exactly():
    s = Stream(74, 0)
    x = [int(v) for v in s.below(1 << 62, 16)]                 # quotients
    r = [int(v) - (1 << 40) for v in s.below(1 << 41, 16)]     # |r| < p_sp / 2
    qp = KP.qp
    Qp = KP.Q * KP.special
    u = np.zeros((L + 1, N), dtype=np.uint64)
    for k in range(16):
        val = (KP.special * x[k] + r[k]) % Qp
        for i, q in enumerate(qp):
            u[i, k] = val % q
    v = zp.mod_down(u, KP)
    for k in range(16):
        for i, q in enumerate(KP.moduli):
            assert int(v[i, k]) == x[k] % q


def _keys(seed, g=5):
    s = Stream(seed, 0)
    sk = s.ternary(N)
    a = np.stack([np.stack([s.below(q, N) for q in KP.qp]) for _ in range(L)])
    e = np.stack([s.rounded_gaussian(N) for _ in range(L)])
    return s, sk, zp.galois_key(KP, sk, g, a, e)


def _encrypt(s, params, sk, poly):
    a = np.stack([s.below(q, N) for q in params.moduli])
    return bfv.encrypt(params, sk, poly, a, s.rounded_gaussian(N))


def test_rotation_decrypts_to_rotated_slots_with_small_noise():
    s, sk, gk = _keys(75)
    params = zp.bfv_params(N, KP.moduli, P)
    m = _slots(s)
    ct = _encrypt(s, params, sk, zp.encode(m, N, P))
    rot = zp.rotate(ct, gk, 5, KP)
    ks = list(range(N))
    got = bfv.decrypt_at(params, sk, rot, ks)
    assert np.array_equal(zp.decode(got.astype(np.uint64), N, P), np.roll(m, -1, axis=1))
    noise = bfv.noise_at(params, sk, rot, ks[:64], zp.encode(np.roll(m, -1, axis=1), N, P)[:64])
    assert max(abs(v) for v in noise) < (1 << 40)              # Delta is about 2^83
    # a wrong key (another secret) does not rotate
    _, sk2, gk2 = _keys(76)
    bad = bfv.decrypt_at(params, sk, zp.rotate(ct, gk2, 5, KP), ks[:64])
    assert not np.array_equal(bad, got[:64])


def test_mac_rotate_decrypts_to_the_slot_formula():
    s, sk, gk = _keys(77)
    params = zp.bfv_params(N, KP.moduli, P)
    m = _slots(s)
    ws = [_slots(s) for _ in range(3)]
    ct = _encrypt(s, params, sk, zp.encode(m, N, P))
    lifts = [zp.lift_plain(zp.encode(w, N, P), P, KP.moduli) for w in ws]
    out = zp.mac_rotate(ct, lifts, gk, 5, KP)
    got = bfv.decrypt_at(params, sk, out, list(range(N)))
    assert np.array_equal(zp.decode(got.astype(np.uint64), N, P), zp.slot_mac_rotate(m, ws, P))


@pytest.mark.parametrize("n_out, n_in", [(1, 1), (3, 5), (8, 8), (16, 11), (64, 64)])
def test_matvec_diagonals_give_the_matrix_product(n_out, n_in):
    """The diagonal method on slot vectors (no encryption): sum_i rot^i(vtilde * w_i)
    equals W v mod P at every slot, held periodically, for square, rectangular and
    degenerate (1 x 1) matrices; checked against a plain integer matrix product."""
    s = Stream(76, n_out * 100 + n_in)
    Wm = s.below(P, n_out * n_in).astype(np.int64).reshape(n_out, n_in)
    v = s.below(P, n_in).astype(np.int64)
    n = zp.matvec_size(n_out, n_in)
    vp = np.zeros(n, dtype=np.int64)
    vp[:n_in] = v
    ws = zp.matvec_diagonals(Wm, N, P)
    assert ws.shape == (n, 2, N // 2)
    got = zp.slot_mac_rotate(zp.periodic_slots(vp, N), list(ws), P)
    want = np.zeros(n, dtype=object)
    for j in range(n_out):                                   # plain matrix product, big integers
        want[j] = sum(int(Wm[j, k]) * int(v[k]) for k in range(n_in)) % P
    assert np.array_equal(got, zp.periodic_slots(want.astype(np.int64), N))


def test_matvec_through_encryption():
    """The same product through BFV: encode the periodic input, encrypt, run the
    oracle's multiply-accumulate-rotate with the encoded diagonals, decrypt, decode."""
    n = 4
    s = Stream(77, 0)
    Wm = s.below(P, n * n).astype(np.int64).reshape(n, n)
    v = s.below(P, n).astype(np.int64)
    s2, sk, gk = _keys(78)
    params = zp.bfv_params(N, KP.moduli, P)
    ct = _encrypt(s2, params, sk, zp.encode(zp.periodic_slots(v, N), N, P))
    lifts = [zp.lift_plain(zp.encode(w, N, P), P, KP.moduli) for w in zp.matvec_diagonals(Wm, N, P)]
    out = zp.mac_rotate(ct, lifts, gk, 5, KP)
    dec = bfv.decrypt_at(params, sk, out, list(range(N)))
    want = (Wm.astype(object) @ v.astype(object)) % P
    assert np.array_equal(zp.decode(dec.astype(np.uint64), N, P), zp.periodic_slots(want.astype(np.int64), N))
