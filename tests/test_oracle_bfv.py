"""Pins of the oracle's BFV encryption / decryption (App. C): round trip,
homomorphic addition and plaintext multiplication against exact integer
arithmetic, and the noise budget."""
import numpy as np
import pytest

from oracle import bfv, core
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream


def _negacyclic_int(a, b):
    N = len(a)
    lin = [0] * (2 * N)
    for i in range(N):
        ai = int(a[i])
        if ai:
            for j in range(N):
                bj = int(b[j])
                if bj:
                    lin[i + j] += ai * bj
    return [lin[k] - lin[k + N] for k in range(N)]


def _setup(N, L, seed):
    params = bfv.Params(N, CANONICAL_PRIMES[:L], T_PLAIN)
    s = Stream(seed, 0)
    sk = s.ternary(N)
    return params, s, sk


def _enc(params, s, sk, m):
    a = np.stack([s.below(q, params.N) for q in params.moduli])
    e = s.rounded_gaussian(params.N)
    return bfv.encrypt(params, sk, m, a, e)


@pytest.mark.parametrize("N,L", [(64, 2), (256, 3), (1024, 4)])
def test_roundtrip(N, L):
    params, s, sk = _setup(N, L, 21)
    m = s.below(T_PLAIN, N).astype(np.int64)
    ct = _enc(params, s, sk, m)
    ks = list(range(N))
    assert np.array_equal(bfv.decrypt_at(params, sk, ct, ks), m)
    noise = bfv.noise_at(params, sk, ct, ks, m)
    assert max(abs(v) for v in noise) <= 19   # |e| <= 6 sigma


def test_sign_convention_and_components():
    params, s, sk = _setup(64, 2, 3)
    m = s.below(T_PLAIN, 64).astype(np.int64)
    a = np.stack([s.below(q, 64) for q in params.moduli])
    e = np.zeros(64, dtype=np.int64)
    ct = bfv.encrypt(params, sk, m, a, e)
    assert np.array_equal(ct[1], a)
    # c0 + c1*sk = delta*m exactly when e = 0
    for li, q in enumerate(params.moduli):
        c1s = core.negacyclic(ct[1, li], core.lift_small(sk, q), q)
        lhs = (ct[0, li].astype(object) + c1s.astype(object)) % q
        rhs = (params.delta % q) * m.astype(object) % q
        assert np.array_equal(lhs, rhs)


def test_homomorphic_add_and_plain_mult():
    N, L = 128, 3
    params, s, sk = _setup(N, L, 8)
    m1 = s.below(T_PLAIN, N).astype(np.int64)
    m2 = s.below(T_PLAIN, N).astype(np.int64)
    c1, c2 = _enc(params, s, sk, m1), _enc(params, s, sk, m2)
    csum = np.zeros_like(c1)
    for li, q in enumerate(params.moduli):
        csum[:, li] = (c1[:, li].astype(object) + c2[:, li].astype(object)) % q
    ks = list(range(N))
    assert np.array_equal(bfv.decrypt_at(params, sk, csum, ks), (m1 + m2) % T_PLAIN)
    # multiply by a small plaintext polynomial w (int8 coefficients)
    w = s.int8(N).astype(np.int64)
    cw = np.zeros_like(c1)
    for li, q in enumerate(params.moduli):
        wq = core.lift_small(w, q)
        for comp in range(2):
            cw[comp, li] = core.negacyclic(c1[comp, li], wq, q)
    want = np.array([x % T_PLAIN for x in _negacyclic_int(m1, w)], dtype=np.int64)
    assert np.array_equal(bfv.decrypt_at(params, sk, cw, ks), want)


def test_crt_helper():
    moduli = CANONICAL_PRIMES[:3]
    Q = moduli[0] * moduli[1] * moduli[2]
    xs = [0, 1, Q - 1, Q // 2, 123456789123456789123456789]
    res = [[x % q for x in xs] for q in moduli]
    assert bfv.crt(res, moduli) == [x % Q for x in xs]
