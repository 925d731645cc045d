"""Pins of the oracle's NTT / INTT (App. C.1) and negacyclic product (App. C,
Sec. 2.1) against a hand-worked example, Horner evaluation, closed forms,
invariants, an exact integer product and CRT reconstruction."""
import os
import random

import numpy as np
import pytest

from oracle import core
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, Stream

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            vals[k] = [int(x) for x in v]
    return vals


def _rev(k, logn):
    return int(format(k, "0%db" % logn)[::-1], 2) if logn else 0


def _horner(a, x, q):
    r = 0
    for c in reversed(list(a)):
        r = (r * x + int(c)) % q
    return r


def _negacyclic_int(a, b):
    """Exact integer product in Z[X]/(X^N+1) (Python ints)."""
    N = len(a)
    lin = [0] * (2 * N)
    for i in range(N):
        if a[i]:
            for j in range(N):
                lin[i + j] += int(a[i]) * int(b[j])
    return [lin[k] - lin[k + N] for k in range(N)]


def test_golden_n4_q17():
    g = _golden("ntt_n4_q17.txt")
    q, N, psi = g["q"][0], g["N"][0], g["psi"][0]
    assert core.min_psi(q, N) == psi
    assert list(core.ntt(g["a"], q, psi)) == g["ntt"]
    assert list(core.ntt(g["b"], q, psi)) == g["ntt_b"]
    assert list(core.negacyclic(g["a"], g["b"], q)) == g["ab"]
    assert list(core.intt(g["ntt"], q, psi)) == g["a"]


@pytest.mark.parametrize("N,q", [(8, 17), (16, 97), (32, 193), (64, 257), (128, 7681)])
def test_ntt_tiny_bruteforce(N, q):
    psi = core.min_psi(q, N)
    logn = N.bit_length() - 1
    rng = random.Random(N)
    a = [rng.randrange(q) for _ in range(N)]
    want = [_horner(a, pow(psi, 2 * _rev(k, logn) + 1, q), q) for k in range(N)]
    assert list(core.ntt(a, q, psi)) == want
    assert list(core.intt(want, q, psi)) == a


@pytest.mark.parametrize("N", [64, 256])
def test_ntt_closed_forms(N):
    q = CANONICAL_PRIMES[0]
    psi = core.min_psi(q, N)
    logn = N.bit_length() - 1
    delta = np.zeros(N, dtype=np.uint64)
    delta[0] = 1
    assert np.all(core.ntt(delta, q, psi) == 1)
    for k in [1, 2, 7, N - 1]:
        mono = np.zeros(N, dtype=np.uint64)
        mono[k] = 1
        want = [pow(psi, (2 * _rev(i, logn) + 1) * k, q) for i in range(N)]
        assert list(core.ntt(mono, q, psi)) == want


@pytest.mark.parametrize("N", [64, 512])
def test_ntt_inverse_and_linearity(N):
    s = Stream(3, N)
    for q in CANONICAL_PRIMES[:3]:
        psi = core.min_psi(q, N)
        a = s.below(q, N)
        b = s.below(q, N)
        A = core.ntt(a, q, psi)
        assert np.array_equal(core.intt(A, q, psi), a)
        assert np.array_equal(core.ntt(core.intt(a, q, psi), q, psi), a)
        apb = (a.astype(object) + b.astype(object)) % q
        lhs = core.ntt(np.array(apb, dtype=np.uint64), q, psi).astype(object)
        rhs = (A.astype(object) + core.ntt(b, q, psi).astype(object)) % q
        assert np.array_equal(lhs, rhs)
        # sampled output indices agree with the full transform
        ks = [0, 5, N - 1, N // 2]
        assert np.array_equal(core.ntt(a, q, psi, ks), A[ks])
        assert np.array_equal(core.intt(A, q, psi, ks), a[ks])


@pytest.mark.parametrize("N", [32, 128])
def test_convolution_theorem(N):
    """INTT(NTT(a) . NTT(b)) equals the schoolbook negacyclic product."""
    s = Stream(4, N)
    for q in CANONICAL_PRIMES[:2]:
        psi = core.min_psi(q, N)
        a, b = s.below(q, N), s.below(q, N)
        A, B = core.ntt(a, q, psi), core.ntt(b, q, psi)
        C = np.array([(int(x) * int(y)) % q for x, y in zip(A, B)], dtype=np.uint64)
        assert np.array_equal(core.intt(C, q, psi), core.negacyclic(a, b, q))


def test_negacyclic_monomials():
    N, q = 64, CANONICAL_PRIMES[1]
    for a_exp, b_exp in [(0, 0), (3, 5), (40, 30), (63, 63), (63, 1), (32, 32)]:
        a = np.zeros(N, dtype=np.uint64)
        b = np.zeros(N, dtype=np.uint64)
        a[a_exp] = 1
        b[b_exp] = 1
        c = core.negacyclic(a, b, q)
        want = np.zeros(N, dtype=np.uint64)
        e = a_exp + b_exp
        want[e % N] = 1 if e < N else q - 1
        assert np.array_equal(c, want)


@pytest.mark.parametrize("N", [16, 64, 128])
def test_negacyclic_vs_exact_integer_product(N):
    rng = random.Random(N)
    for q in CANONICAL_PRIMES[:3]:
        a = [rng.randrange(q) for _ in range(N)]
        b = [rng.randrange(q) for _ in range(N)]
        want = [x % q for x in _negacyclic_int(a, b)]
        assert list(core.negacyclic(a, b, q)) == want
        assert list(core.negacyclic(b, a, q)) == want
        ks = [0, N - 1, N // 3]
        assert list(core.negacyclic(a, b, q, ks)) == [want[k] for k in ks]


def test_crt_consistency_across_limbs():
    """Small-integer polys: per-limb residues CRT back to the exact integer product."""
    N, L = 64, 3
    moduli = CANONICAL_PRIMES[:L]
    Q = 1
    for q in moduli:
        Q *= q
    rng = random.Random(9)
    a = [rng.randrange(-(1 << 40), 1 << 40) for _ in range(N)]
    b = [rng.randrange(-(1 << 40), 1 << 40) for _ in range(N)]
    exact = _negacyclic_int(a, b)
    res = []
    for q in moduli:
        aq = np.array([x % q for x in a], dtype=np.uint64)
        bq = np.array([x % q for x in b], dtype=np.uint64)
        res.append(core.negacyclic(aq, bq, q))
    for k in range(N):
        x = 0
        for li, q in enumerate(moduli):
            Qi = Q // q
            x += int(res[li][k]) * Qi * pow(Qi, -1, q)
        x %= Q
        if x > Q // 2:
            x -= Q
        assert x == exact[k]


def test_sparse_and_batch_agree_with_dense():
    N = 128
    moduli = CANONICAL_PRIMES[:2]
    s = Stream(8, 0)
    a = np.stack([s.below(q, N) for q in moduli])
    w = s.int8(N).astype(np.int64)
    w[::3] = 0
    sparse = core.sparse_of(w)
    for li, q in enumerate(moduli):
        dense = core.negacyclic(a[li], core.lift_small(w, q), q)
        assert np.array_equal(core.negacyclic_sparse(a[li], sparse, N, q), dense)
        ks = [1, 77, 127]
        assert np.array_equal(core.negacyclic_sparse(a[li], sparse, N, q, ks), dense[ks])
    b = np.stack([core.lift_small(w, q) for q in moduli])
    batch = core.negacyclic_batch(a[None], b[None], moduli)[0]
    for li, q in enumerate(moduli):
        assert np.array_equal(batch[li], core.negacyclic(a[li], b[li], q))


def test_ternary_agrees_with_dense():
    N = 256
    s = Stream(12, 0)
    for q in CANONICAL_PRIMES[:2]:
        a = s.below(q, N)
        t = s.ternary(N)
        dense = core.negacyclic(a, core.lift_small(t, q), q)
        assert np.array_equal(core.negacyclic_ternary(a, core.ternary_of(t), N, q), dense)
        ks = [0, 3, 255]
        assert np.array_equal(core.negacyclic_ternary(a, core.ternary_of(t), N, q, ks), dense[ks])
