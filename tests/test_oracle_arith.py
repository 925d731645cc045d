"""Pins of the oracle's scalar arithmetic, primes and psi against independent
computations (Python integers, sympy, trial division, enumeration)."""
import random

import pytest
import sympy

from oracle import core
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES


def test_mulmod_powmod_edges():
    rng = random.Random(11)
    qs = list(CANONICAL_PRIMES) + [17, 97, 193, (1 << 61) - 1, (1 << 62) - 57]
    for q in qs:
        vals = [0, 1, 2, q - 1, q - 2, q // 2] + [rng.randrange(q) for _ in range(40)]
        for a in vals:
            for b in vals[:10]:
                assert core.mulmod(a, b, q) == (a * b) % q
            e = rng.randrange(1 << 62)
            assert core.powmod(a, e, q) == pow(a, e, q)
        assert core.lib().or_addmod(q - 1, q - 1, q) == q - 2
        assert core.lib().or_submod(0, 1, q) == q - 1


def test_is_prime_vs_trial_division():
    def trial(n):
        if n < 2:
            return False
        d = 2
        while d * d <= n:
            if n % d == 0:
                return False
            d += 1
        return True

    for n in range(0, 20000):
        assert core.is_prime(n) == trial(n), n


def test_is_prime_strong_pseudoprimes_and_sympy():
    # strong pseudoprimes to the first few prime bases (textbook values)
    for n in [2047, 1373653, 25326001, 3215031751, 2152302898747, 3474749660383,
              341550071728321, 3825123056546413051, 561, 1105, 1729, 2465, 2821]:
        assert not core.is_prime(n)
    rng = random.Random(5)
    for _ in range(3000):
        n = rng.randrange(1 << 40, 1 << 63) | 1
        assert core.is_prime(n) == sympy.isprime(n), n
    for q in CANONICAL_PRIMES:
        assert core.is_prime(q)


def test_canonical_primes():
    qs = core.ntt_primes(50, 15, 6)
    assert tuple(qs) == CANONICAL_PRIMES
    step = 1 << 15
    top = ((1 << 50) - 1) // step * step + 1
    # every candidate from 2^50 down to the 6th prime is either listed or composite
    cand = top
    while cand >= qs[-1]:
        assert (cand in qs) == bool(sympy.isprime(cand)), cand
        cand -= step
    for q in qs:
        assert q < (1 << 50) and q % step == 1


def _brute_min_psi(q, N):
    return min(x for x in range(1, q) if pow(x, N, q) == q - 1)


@pytest.mark.parametrize("q,N", [(17, 4), (17, 8), (97, 16), (193, 32), (257, 64),
                                 (7681, 256), (12289, 1024), (40961, 2048), (65537, 4096)])
def test_min_psi_bruteforce(q, N):
    assert core.min_psi(q, N) == _brute_min_psi(q, N)


@pytest.mark.parametrize("N", [1024, 4096, 8192, 16384])
def test_min_psi_large(N):
    for q in CANONICAL_PRIMES[:4]:
        psi = core.min_psi(q, N)
        assert pow(psi, N, q) == q - 1 and pow(psi, 2 * N, q) == 1
        # the primitive 2N-th roots are exactly root^k for odd k: enumerate them
        # from a root found independently (a generator via sympy) and check
        # the minimum.
        g = sympy.primitive_root(q)
        w = pow(g, (q - 1) // (2 * N), q)
        w2 = w * w % q
        cur, best = w, w
        for _ in range(N):
            best = min(best, cur)
            cur = cur * w2 % q
        assert psi == best


def test_min_psi_rejects_bad_modulus():
    assert core.min_psi(97, 64) == 0   # 128 does not divide 96


def test_bitrev():
    for logn in range(1, 15):
        for k in [0, 1, 2, 3, (1 << logn) - 1, (1 << logn) // 3]:
            if k >= (1 << logn):
                continue
            s = format(k, "0%db" % logn)
            assert core.bitrev(k, logn) == int(s[::-1], 2)
