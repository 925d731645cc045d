"""BFV secret-key encryption and decryption over RNS limbs.  TEST INFRASTRUCTURE ONLY.

Client-side harness (Sec. 6.3: the GPU server never touches the secret key).
Follows the RLWE ciphertext of App. C: ct = (a, b) with b = a*sk + delta*m +
eps*e, sk uniform ternary, e a small zero-mean discrete Gaussian of standard
deviation sigma.  Readings where the paper is silent: delta = floor(Q/t),
eps = 1, sigma = 3.2 (rounded Gaussian, truncated at 6 sigma -- the sampling
happens in the input generator, this module only receives e), and the SEAL
sign convention ct = (c0, c1) = (-a*sk + delta*m + e, a), so that
c0 + c1*sk = delta*m + e (mod Q) and

    m = round(t * [c0 + c1*sk]_Q / Q)  mod t.

Q = prod q_i is odd and t = 2^37 is a power of two, so t*x/Q is never a
half-integer for x != 0: rounding has no ties.  CRT and rounding use exact
Python integers; the products c1*sk and a*sk use the oracle's ternary
schoolbook (sk has coefficients in {-1, 0, 1}).

Parity: pinned by decrypt(encrypt(m)) == m, by the additive and
plaintext-multiplicative homomorphisms against plain integer arithmetic, and
end to end by the convolution test (tests/test_oracle_bfv.py,
tests/test_oracle_conv.py).
"""
from dataclasses import dataclass

import numpy as np

from . import core


@dataclass
class Params:
    N: int
    moduli: tuple
    t: int

    @property
    def Q(self):
        r = 1
        for q in self.moduli:
            r *= q
        return r

    @property
    def delta(self):
        return self.Q // self.t


def _centered_to_residue(v, q):
    return core.lift_small(v, q)


def encrypt(params: Params, sk, m, a, e):
    """m: [N] ints in [0, t); a: [L][N] uniform residues; e: [N] small ints.
    Returns ct [2][L][N] uint64 = (c0, c1) with c0 = -a*sk + delta*m + e, c1 = a."""
    N, L = params.N, len(params.moduli)
    tern_sk = core.ternary_of(sk)
    m_obj = np.asarray(m, dtype=np.int64).astype(object)
    e = np.asarray(e, dtype=np.int64)
    ct = np.zeros((2, L, N), dtype=np.uint64)
    for li, q in enumerate(params.moduli):
        a_l = np.ascontiguousarray(a[li], dtype=np.uint64)
        as_ = core.negacyclic_ternary(a_l, tern_sk, N, q).astype(object)
        d = params.delta % q
        c0 = (-as_ + d * m_obj + e.astype(object)) % q
        ct[0, li] = c0.astype(np.uint64)
        ct[1, li] = a_l
    return ct


def crt(residues, moduli):
    """residues: [L][n] -> list of n Python ints in [0, Q)."""
    Q = 1
    for q in moduli:
        Q *= q
    coef = []
    for q in moduli:
        Qi = Q // q
        coef.append(Qi * pow(Qi, -1, q))
    n = len(residues[0])
    out = []
    for k in range(n):
        x = 0
        for li in range(len(moduli)):
            x += int(residues[li][k]) * coef[li]
        out.append(x % Q)
    return out


def phase_at(params: Params, sk, ct, ks):
    """[c0 + c1*sk]_Q at coefficient indices ks, as Python ints in [0, Q)."""
    tern_sk = core.ternary_of(sk)
    res = []
    for li, q in enumerate(params.moduli):
        c1s = core.negacyclic_ternary(ct[1, li], tern_sk, params.N, q, ks)
        c0 = np.asarray(ct[0, li])[np.asarray(ks, dtype=np.int64)]
        res.append((c0.astype(object) + c1s.astype(object)) % q)
    return crt(res, params.moduli)


def decrypt_at(params: Params, sk, ct, ks):
    """Decrypted plaintext coefficients (ints in [0, t)) at indices ks."""
    Q, t = params.Q, params.t
    out = []
    for x in phase_at(params, sk, ct, ks):
        out.append(((2 * t * x + Q) // (2 * Q)) % t)
    return np.array(out, dtype=np.int64)


def noise_at(params: Params, sk, ct, ks, m_expected):
    """Signed noise v = [c0 + c1*sk - delta*m]_Q (centered) at ks, for the budget check."""
    Q = params.Q
    out = []
    for x, m in zip(phase_at(params, sk, ct, ks), m_expected):
        v = (x - params.delta * int(m)) % Q
        if v > Q // 2:
            v -= Q
        out.append(v)
    return out
