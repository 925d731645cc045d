"""BFV over Z_P with SIMD slots, slot rotations by key switching, and the
iterated multiply-accumulate-rotate of HELiKs-style linear layers.
TEST INFRASTRUCTURE ONLY.

SecONNds-P runs its linear layers with HELiKs' kernels over the plaintext space
Z_P^N, P a prime (Sec. 6.1; Sec. 2.3): an iterative algorithm in which each
iteration multiplies the input ciphertext by an NTT-preprocessed weight
plaintext, accumulates the product into the previous iteration's result, and
rotates the accumulator by one slot (Sec. 6.1; the 1-step rotations and NTT
preprocessing of Sec. 2.3).  Rotations are Galois automorphisms followed by
key switching (Sec. 2.1: rotations need a key-switching step with public
evaluation keys; App. C).  The paper prints none of the formulas; this module
holds the textbook reading the build uses:

SIMD slots.  P = 1 mod 2N; zeta the minimal primitive 2N-th root mod P.  Slot
(r, c), r in {0, 1}, c < N/2, holds p(zeta^e) with e = 5^c mod 2N for r = 0
and e = -5^c mod 2N for r = 1.  With core.ntt's order (slot k holds
p(psi^(2 rev(k) + 1))) slot (r, c) is NTT index rev((e - 1) / 2).

Galois automorphism.  sigma_g(p)(X) = p(X^g) for odd g: coefficient i moves
to i*g mod 2N, negated when that lands in [N, 2N).  sigma_5 rotates both slot
rows left by one: slot (r, c) of sigma_5(p) holds slot (r, c + 1) of p.

Key switching (one special prime p_sp, one digit per ciphertext limb).  The
Galois key for g is, for every digit j < L, an RLWE pair over Q*p_sp
    k_j = (b_j, a_j),  b_j = -a_j s + e_j + p_sp * Qh_j * [Qh_j^-1]_{q_j} * sigma_g(s),
with Qh_j = Q / q_j.  A ciphertext (c0, c1) under s rotates to
    d = sigma_g(c1);  D_j = d mod q_j (integers in [0, q_j));
    (u0, u1) = sum_j D_j * k_j  over Q*p_sp;
    v = (u - [u]_{p_sp}) / p_sp over Q, [.] the centered residue (rounding);
    out = (sigma_g(c0) + v0, v1),
which decrypts to sigma_g(m) up to small noise: u0 + u1 s = sum_j D_j e_j +
p_sp * (d + Q k) * sigma_g(s) for an integer polynomial k, and p_sp Q = 0 mod
Q p_sp.

Multiply-accumulate-rotate.  For ciphertext x and NTT-preprocessed weights
w_0 .. w_{n-1}: acc = x * w_{n-1}; for i = n-2 .. 0: acc = rot(acc) + x * w_i.
The result decrypts to sum_i rot^i(m * w_i) slot-wise mod P.

Matrix-vector products with it (the diagonal method).  A vector v of length
n, n a power of two dividing N/2, is held periodically: slot (r, t) holds
v[t mod n] in both rows r.  For an n x n matrix W put
    w_i[r][t] = W[(t - i) mod n][t mod n],   i < n;
then sum_i rot^i(vtilde * w_i) at slot (r, j) is sum_i W[j][(j + i) mod n]
v[(j + i) mod n] = (W v)[j mod n]: the product, held periodically again, so
the output has the input's format.  A rectangular matrix is padded with zero
rows and columns to the next such n.

Parity: pinned by SIMD encode/decode round trips and slot-wise products, the
automorphism's closed form on monomials and its action on slots, decryption of
rotated ciphertexts to rotated slot vectors, the key-switching noise bound,
and the iteration against the plain slot-wise formula
(tests/test_oracle_zp.py).
"""
from dataclasses import dataclass

import numpy as np

from . import bfv, core


# ---- plaintext prime and SIMD slots ------------------------------------------------

def plaintext_prime(N, bits=37):
    """The largest prime below 2^bits that is 1 mod 2N."""
    return core.ntt_primes(bits, (2 * N).bit_length() - 1, 1)[0]


def slot_exponents(N):
    """[2][N/2] odd exponents e: slot (r, c) is the evaluation at zeta^e."""
    half = N // 2
    e = np.zeros((2, half), dtype=np.int64)
    g = 1
    for c in range(half):
        e[0, c] = g
        e[1, c] = (2 * N - g) % (2 * N)
        g = g * 5 % (2 * N)
    return e


def slot_index(N):
    """[2][N/2] NTT indices (core.ntt order) of the slots."""
    logn = N.bit_length() - 1
    e = slot_exponents(N)
    return np.vectorize(lambda x: core.bitrev((int(x) - 1) // 2, logn))(e).astype(np.int64)


def encode(m, N, P):
    """Slot values m [2][N/2] in [0, P) -> plaintext polynomial [N] with those slots."""
    zeta = core.min_psi(P, N)
    A = np.zeros(N, dtype=np.uint64)
    A[slot_index(N).reshape(-1)] = np.asarray(m, dtype=np.uint64).reshape(-1)
    return core.intt(A, P, zeta)


def decode(p, N, P):
    """Plaintext polynomial [N] in [0, P) -> slot values [2][N/2]."""
    zeta = core.min_psi(P, N)
    A = core.ntt(np.asarray(p, dtype=np.uint64), P, zeta)
    return A[slot_index(N)]


# ---- automorphism -------------------------------------------------------------------

def automorphism(a, g, q):
    """sigma_g(a)(X) = a(X^g) mod (X^N + 1, q), a [N] residues in [0, q)."""
    a = np.asarray(a, dtype=np.uint64)
    N = a.size
    out = np.zeros(N, dtype=np.uint64)
    for i in range(N):
        j = i * g % (2 * N)
        v = int(a[i])
        if j < N:
            out[j] = v
        else:
            out[j - N] = (q - v) % q
    return out


def automorphism_small(s, g):
    """sigma_g of a polynomial with small signed integer coefficients."""
    s = np.asarray(s, dtype=np.int64)
    N = s.size
    out = np.zeros(N, dtype=np.int64)
    for i in range(N):
        j = i * g % (2 * N)
        if j < N:
            out[j] = s[i]
        else:
            out[j - N] = -s[i]
    return out


# ---- Galois keys and key switching ------------------------------------------------------

@dataclass
class KsParams:
    N: int
    moduli: tuple      # q_0 .. q_{L-1}
    special: int       # p_sp

    @property
    def L(self):
        return len(self.moduli)

    @property
    def qp(self):
        return tuple(self.moduli) + (self.special,)

    @property
    def Q(self):
        r = 1
        for q in self.moduli:
            r *= q
        return r


def galois_key(kp: KsParams, sk, g, a, e):
    """[L][2][L+1][N] uint64: digit j's pair (b_j, a_j) over Q*p_sp.
    a: [L][L+1][N] uniform residues; e: [L][N] small noise."""
    N, L = kp.N, kp.L
    tern = core.ternary_of(sk)
    s_g = automorphism_small(sk, g)
    Q = kp.Q
    out = np.zeros((L, 2, L + 1, N), dtype=np.uint64)
    for j in range(L):
        qj = kp.moduli[j]
        Qh = Q // qj
        scal = kp.special * Qh * pow(Qh % qj, -1, qj)
        for i, q in enumerate(kp.qp):
            a_ji = np.ascontiguousarray(a[j][i], dtype=np.uint64)
            as_ = core.negacyclic_ternary(a_ji, tern, N, q).astype(object)
            sg = core.lift_small(s_g, q).astype(object)
            ej = core.lift_small(e[j], q).astype(object)
            b = (-as_ + ej + (scal % q) * sg) % q
            out[j, 0, i] = b.astype(np.uint64)
            out[j, 1, i] = a_ji
    return out


def mod_down(u, kp: KsParams):
    """[L+1][N] residues over Q*p_sp -> [L][N]: (u - [u]_{p_sp}) / p_sp mod q_i with the
    centered residue [u]_{p_sp} in (-p_sp/2, p_sp/2]."""
    p = kp.special
    usp = u[kp.L].astype(object)
    cen = np.where(usp > (p - 1) // 2, usp - p, usp)
    out = np.zeros((kp.L, kp.N), dtype=np.uint64)
    for i, q in enumerate(kp.moduli):
        pinv = pow(p % q, -1, q)
        out[i] = (((u[i].astype(object) - cen) % q) * pinv % q).astype(np.uint64)
    return out


def rotate(ct, gk, g, kp: KsParams):
    """Ciphertext [2][L][N] (coefficient domain) -> sigma_g applied and switched back to s."""
    N, L = kp.N, kp.L
    r0 = np.stack([automorphism(ct[0, i], g, q) for i, q in enumerate(kp.moduli)])
    d = np.stack([automorphism(ct[1, i], g, q) for i, q in enumerate(kp.moduli)])
    u = np.zeros((2, L + 1, N), dtype=object)
    for j in range(L):
        Dj = d[j].astype(object)                   # integers in [0, q_j)
        for i, q in enumerate(kp.qp):
            Dji = (Dj % q).astype(np.uint64)
            for comp in range(2):
                u[comp, i] += core.negacyclic(Dji, gk[j, comp, i], q).astype(object)
    for i, q in enumerate(kp.qp):
        u[:, i] %= q
    v0, v1 = mod_down(u[0], kp), mod_down(u[1], kp)
    out = np.zeros((2, L, N), dtype=np.uint64)
    for i, q in enumerate(kp.moduli):
        out[0, i] = ((r0[i].astype(object) + v0[i].astype(object)) % q).astype(np.uint64)
        out[1, i] = v1[i]
    return out


# ---- plaintext multiply and the multiply-accumulate-rotate iteration ---------------------

def lift_plain(p, P, moduli):
    """Plaintext polynomial [N] in [0, P) -> [L][N] centered lift mod every q_i."""
    p = np.asarray(p, dtype=np.int64)
    cen = np.where(p > (P - 1) // 2, p - P, p)
    return np.stack([core.lift_small(cen, q) for q in moduli])


def mul_plain(ct, w_lift, moduli):
    """(c0 * w, c1 * w) over R_Q for a lifted plaintext w [L][N]."""
    out = np.zeros_like(ct)
    for comp in range(2):
        for i, q in enumerate(moduli):
            out[comp, i] = core.negacyclic(ct[comp, i], w_lift[i], q)
    return out


def add(a, b, moduli):
    out = np.zeros_like(a)
    for i, q in enumerate(moduli):
        out[:, i] = ((a[:, i].astype(object) + b[:, i].astype(object)) % q).astype(np.uint64)
    return out


def mac_rotate(ct, w_lifts, gk, g, kp: KsParams):
    """acc = ct * w_{n-1}; for i = n-2 .. 0: acc = rot(acc) + ct * w_i."""
    n = len(w_lifts)
    acc = mul_plain(ct, w_lifts[n - 1], kp.moduli)
    for i in range(n - 2, -1, -1):
        acc = add(rotate(acc, gk, g, kp), mul_plain(ct, w_lifts[i], kp.moduli), kp.moduli)
    return acc


def slot_mac_rotate(m, ws, P):
    """The plain counterpart on slot vectors [2][N/2]: sum_i rot^i(m * w_i) mod P, rot =
    left rotation of both rows by one."""
    m = np.asarray(m, dtype=object)
    acc = np.zeros_like(m)
    for i, w in enumerate(ws):
        acc = (acc + np.roll((m * np.asarray(w, dtype=object)) % P, -i, axis=1)) % P
    return acc.astype(np.int64)


def periodic_slots(v, N):
    """Vector v of length n (a power of two dividing N/2) -> slots [2][N/2], slot (r, t) = v[t mod n]."""
    v = np.asarray(v, dtype=np.int64)
    n = v.size
    assert n >= 1 and (N // 2) % n == 0 and n & (n - 1) == 0
    return np.tile(v, (2, (N // 2) // n))


def matvec_size(n_out, n_in):
    """The padded size n: the smallest power of two >= max(n_out, n_in)."""
    n = 1
    while n < max(n_out, n_in):
        n *= 2
    return n


def matvec_diagonals(Wm, N, P):
    """n x n (after padding) weight slot vectors [n][2][N/2] of the diagonal method for the
    integer matrix Wm [n_out][n_in], residues mod P: w_i[r][t] = W[(t - i) mod n][t mod n]."""
    Wm = np.asarray(Wm, dtype=np.int64)
    n_out, n_in = Wm.shape
    n = matvec_size(n_out, n_in)
    assert (N // 2) % n == 0
    Wp = np.zeros((n, n), dtype=np.int64)
    Wp[:n_out, :n_in] = Wm % P
    t = np.arange(N // 2)
    out = np.zeros((n, 2, N // 2), dtype=np.int64)
    for i in range(n):
        row = Wp[(t - i) % n, t % n]
        out[i, 0] = row
        out[i, 1] = row
    return out


def bfv_params(N, moduli, P):
    return bfv.Params(N, tuple(moduli), P)


# ---- convolution layers over Z_P ----------------------------------------------------------
#
# Reading (SecONNds-P runs its convolutions with HELiKs' kernels over Z_P^N, Sec. 6.1 and
# Sec. 2.3; the paper cites those kernels and prints none of their packings).  A stride-1
# convolution of C input channels of H x W (zero padding p, kernel kh x kw) into M output
# channels, as the multiply-accumulate-rotate iteration:
#   * input channel c is one ciphertext whose two slot rows both hold the zero-padded image,
#     Hp = H + 2p rows of Wp = W + 2p slots, row-major from slot 0 (Hp*Wp <= N/2, zeros
#     after it);
#   * output ciphertext y holds output channel 2y + r in slot row r, output pixel (i, j) at
#     slot i*Wp + j (i < Ho = Hp - kh + 1, j < Wo = Wp - kw + 1; other slots unspecified);
#   * kernel offset i = l*kw + l' shifts by delta_i = l*Wp + l'; the weight plaintext
#     w_{y,i,c} holds the constant K[2y + r][c][l][l'] in slot row r (0 past M);
#   * each iteration's product is the sum over the input channels,
#         P_i = sum_c x_c * w_{y,i,c};  acc = P_{n-1};  acc = rot^(delta_{i+1} - delta_i)(acc) + P_i,
#     which leaves sum_i rot^(delta_i)(P_i), whose slot (r, i*Wp + j) is
#         sum_{c,l,l'} K[2y+r][c][l][l'] * x_pad[c][i + l][j + l'] = conv(x, K)[2y + r][i][j] mod P;
#   * a rotation by s slots is sigma_g with g = 5^s mod 2N; the steps are 1 (within a
#     kernel row) and Wp - kw + 1 (to the next kernel row), so two Galois keys serve a
#     layer; an output slot reads slots up to Hp*Wp - 1 < N/2, so no row wraps around.

@dataclass
class ConvShape:
    C: int
    H: int
    W: int
    M: int
    kh: int
    kw: int
    pad: int
    N: int

    @property
    def Hp(self):
        return self.H + 2 * self.pad

    @property
    def Wp(self):
        return self.W + 2 * self.pad

    @property
    def Ho(self):
        return self.Hp - self.kh + 1

    @property
    def Wo(self):
        return self.Wp - self.kw + 1

    @property
    def Y(self):
        """Output ciphertexts: two output channels each."""
        return (self.M + 1) // 2

    @property
    def offsets(self):
        """delta_i = l*Wp + l' for kernel offset i = l*kw + l'."""
        return [l * self.Wp + m for l in range(self.kh) for m in range(self.kw)]

    @property
    def steps(self):
        """Rotation before adding P_i, i < n - 1: delta_{i+1} - delta_i."""
        d = self.offsets
        return [d[i + 1] - d[i] for i in range(len(d) - 1)]

    def fits(self):
        return self.Hp * self.Wp <= self.N // 2 and self.Ho >= 1 and self.Wo >= 1


def galois_step(s, N):
    """The Galois element of a left rotation of both slot rows by s slots."""
    return pow(5, s, 2 * N)


def conv_input_slots(x, shape: ConvShape, P):
    """x [C][H][W] residues mod P -> slot vectors [C][2][N/2] (padded image in both rows)."""
    x = np.asarray(x, dtype=np.int64) % P
    out = np.zeros((shape.C, 2, shape.N // 2), dtype=np.int64)
    for c in range(shape.C):
        img = np.zeros((shape.Hp, shape.Wp), dtype=np.int64)
        img[shape.pad:shape.pad + shape.H, shape.pad:shape.pad + shape.W] = x[c]
        out[c, :, :shape.Hp * shape.Wp] = img.reshape(-1)
    return out


def conv_weight_slots(K, shape: ConvShape, P):
    """K [M][C][kh][kw] residues mod P -> slot vectors [Y][kh*kw][C][2][N/2]: slot row r of
    w_{y,i,c} is the constant K[2y + r][c][l][l'] (0 past M)."""
    K = np.asarray(K, dtype=np.int64) % P
    n = shape.kh * shape.kw
    out = np.zeros((shape.Y, n, shape.C, 2, shape.N // 2), dtype=np.int64)
    for y in range(shape.Y):
        for r in range(2):
            m = 2 * y + r
            if m >= shape.M:
                continue
            for i in range(n):
                l, lp = divmod(i, shape.kw)
                for c in range(shape.C):
                    out[y, i, c, r, :] = K[m, c, l, lp]
    return out


def conv_output(slots, shape: ConvShape):
    """Output slot vectors [Y][2][N/2] -> y [M][Ho][Wo]."""
    out = np.zeros((shape.M, shape.Ho, shape.Wo), dtype=np.int64)
    for m in range(shape.M):
        y, r = divmod(m, 2)
        for i in range(shape.Ho):
            out[m, i] = slots[y][r][i * shape.Wp:i * shape.Wp + shape.Wo]
    return out


def slot_conv(xs, ws, shape: ConvShape, P):
    """The plain counterpart on slot vectors: sum_i rot^(delta_i)(sum_c xs[c] * ws[y][i][c]) mod P,
    rot = left rotation of both rows; returns [Y][2][N/2]."""
    xs = np.asarray(xs, dtype=object)
    out = np.zeros((shape.Y, 2, shape.N // 2), dtype=object)
    for y in range(shape.Y):
        for i, d in enumerate(shape.offsets):
            p = sum((xs[c] * np.asarray(ws[y][i][c], dtype=object)) % P for c in range(shape.C)) % P
            out[y] = (out[y] + np.roll(p, -d, axis=1)) % P
    return out.astype(np.int64)


def conv2d_mod(x, K, pad, P):
    """Plain stride-1 cross-correlation mod P by a direct loop (big integers)."""
    x = np.asarray(x, dtype=object)
    K = np.asarray(K, dtype=object)
    C, H, W = x.shape
    M, _, kh, kw = K.shape
    xp = np.zeros((C, H + 2 * pad, W + 2 * pad), dtype=object)
    xp[:, pad:pad + H, pad:pad + W] = x
    Ho, Wo = H + 2 * pad - kh + 1, W + 2 * pad - kw + 1
    out = np.zeros((M, Ho, Wo), dtype=object)
    for m in range(M):
        for i in range(Ho):
            for j in range(Wo):
                out[m, i, j] = int((xp[:, i:i + kh, j:j + kw] * K[m]).sum()) % P
    return out.astype(np.int64)


def centered(p, P):
    """Plaintext polynomial [N] in [0, P) -> its centered integer coefficients."""
    p = np.asarray(p, dtype=np.int64)
    return np.where(p > (P - 1) // 2, p - P, p)


def mul_plain_small(ct, w_cen, moduli):
    """(c0 * w, c1 * w) over R_Q for a plaintext given by its centered integer coefficients:
    the product of mul_plain with lift_plain(w), summed over w's nonzero terms only."""
    sp = core.sparse_of(w_cen)
    N = ct.shape[-1]
    out = np.zeros_like(ct)
    for comp in range(2):
        for i, q in enumerate(moduli):
            out[comp, i] = core.negacyclic_sparse(ct[comp, i], sp, N, q)
    return out


def conv_mac_rotate(cts, w_polys, keys, shape: ConvShape, kp: KsParams, P):
    """The layer on ciphertexts: cts [C][2][L][N] (coefficient domain), w_polys
    [Y][kh*kw][C][N] encoded weight plaintexts in [0, P), keys {step s: Galois key of
    5^s}; returns [Y][2][L][N]:
        P_i = sum_c cts[c] * w_{y,i,c};  acc = P_{n-1};  acc = rot^(step_i)(acc) + P_i."""
    n = shape.kh * shape.kw
    out = np.zeros((shape.Y, 2, kp.L, kp.N), dtype=np.uint64)
    for y in range(shape.Y):
        prods = []
        for i in range(n):
            acc = None
            for c in range(shape.C):
                t = mul_plain_small(cts[c], centered(w_polys[y][i][c], P), kp.moduli)
                acc = t if acc is None else add(acc, t, kp.moduli)
            prods.append(acc)
        acc = prods[n - 1]
        for i in range(n - 2, -1, -1):
            s = shape.steps[i]
            acc = add(rotate(acc, keys[s], galois_step(s, kp.N), kp), prods[i], kp.moduli)
        out[y] = acc
    return out
