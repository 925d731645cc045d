"""Cheetah-style coefficient packing of a stride-1 convolution.  TEST INFRASTRUCTURE ONLY.

The paper runs its linear layers with Cheetah's coefficient-encoded HE kernels
(Sec. 2.3, Sec. 6.1): values sit directly in polynomial coefficients so that a
single negacyclic product computes many dot products, the result is sparse, and
only the output coefficients are extracted.  Weights are packed, lifted and
NTT'd once, offline (Sec. 6.2, Sec. 7); online, every input ciphertext is NTT'd,
all MACs run in the NTT domain, and only the final sums are transformed back
(Sec. 6.2).  The paper prints no packing formula; this module holds the reading
the build uses:

  padded input x~ (C x (H+2p) x (W+2p)), channel groups of Cw, spatial blocks
  of Hw x Ww that overlap by kh-1 rows / kw-1 columns, each block producing
  (Hw-kh+1) x (Ww-kw+1) outputs;  Cw*Hw*Ww <= N.

  input poly (g, b)  : coeff [c*Hw*Ww + i*Ww + j]       = x~[g*Cw+c, i0+i, j0+j]
  weight poly (m, g) : coeff [O - c*Hw*Ww - l*Ww - l']  = K[m, g*Cw+c, l, l']
                       with O = (Cw-1)*Hw*Ww + (kh-1)*Ww + (kw-1)
  output (m, b)      : coeff [O + i*Ww + j] of sum_g in(g,b) * w(m,g) holds
                       y[m, i0+i, j0+j] = sum_{c,l,l'} x~[c, i0+i+l, j0+j+l'] K[m,c,l,l']

  (no product term wraps past X^N, so the negacyclic sign never reaches an
  extracted coefficient).  Ordering: input ct i = g*B + b, weight poly
  p = m*G + g, output ct o = m*B + b, block b = bh*Bw + bw.

Canonical partition: minimise the polynomials moved, 2I + P + 2O (I = G*B input
cts, P = M*G weight plaintexts, O = M*B output cts); ties go to the larger
Hw*Ww, then the larger Cw, then the larger Ww.

Parity: pinned end to end -- encrypt -> schoolbook ct x pt conv -> decrypt
equals the plaintext convolution mod t (tests/test_oracle_conv.py), and the
plaintext convolution is pinned against a direct quadruple loop.
"""
from dataclasses import dataclass

import numpy as np

from . import core


@dataclass(frozen=True)
class Partition:
    C: int
    H: int
    W: int
    M: int
    kh: int
    kw: int
    pad: int
    N: int
    Cw: int
    Hw: int
    Ww: int

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
    def G(self):
        return -(-self.C // self.Cw)

    @property
    def oh(self):  # outputs per block, rows
        return self.Hw - self.kh + 1

    @property
    def ow(self):  # outputs per block, columns
        return self.Ww - self.kw + 1

    @property
    def Bh(self):
        return -(-self.Ho // self.oh)

    @property
    def Bw(self):
        return -(-self.Wo // self.ow)

    @property
    def B(self):
        return self.Bh * self.Bw

    @property
    def I(self):
        return self.G * self.B

    @property
    def P(self):
        return self.M * self.G

    @property
    def O(self):
        return self.M * self.B

    @property
    def offset(self):
        return (self.Cw - 1) * self.Hw * self.Ww + (self.kh - 1) * self.Ww + (self.kw - 1)

    @property
    def products(self):
        return self.M * self.G * self.B

    def cost(self):
        return 2 * self.I + self.P + 2 * self.O


def partition_cost(C, H, W, M, kh, kw, pad, N, Cw, Hw, Ww):
    return Partition(C, H, W, M, kh, kw, pad, N, Cw, Hw, Ww).cost()


def canonical_partition(C, H, W, M, kh, kw, pad, N):
    """Exhaustive search over Cw in [1, C], Hw in [kh, H+2p], Ww in [kw, W+2p],
    Cw*Hw*Ww <= N.  Returns the Partition with minimal 2I + P + 2O; ties go to
    larger Hw*Ww, then larger Cw, then larger Ww."""
    Hp, Wp = H + 2 * pad, W + 2 * pad
    if kh > Hp or kw > Wp or kh * kw > N:
        raise ValueError("kernel does not fit")
    best_key, best = None, None
    for Cw in range(1, C + 1):
        if Cw * kh * kw > N:
            break
        for Hw in range(kh, Hp + 1):
            if Cw * Hw * kw > N:
                break
            Ww = min(Wp, N // (Cw * Hw))
            for w in range(kw, Ww + 1):
                p = Partition(C, H, W, M, kh, kw, pad, N, Cw, Hw, w)
                key = (p.cost(), -(Hw * w), -Cw, -w)
                if best_key is None or key < best_key:
                    best_key, best = key, p
    return best


# ---- packing --------------------------------------------------------------

def pad_input(x, pad):
    return np.pad(np.asarray(x, dtype=np.int64), ((0, 0), (pad, pad), (pad, pad)))


def block_origin(p: Partition, b):
    bh, bw = divmod(b, p.Bw)
    return bh * p.oh, bw * p.ow


def pack_input(x, p: Partition):
    """Input activations (C, H, W) of small non-negative ints -> [I][N] int64 polys."""
    xp = pad_input(x, p.pad)
    out = np.zeros((p.I, p.N), dtype=np.int64)
    for g in range(p.G):
        for b in range(p.B):
            i0, j0 = block_origin(p, b)
            poly = out[g * p.B + b]
            for c in range(p.Cw):
                ch = g * p.Cw + c
                if ch >= p.C:
                    break
                for i in range(p.Hw):
                    r = i0 + i
                    if r >= p.Hp:
                        break
                    for j in range(p.Ww):
                        s = j0 + j
                        if s >= p.Wp:
                            break
                        poly[c * p.Hw * p.Ww + i * p.Ww + j] = xp[ch, r, s]
    return out


def pack_weights(K, p: Partition):
    """Weights (M, C, kh, kw) small signed ints -> [P][N] int64 polys (p = m*G + g)."""
    K = np.asarray(K, dtype=np.int64)
    out = np.zeros((p.P, p.N), dtype=np.int64)
    O = p.offset
    for m in range(p.M):
        for g in range(p.G):
            poly = out[m * p.G + g]
            for c in range(p.Cw):
                ch = g * p.Cw + c
                if ch >= p.C:
                    break
                for l in range(p.kh):
                    for l2 in range(p.kw):
                        poly[O - c * p.Hw * p.Ww - l * p.Ww - l2] = K[m, ch, l, l2]
    return out


def output_slots(p: Partition, b):
    """For output block b: list of (coefficient index, out row, out col) that hold outputs."""
    i0, j0 = block_origin(p, b)
    res = []
    for i in range(p.oh):
        if i0 + i >= p.Ho:
            break
        for j in range(p.ow):
            if j0 + j >= p.Wo:
                break
            res.append((p.offset + i * p.Ww + j, i0 + i, j0 + j))
    return res


# ---- plaintext convolution mod t --------------------------------------------

def conv2d_mod_t(x, K, pad, t):
    """y[m, r, s] = sum_{c,l,l'} x~[c, r+l, s+l'] K[m, c, l, l'] mod t (stride 1)."""
    xp = pad_input(x, pad)
    K = np.asarray(K, dtype=np.int64)
    M, C, kh, kw = K.shape
    Ho, Wo = xp.shape[1] - kh + 1, xp.shape[2] - kw + 1
    # exact in int64: |x| < 2^40, |K| <= 2^7 and at most 2^15 terms keep every
    # partial sum below 2^62
    assert int(np.abs(xp).max(initial=0)) < (1 << 40) and int(np.abs(K).max(initial=0)) <= 128
    assert C * kh * kw <= (1 << 15)
    y = np.zeros((M, Ho, Wo), dtype=np.int64)
    for l in range(kh):
        for l2 in range(kw):
            win = xp[:, l:l + Ho, l2:l2 + Wo]
            y += np.tensordot(K[:, :, l, l2], win, axes=([1], [0]))
    return np.mod(y, t)


# ---- ct x pt convolution by schoolbook products ------------------------------

def conv_ct_pt(ct_in, Kpoly, p: Partition, moduli, ks=None, outputs=None):
    """out[o=(m,b)][comp][limb] = sum_g ct_in[g*B+b][comp][limb] * Kpoly[m*G+g]  in R_q.

    ct_in  : [I][2][L][N] uint64 residues; Kpoly: [P][N] small signed ints.
    ks     : coefficient indices to compute (all N if None).
    outputs: output ciphertext indices o to compute (all O if None); the
             result then has len(outputs) rows in that order.
    Uses the sparse-aware schoolbook product (same definition, visits only the
    nonzero weight coefficients).  Returns [O][2][L][len(ks) or N] uint64."""
    L = len(moduli)
    nk = p.N if ks is None else len(ks)
    outs = list(range(p.O)) if outputs is None else [int(o) for o in outputs]
    out = np.zeros((len(outs), 2, L, nk), dtype=np.uint64)
    sparse = {}
    for row, o in enumerate(outs):
        m, b = divmod(o, p.B)
        for g in range(p.G):
            if m * p.G + g not in sparse:
                sparse[m * p.G + g] = core.sparse_of(Kpoly[m * p.G + g])
        for comp in range(2):
            for li, q in enumerate(moduli):
                acc = np.zeros(nk, dtype=object)
                for g in range(p.G):
                    prod = core.negacyclic_sparse(ct_in[g * p.B + b, comp, li], sparse[m * p.G + g],
                                                  p.N, q, ks)
                    acc += prod.astype(object)
                out[row, comp, li] = np.mod(acc, q).astype(np.uint64)
    return out


# ---- the server's step around the convolution (Sec. 7, Sec. 6.2) ---------------
# The client sends encryptions of its activation share; the server adds its own
# share, runs the convolution with the NTT-preprocessed weights, subtracts a
# random mask (its output share) and returns only the output coefficients.
# With Delta = floor(Q/t) (the BFV scale of bfv.Params), adding Delta*m to c0
# adds m to the plaintext, and subtracting Delta*r from c0 subtracts r.

def delta_residues(moduli, t):
    """Delta = floor(prod(moduli) / t) reduced mod every q_i (exact integers)."""
    Q = 1
    for q in moduli:
        Q *= int(q)
    d = Q // int(t)
    return [d % int(q) for q in moduli]


def share_add(ct_in, x_s, p: Partition, moduli, t):
    """Client ciphertexts [I][2][L][N] plus the server share x_s (C, H, W) in [0, t),
    packed like the input: c0 += Delta * pack(x_s) mod q_i; c1 unchanged."""
    packed = pack_input(np.asarray(x_s, dtype=np.int64), p).astype(object)   # [I][N], values < t
    out = np.array(ct_in, dtype=np.uint64, copy=True)
    d = delta_residues(moduli, t)
    for li, q in enumerate(moduli):
        c0 = out[:, 0, li].astype(object)
        out[:, 0, li] = ((c0 + d[li] * packed) % int(q)).astype(np.uint64)
    return out


def slot_count(p: Partition):
    return p.oh * p.ow


def extract_masked(ct_out, r, p: Partition, moduli, t):
    """Output ciphertexts [O][2][L][N] and the server's output mask r (M, Ho, Wo) in
    [0, t) -> [O][L][S] with S = oh*ow: slot s = i*ow + j of output (m, b) holds
    c0[offset + i*Ww + j] - Delta * r[m, i0+i, j0+j] mod q_l for outputs inside the
    Ho x Wo map, and 0 for the slots of an edge block that fall outside it."""
    S = slot_count(p)
    d = delta_residues(moduli, t)
    out = np.zeros((p.O, len(moduli), S), dtype=np.uint64)
    for m in range(p.M):
        for b in range(p.B):
            o = m * p.B + b
            i0, j0 = block_origin(p, b)
            for k, row, col in output_slots(p, b):
                rel = k - p.offset
                s = (rel // p.Ww) * p.ow + rel % p.Ww
                for li, q in enumerate(moduli):
                    out[o, li, s] = (int(ct_out[o, 0, li, k]) - d[li] * int(r[m, row, col])) % int(q)
    return out
