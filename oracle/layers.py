"""Strided convolutions and fully connected layers as coefficient-packed
products.  TEST INFRASTRUCTURE ONLY.

The paper's networks contain linear layers beyond stride-1 convolutions: the
stride-2 first convolutions of SqueezeNet-1.1 and ResNet-50 (a 7x7 one in
ResNet-50), ResNet-50's stride-2 downsampling convolutions, and ResNet-50's
fully connected classifier (Sec. 8.1 lists both networks; Sec. 6.1 runs all
linear layers with Cheetah's coefficient encoding).  The paper prints no
packing for them either.  This module holds the reading the build uses:

Strided convolution (polyphase reading).  A stride-s convolution with zero
padding p, y[m, r, c] = sum_{ch,l,l'} x~[ch, s*r + l, s*c + l'] K[m, ch, l, l']
(x~ the padded input), equals a stride-1 convolution without padding of the
phase-split input
    x'[(a*pb + b)*C + ch, i, j] = x~[ch, s*i + a, s*j + b]   (0 past x~'s edge)
with the phase-split kernel
    K'[m, (a*pb + b)*C + ch, u, v] = K[m, ch, s*u + a, s*v + b]   (0 past kh, kw)
for phases a < pa = min(s, kh), b < pb = min(s, kw), kernel size
kh' = ceil(kh/s), kw' = ceil(kw/s), and x' of height Ho + kh' - 1 and width
Wo + kw' - 1, where Ho = (H + 2p - kh)//s + 1, Wo = (W + 2p - kw)//s + 1 are
the strided output sizes.  (Write l = s*u + a: s*r + l = s*(r + u) + a.)  The
stride-1 layer is then packed by ``conv`` with its canonical partition; the
client packs x' instead of x.  Phases a >= kh never meet a nonzero weight
and are dropped (a 1x1 stride-2 convolution keeps only phase (0, 0)).

Fully connected layer (matrix-vector reading).  y[m] = sum_c Wm[m, c] x[c].
Input chunks of Cw values, No output rows per output polynomial, No*Cw <= N:
    input poly g            : coeff [c]                = x[g*Cw + c]
    weight poly p = m'*G + g : coeff [r*Cw + Cw-1 - c]  = Wm[m'*No + r, g*Cw + c]
    output poly m'           : coeff [r*Cw + Cw-1] of sum_g in(g) * w(m', g)
                               holds y[m'*No + r]
G = ceil(C/Cw) inputs, Mp = ceil(M/No) outputs, P = Mp*G weight polys.  A
product term lands at r*Cw + Cw-1 + (c_in - c) with |c_in - c| < Cw, so no
term of another row r reaches an extracted coefficient, and a term past X^N
wraps to an index below Cw - 1, so the negacyclic sign never reaches one
either.  With No = 1 this is the packing of a 1x1 convolution on a 1x1 image.
Canonical partition: minimise 2I + P + 2O = 2G + Mp*G + 2Mp; ties go to fewer
weight polys P, then larger Cw, then smaller No.

Parity: the strided convolution is pinned against a direct loop, against the
stride-1 convolution it subsamples, and against a library convolution; the
polyphase reading against the strided definition by brute force; the FC
packing against the exact integer matrix-vector product and end to end
through BFV (tests/test_oracle_layers.py).
"""
from dataclasses import dataclass

import numpy as np

from . import conv


# ---- strided convolution ------------------------------------------------------

def strided_out_size(H, W, kh, kw, stride, pad):
    """(Ho, Wo) of a stride-s convolution with zero padding pad."""
    Hp, Wp = H + 2 * pad, W + 2 * pad
    if kh > Hp or kw > Wp:
        raise ValueError("kernel larger than the padded input")
    return (Hp - kh) // stride + 1, (Wp - kw) // stride + 1


def conv2d_strided_mod_t(x, K, stride, pad, t):
    """Plain definition: y[m, r, c] = sum_{ch,l,l'} x~[ch, s*r+l, s*c+l'] K[m,ch,l,l'] mod t."""
    xp = conv.pad_input(x, pad)
    K = np.asarray(K, dtype=np.int64)
    M, C, kh, kw = K.shape
    Ho, Wo = strided_out_size(x.shape[1], x.shape[2], kh, kw, stride, pad)
    assert int(np.abs(xp).max(initial=0)) < (1 << 40) and int(np.abs(K).max(initial=0)) <= 128
    assert C * kh * kw <= (1 << 15)
    y = np.zeros((M, Ho, Wo), dtype=np.int64)
    for l in range(kh):
        for l2 in range(kw):
            win = xp[:, l:l + stride * (Ho - 1) + 1:stride, l2:l2 + stride * (Wo - 1) + 1:stride]
            y += np.tensordot(K[:, :, l, l2], win, axes=([1], [0]))
    return np.mod(y, t)


@dataclass(frozen=True)
class Polyphase:
    """Shapes of the stride-1 layer a strided convolution becomes."""
    C: int
    H: int
    W: int
    kh: int
    kw: int
    stride: int
    pad: int
    pa: int      # row phases kept
    pb: int      # column phases kept
    C1: int      # channels of x'
    H1: int      # height of x'
    W1: int      # width of x'
    kh1: int
    kw1: int
    Ho: int
    Wo: int


def polyphase_shape(C, H, W, kh, kw, stride, pad):
    Ho, Wo = strided_out_size(H, W, kh, kw, stride, pad)
    pa, pb = min(stride, kh), min(stride, kw)
    kh1, kw1 = -(-kh // stride), -(-kw // stride)
    return Polyphase(C, H, W, kh, kw, stride, pad, pa, pb, pa * pb * C, Ho + kh1 - 1, Wo + kw1 - 1,
                     kh1, kw1, Ho, Wo)


def polyphase_input(x, ph: Polyphase):
    """x (C, H, W) -> x' (C1, H1, W1): x'[(a*pb+b)*C + ch, i, j] = x~[ch, s*i+a, s*j+b]."""
    xp = conv.pad_input(x, ph.pad)
    s = ph.stride
    out = np.zeros((ph.C1, ph.H1, ph.W1), dtype=np.int64)
    for a in range(ph.pa):
        for b in range(ph.pb):
            sub = xp[:, a::s, b::s][:, :ph.H1, :ph.W1]
            base = (a * ph.pb + b) * ph.C
            out[base:base + ph.C, :sub.shape[1], :sub.shape[2]] = sub
    return out


def polyphase_kernel(K, ph: Polyphase):
    """K (M, C, kh, kw) -> K' (M, C1, kh1, kw1): K'[m, (a*pb+b)*C + ch, u, v] = K[m, ch, s*u+a, s*v+b]."""
    K = np.asarray(K, dtype=np.int64)
    M = K.shape[0]
    s = ph.stride
    out = np.zeros((M, ph.C1, ph.kh1, ph.kw1), dtype=np.int64)
    for a in range(ph.pa):
        for b in range(ph.pb):
            sub = K[:, :, a::s, b::s]
            base = (a * ph.pb + b) * ph.C
            out[:, base:base + ph.C, :sub.shape[2], :sub.shape[3]] = sub
    return out


def strided_partition(C, H, W, M, kh, kw, stride, pad, N):
    """(Polyphase, canonical conv.Partition of the stride-1 layer without padding)."""
    ph = polyphase_shape(C, H, W, kh, kw, stride, pad)
    return ph, conv.canonical_partition(ph.C1, ph.H1, ph.W1, M, ph.kh1, ph.kw1, 0, N)


# ---- fully connected layer -------------------------------------------------------

@dataclass(frozen=True)
class FcPartition:
    """Matrix-vector packing of y = Wm x (Wm: M x C) for ring degree N.  Exposes
    B, G, O, N like conv.Partition so that conv.conv_ct_pt computes its products."""
    C: int
    M: int
    N: int
    Cw: int
    No: int

    @property
    def G(self):
        return -(-self.C // self.Cw)

    @property
    def Mp(self):
        return -(-self.M // self.No)

    B = 1

    @property
    def I(self):
        return self.G

    @property
    def P(self):
        return self.Mp * self.G

    @property
    def O(self):
        return self.Mp

    @property
    def products(self):
        return self.P

    def cost(self):
        return 2 * self.I + self.P + 2 * self.O


def canonical_fc_partition(C, M, N):
    """Exhaustive search over Cw in [1, min(C, N)], No in [1, min(M, N // Cw)]:
    minimal 2I + P + 2O, then fewer P, then larger Cw, then smaller No."""
    best_key, best = None, None
    for Cw in range(1, min(C, N) + 1):
        for No in range(1, min(M, N // Cw) + 1):
            p = FcPartition(C, M, N, Cw, No)
            key = (p.cost(), p.P, -Cw, No)
            if best_key is None or key < best_key:
                best_key, best = key, p
    return best


def pack_fc_input(x, fp: FcPartition):
    """x (C,) small non-negative ints -> [G][N] int64 polys: coeff [c] of poly g = x[g*Cw + c]."""
    x = np.asarray(x, dtype=np.int64).reshape(-1)
    out = np.zeros((fp.G, fp.N), dtype=np.int64)
    for g in range(fp.G):
        chunk = x[g * fp.Cw:(g + 1) * fp.Cw]
        out[g, :len(chunk)] = chunk
    return out


def pack_fc_weights(Wm, fp: FcPartition):
    """Wm (M, C) small signed ints -> [P][N] int64 polys (p = m'*G + g):
    coeff [r*Cw + Cw-1 - c] = Wm[m'*No + r, g*Cw + c]."""
    Wm = np.asarray(Wm, dtype=np.int64)
    out = np.zeros((fp.P, fp.N), dtype=np.int64)
    for mp in range(fp.Mp):
        for g in range(fp.G):
            poly = out[mp * fp.G + g]
            for r in range(fp.No):
                m = mp * fp.No + r
                if m >= fp.M:
                    break
                for c in range(fp.Cw):
                    ch = g * fp.Cw + c
                    if ch >= fp.C:
                        break
                    poly[r * fp.Cw + fp.Cw - 1 - c] = Wm[m, ch]
    return out


def fc_output_coeff(fp: FcPartition, m):
    """(output poly m', coefficient) that holds y[m]."""
    mp, r = divmod(m, fp.No)
    return mp, r * fp.Cw + fp.Cw - 1


def fc_mod_t(x, Wm, t):
    """y[m] = sum_c Wm[m, c] x[c] mod t (exact integers)."""
    x = [int(v) for v in np.asarray(x).reshape(-1)]
    Wm = np.asarray(Wm, dtype=np.int64)
    return np.array([sum(int(Wm[m, c]) * x[c] for c in range(len(x))) % t for m in range(Wm.shape[0])],
                    dtype=np.int64)


# ---- the server's step for these layers (Sec. 7, Sec. 6.2) -----------------------

def strided_share_add(ct_in, x_s, ph: Polyphase, p: conv.Partition, moduli, t):
    """c0 += Delta * pack(x'_s): the server share goes through the same phase split."""
    return conv.share_add(ct_in, polyphase_input(x_s, ph), p, moduli, t)


def fc_share_add(ct_in, x_s, fp: FcPartition, moduli, t):
    """Client ciphertexts [G][2][L][N] plus the server share x_s (C,) in [0, t)."""
    packed = pack_fc_input(x_s, fp).astype(object)
    out = np.array(ct_in, dtype=np.uint64, copy=True)
    d = conv.delta_residues(moduli, t)
    for li, q in enumerate(moduli):
        c0 = out[:, 0, li].astype(object)
        out[:, 0, li] = ((c0 + d[li] * packed) % int(q)).astype(np.uint64)
    return out


def fc_extract_masked(ct_out, r, fp: FcPartition, moduli, t):
    """Output ciphertexts [Mp][2][L][N] and the output mask r (M,) in [0, t) ->
    [Mp][L][No]: slot j of output m' holds c0[j*Cw + Cw-1] - Delta*r[m'*No + j]
    mod q_l, and 0 for j with m'*No + j >= M."""
    d = conv.delta_residues(moduli, t)
    out = np.zeros((fp.Mp, len(moduli), fp.No), dtype=np.uint64)
    for m in range(fp.M):
        mp, k = fc_output_coeff(fp, m)
        j = m - mp * fp.No
        for li, q in enumerate(moduli):
            out[mp, li, j] = (int(ct_out[mp, 0, li, k]) - d[li] * int(r[m])) % int(q)
    return out
