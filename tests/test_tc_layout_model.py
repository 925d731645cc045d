"""Host model of the tensor-core MAC's operands (csrc/hc_mac_tc.cu, the MAC of
Sec. 6.2 on tcgen05 MMAs): the A image (K-major, 128-byte swizzle, two slots
block-diagonal over a shared zero block) and the B arrays (K-major without
swizzle, rows 16 bytes apart, core matrices 16 bytes apart along K and 128
bytes along N, so that one linear array of 7 chunks per (slot, column block)
is read as the whole limb-shifted matrix) are built byte for byte as the
kernel builds them, read back through the descriptors' address rules, and
multiplied: every column sum must stay below 2^22 (exact in fp32 in any order)
and the recombined sum_t S_t 2^(8t) must equal the integer dot product
sum_g w_g x_g for every (slot, channel, column block), for random residues
and for the largest ones (every 8-bit limb 255)."""
import numpy as np
import pytest

KB_B = 144 * 16  # one slot's B array, bytes


def chunk_off(r, c):
    """swizzled byte offset of 16-byte chunk c of row r in a K-block (128-byte rows)"""
    return (r // 8) * 1024 + (r % 8) * 128 + ((c ^ (r % 8)) << 4)


def limb(v, i):
    return (int(v) >> (8 * i)) & 0xFF


def build(W, X, G, P):
    """A image (24 KB) and B arrays (two slots) as f16 values, K = (i' = 7 - i, g)."""
    A = np.zeros(24576 // 2)
    B = np.zeros(2 * KB_B // 2)
    for s in range(2):
        for m in range(W.shape[1]):
            for ip in range(8):
                off = s * 16384 + chunk_off(m, ip)  # slot 1's rows 64.. of K-block 1 (at 8 KB)
                A[off // 2:off // 2 + 8] = [limb(W[s, m, g], 7 - ip) if g < G else 0 for g in range(8)]
        for p in range(P):
            for j in range(7):
                off = s * KB_B + (16 * p + 7 + j) * 16
                B[off // 2:off // 2 + 8] = [limb(X[s, g, p], j) if g < G else 0 for g in range(8)]
    return A, B


def read_sw128(A, start, rows):
    """rows x 16 K values of one MMA step: row r at start + (r/8)*1024 + (r%8)*128,
    the address's bits 4-6 xor-ed with bits 7-9 (the 128-byte swizzle)"""
    out = np.zeros((rows, 16))
    for r in range(rows):
        for k in range(16):
            a = start + (r // 8) * 1024 + (r % 8) * 128 + 2 * k
            a ^= ((a >> 7) & 7) << 4
            out[r, k] = A[a // 2]
    return out


def read_plain(B, start, rows, lbo=16, sbo=128):
    """the same without swizzle: row r of a core matrix 16 r bytes in, core
    matrices lbo bytes apart along K and sbo bytes apart along N"""
    out = np.zeros((rows, 16))
    for r in range(rows):
        for k in range(16):
            a = start + (r // 8) * sbo + (r % 8) * 16 + (k // 8) * lbo + 2 * (k % 8)
            out[r, k] = B[a // 2]
    return out


@pytest.mark.parametrize("G, P, worst", [(8, 8, False), (8, 8, True), (3, 2, False), (1, 6, True), (5, 4, False)])
def test_tensor_core_mac_layout_recombines_exactly(G, P, worst):
    q = (1 << 50) - 27
    rng = np.random.default_rng(G * 10 + P)
    W = rng.integers(0, q, size=(2, 64, G), dtype=np.uint64)
    X = rng.integers(0, q, size=(2, G, P), dtype=np.uint64)
    if worst:
        W[:] = (1 << 50) - 1
        X[:] = (1 << 50) - 1
    A, B = build(W, X, G, P)
    D = np.zeros((128, 16 * P))
    for kb in range(2):          # K-block kb: slot kb (block-diagonal)
        for ks in range(4):      # K steps of 16 within the K-block
            D += read_sw128(A, kb * 8192 + ks * 32, 128) @ read_plain(B, kb * KB_B + ks * 32, 16 * P).T
    assert D.max() < 2 ** 22     # every partial sum of non-negative terms is below this: exact in fp32
    for s in range(2):
        for m in range(64):
            for p in range(P):
                V = sum(int(D[64 * s + m, 16 * p + t]) << (8 * t) for t in range(13))
                assert V == sum(int(W[s, m, g]) * int(X[s, g, p]) for g in range(G)), (s, m, p)
                # the unused columns t = 13..15 of the block read only zero chunks
                assert not D[64 * s + m, 16 * p + 13:16 * p + 16].any()
