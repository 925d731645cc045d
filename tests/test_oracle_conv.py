"""Pins of the oracle's convolution packing (Sec. 6.1-6.2 reading), canonical
partition and plaintext convolution, end to end through BFV."""
import numpy as np
import pytest

from oracle import bfv, conv
from paper_2506_11586_gb300.inputs import (CANONICAL_PRIMES, CONV_56x56x64, SQUEEZENET_1_1,
                                           T_PLAIN, Stream, conv_tensors)


def _direct_conv(x, K, pad, t):
    """Quadruple loop over Python ints: y[m,r,s] = sum x~[c,r+l,s+l'] K[m,c,l,l'] mod t."""
    C, H, W = x.shape
    M, _, kh, kw = K.shape
    Hp, Wp = H + 2 * pad, W + 2 * pad
    Ho, Wo = Hp - kh + 1, Wp - kw + 1

    def xp(c, r, s):
        r -= pad
        s -= pad
        if 0 <= r < H and 0 <= s < W:
            return int(x[c, r, s])
        return 0

    y = np.zeros((M, Ho, Wo), dtype=np.int64)
    for m in range(M):
        for r in range(Ho):
            for s in range(Wo):
                acc = 0
                for c in range(C):
                    for l in range(kh):
                        for l2 in range(kw):
                            acc += xp(c, r + l, s + l2) * int(K[m, c, l, l2])
                y[m, r, s] = acc % t
    return y


def test_plain_conv_vs_direct_loop():
    s = Stream(2, 0)
    x = s.below(T_PLAIN, 3 * 5 * 6).astype(np.int64).reshape(3, 5, 6)
    K = s.int8(4 * 3 * 3 * 3).astype(np.int64).reshape(4, 3, 3, 3)
    for pad in (0, 1):
        assert np.array_equal(conv.conv2d_mod_t(x, K, pad, T_PLAIN), _direct_conv(x, K, pad, T_PLAIN))


def test_canonical_partition_config_56x56x64():
    sh = CONV_56x56x64
    p = conv.canonical_partition(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, sh.pad, 8192)
    assert (p.Cw, p.Hw, p.Ww) == (8, 32, 32)
    assert (p.G, p.B, p.I, p.P, p.O, p.products) == (8, 4, 32, 512, 256, 2048)


def test_partition_invariants_squeezenet():
    for sh in SQUEEZENET_1_1:
        p = conv.canonical_partition(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, sh.pad, 8192)
        assert p.Cw * p.Hw * p.Ww <= 8192
        assert p.G * p.Cw >= p.C > (p.G - 1) * p.Cw
        # blocks tile the output exactly once
        seen = np.zeros((p.Ho, p.Wo), dtype=np.int64)
        for b in range(p.B):
            for _, r, c in conv.output_slots(p, b):
                seen[r, c] += 1
        assert np.all(seen == 1), sh.name


def _e2e(C, H, W, M, kh, kw, pad, N, L, seed, partition=None):
    s = Stream(seed, 0)
    x = s.below(T_PLAIN, C * H * W).astype(np.int64).reshape(C, H, W)
    K = s.int8(M * C * kh * kw).astype(np.int64).reshape(M, C, kh, kw)
    p = partition or conv.canonical_partition(C, H, W, M, kh, kw, pad, N)
    params = bfv.Params(N, CANONICAL_PRIMES[:L], T_PLAIN)
    sk = s.ternary(N)
    xin = conv.pack_input(x, p)
    ct = np.zeros((p.I, 2, L, N), dtype=np.uint64)
    for i in range(p.I):
        a = np.stack([s.below(q, N) for q in params.moduli])
        ct[i] = bfv.encrypt(params, sk, xin[i], a, s.rounded_gaussian(N))
    Kp = conv.pack_weights(K, p)
    out = conv.conv_ct_pt(ct, Kp, p, params.moduli)
    y = conv.conv2d_mod_t(x, K, pad, T_PLAIN)
    for m in range(M):
        for b in range(p.B):
            slots = conv.output_slots(p, b)
            ks = [k for k, _, _ in slots]
            got = bfv.decrypt_at(params, sk, out[m * p.B + b], ks)
            want = np.array([y[m, r, c] for _, r, c in slots])
            assert np.array_equal(got, want), (m, b)
    return p


@pytest.mark.parametrize("shape", [
    (5, 7, 6, 3, 3, 3, 1, 256, 2),     # ragged channel group and edge blocks
    (4, 6, 6, 2, 1, 1, 0, 64, 2),      # 1x1 convolution
    (3, 9, 4, 2, 3, 1, 0, 128, 3),     # non-square kernel
])
def test_packing_end_to_end(shape):
    p = _e2e(*shape, seed=sum(shape))
    assert p.B >= 1 and p.G >= 1


def test_packing_end_to_end_forced_partition():
    """A deliberately non-canonical partition with several groups and blocks."""
    C, H, W, M, kh, kw, pad, N = 6, 8, 8, 2, 3, 3, 1, 128
    p = conv.Partition(C, H, W, M, kh, kw, pad, N, Cw=4, Hw=5, Ww=6)
    assert p.G == 2 and p.B > 1
    _e2e(C, H, W, M, kh, kw, pad, N, 2, seed=77, partition=p)
