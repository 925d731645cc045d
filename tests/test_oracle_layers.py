"""Pins of the oracle's strided convolutions (polyphase reading) and fully
connected layers (matrix-vector packing): the linear layers of SqueezeNet-1.1
and ResNet-50 beyond stride-1 convolutions (Sec. 8.1; Sec. 6.1 runs every
linear layer with coefficient encoding).  The strided convolution is pinned
against a direct loop, the stride-1 convolution it subsamples and a library
convolution; the polyphase split against the strided definition by brute
force; the FC packing against the exact integer matrix-vector product and end
to end through BFV, with the server's share and mask."""
import numpy as np
import pytest

from oracle import bfv, conv, layers
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream

torch = pytest.importorskip("torch")


def _direct_strided(x, K, stride, pad, t):
    """Loops over Python ints: y[m,r,c] = sum x~[ch, s*r+l, s*c+l'] K[m,ch,l,l'] mod t."""
    C, H, W = x.shape
    M, _, kh, kw = K.shape
    Ho, Wo = (H + 2 * pad - kh) // stride + 1, (W + 2 * pad - kw) // stride + 1
    y = np.zeros((M, Ho, Wo), dtype=np.int64)
    for m in range(M):
        for r in range(Ho):
            for c in range(Wo):
                acc = 0
                for ch in range(C):
                    for l in range(kh):
                        for l2 in range(kw):
                            i, j = stride * r + l - pad, stride * c + l2 - pad
                            if 0 <= i < H and 0 <= j < W:
                                acc += int(x[ch, i, j]) * int(K[m, ch, l, l2])
                y[m, r, c] = acc % t
    return y


def _tensors(s, C, H, W, M, kh, kw, xbound=T_PLAIN):
    x = s.below(xbound, C * H * W).astype(np.int64).reshape(C, H, W)
    K = s.int8(M * C * kh * kw).astype(np.int64).reshape(M, C, kh, kw)
    return x, K


STRIDED = [  # (C, H, W, M, kh, kw, stride, pad)
    (3, 9, 9, 2, 3, 3, 2, 0),      # SqueezeNet conv1 form: 3x3 stride 2, no padding
    (3, 11, 10, 2, 7, 7, 2, 3),    # ResNet-50 conv1 form: 7x7 stride 2, padding 3
    (4, 8, 8, 3, 3, 3, 2, 1),      # ResNet-50 downsampling 3x3 stride 2, padding 1
    (4, 8, 7, 3, 1, 1, 2, 0),      # ResNet-50 projection 1x1 stride 2
    (2, 10, 9, 2, 4, 2, 3, 1),     # stride 3, kernel not a multiple of it, non-square
    (2, 6, 6, 2, 2, 3, 2, 2),      # padding larger than the kernel overhang
]


@pytest.mark.parametrize("shape", STRIDED)
def test_strided_conv_vs_direct_loop(shape):
    C, H, W, M, kh, kw, s_, pad = shape
    x, K = _tensors(Stream(41, sum(shape)), C, H, W, M, kh, kw)
    assert np.array_equal(layers.conv2d_strided_mod_t(x, K, s_, pad, T_PLAIN), _direct_strided(x, K, s_, pad, T_PLAIN))


@pytest.mark.parametrize("shape", STRIDED)
def test_strided_conv_subsamples_stride_one(shape):
    C, H, W, M, kh, kw, s_, pad = shape
    x, K = _tensors(Stream(42, sum(shape)), C, H, W, M, kh, kw)
    y = layers.conv2d_strided_mod_t(x, K, s_, pad, T_PLAIN)
    y1 = conv.conv2d_mod_t(x, K, pad, T_PLAIN)
    assert np.array_equal(y, y1[:, ::s_, ::s_][:, :y.shape[1], :y.shape[2]])
    assert np.array_equal(layers.conv2d_strided_mod_t(x, K, 1, pad, T_PLAIN), y1)


@pytest.mark.parametrize("shape", STRIDED)
def test_strided_conv_vs_library(shape):
    # small activations keep every float64 partial sum exact
    C, H, W, M, kh, kw, s_, pad = shape
    x, K = _tensors(Stream(43, sum(shape)), C, H, W, M, kh, kw, xbound=1 << 12)
    ref = torch.nn.functional.conv2d(torch.tensor(x, dtype=torch.float64)[None], torch.tensor(K, dtype=torch.float64),
                                     stride=s_, padding=pad)[0].numpy().astype(np.int64)
    assert np.array_equal(layers.conv2d_strided_mod_t(x, K, s_, pad, T_PLAIN), np.mod(ref, T_PLAIN))


def test_polyphase_brute_force():
    s = Stream(44, 0)
    n = 0
    for stride in (2, 3):
        for kh in (1, 2, 3, 4, 7):
            for kw in (1, 3):
                for pad in (0, 1, 3):
                    for H in (7, 8, 12):
                        if kh > H + 2 * pad:
                            continue
                        W = H - 1 if kw <= H - 1 + 2 * pad else H
                        x, K = _tensors(s, 2, H, W, 2, kh, kw)
                        ph = layers.polyphase_shape(2, H, W, kh, kw, stride, pad)
                        xs, Ks = layers.polyphase_input(x, ph), layers.polyphase_kernel(K, ph)
                        assert xs.shape == (ph.C1, ph.H1, ph.W1) and Ks.shape == (2, ph.C1, ph.kh1, ph.kw1)
                        got = conv.conv2d_mod_t(xs, Ks, 0, T_PLAIN)
                        assert got.shape == (2, ph.Ho, ph.Wo)
                        assert np.array_equal(got, layers.conv2d_strided_mod_t(x, K, stride, pad, T_PLAIN)), \
                            (stride, kh, kw, pad, H)
                        n += 1
    assert n > 100


def test_polyphase_shapes_of_the_networks():
    # SqueezeNet-1.1 conv1: 3 -> 64, 3x3 stride 2, no padding, 224 x 224
    ph = layers.polyphase_shape(3, 224, 224, 3, 3, 2, 0)
    assert (ph.Ho, ph.C1, ph.H1, ph.kh1) == (111, 12, 112, 2)
    # ResNet-50 conv1: 3 -> 64, 7x7 stride 2, padding 3
    ph = layers.polyphase_shape(3, 224, 224, 7, 7, 2, 3)
    assert (ph.Ho, ph.C1, ph.H1, ph.kh1) == (112, 12, 115, 4)
    # ResNet-50 projection 1x1 stride 2 keeps one phase
    ph = layers.polyphase_shape(256, 56, 56, 1, 1, 2, 0)
    assert (ph.Ho, ph.C1, ph.H1, ph.kh1, ph.pa, ph.pb) == (28, 256, 28, 1, 1, 1)
    # a 1x1 stride-2 layer is the stride-1 layer on the subsampled input
    x, K = _tensors(Stream(45, 0), 3, 9, 8, 2, 1, 1)
    assert np.array_equal(layers.polyphase_input(x, layers.polyphase_shape(3, 9, 8, 1, 1, 2, 0)), x[:, ::2, ::2])


def _encrypt_all(s, params, sk, packed):
    ct = np.zeros((packed.shape[0], 2, len(params.moduli), params.N), dtype=np.uint64)
    for i in range(packed.shape[0]):
        a = np.stack([s.below(q, params.N) for q in params.moduli])
        ct[i] = bfv.encrypt(params, sk, packed[i], a, s.rounded_gaussian(params.N))
    return ct


@pytest.mark.parametrize("shape", [(3, 11, 10, 4, 7, 7, 2, 3, 1024), (4, 9, 9, 3, 3, 3, 2, 1, 256),
                                   (5, 8, 8, 2, 1, 1, 2, 0, 128)])
def test_strided_server_step_end_to_end(shape):
    C, H, W, M, kh, kw, stride, pad, N = shape
    s = Stream(46, sum(shape))
    params = bfv.Params(N, CANONICAL_PRIMES[:2], T_PLAIN)
    sk = s.ternary(N)
    x_c, K = _tensors(s, C, H, W, M, kh, kw)
    x_s, _ = _tensors(s, C, H, W, M, kh, kw)
    ph, p = layers.strided_partition(C, H, W, M, kh, kw, stride, pad, N)
    assert p.pad == 0 and (p.Ho, p.Wo) == (ph.Ho, ph.Wo)
    r = s.below(T_PLAIN, M * p.Ho * p.Wo).astype(np.int64).reshape(M, p.Ho, p.Wo)
    ct = _encrypt_all(s, params, sk, conv.pack_input(layers.polyphase_input(x_c, ph), p))
    ct1 = layers.strided_share_add(ct, x_s, ph, p, params.moduli, T_PLAIN)
    out = conv.conv_ct_pt(ct1, conv.pack_weights(layers.polyphase_kernel(K, ph), p), p, params.moduli)
    slots = conv.extract_masked(out, r, p, params.moduli, T_PLAIN)
    y = layers.conv2d_strided_mod_t((x_c + x_s) % T_PLAIN, K, stride, pad, T_PLAIN)
    checked = 0
    for m in range(M):
        for b in range(p.B):
            o = m * p.B + b
            for k, row, col in conv.output_slots(p, b):
                rel = k - p.offset
                c = out[o].copy()
                c[0, :, k] = slots[o, :, (rel // p.Ww) * p.ow + rel % p.Ww]
                assert int(bfv.decrypt_at(params, sk, c, [k])[0]) == (int(y[m, row, col]) - int(r[m, row, col])) % T_PLAIN
                checked += 1
    assert checked == M * ph.Ho * ph.Wo


# ---- fully connected ------------------------------------------------------------

def _negacyclic_int(a, b):
    """Exact integer product in Z[X]/(X^N + 1) by the schoolbook definition."""
    N = len(a)
    c = [0] * N
    for i in range(N):
        if a[i]:
            for j in range(N):
                k = i + j
                if k < N:
                    c[k] += int(a[i]) * int(b[j])
                else:
                    c[k - N] -= int(a[i]) * int(b[j])
    return c


@pytest.mark.parametrize("C,M,N,Cw,No", [(10, 7, 64, 4, 5), (9, 13, 64, 9, 7), (5, 3, 32, 5, 6), (16, 8, 64, 3, 1)])
def test_fc_packing_integer_matvec(C, M, N, Cw, No):
    s = Stream(47, C * M)
    x = s.below(1 << 20, C).astype(np.int64)
    Wm = s.int8(M * C).astype(np.int64).reshape(M, C)
    fp = layers.FcPartition(C, M, N, Cw, No)
    assert fp.No * fp.Cw <= N
    xin, wp = layers.pack_fc_input(x, fp), layers.pack_fc_weights(Wm, fp)
    want = [sum(int(Wm[m, c]) * int(x[c]) for c in range(C)) for m in range(M)]
    for mp in range(fp.Mp):
        acc = [0] * N
        for g in range(fp.G):
            prod = _negacyclic_int(xin[g], wp[mp * fp.G + g])
            acc = [u + v for u, v in zip(acc, prod)]
        for r in range(fp.No):
            m = mp * fp.No + r
            if m < M:
                assert layers.fc_output_coeff(fp, m) == (mp, r * Cw + Cw - 1)
                assert acc[r * Cw + Cw - 1] == want[m], (mp, r)


def test_fc_with_one_row_is_a_one_by_one_convolution():
    s = Stream(48, 0)
    C, M, N, Cw = 11, 5, 64, 4
    x = s.below(T_PLAIN, C).astype(np.int64)
    Wm = s.int8(M * C).astype(np.int64).reshape(M, C)
    fp = layers.FcPartition(C, M, N, Cw, 1)
    p = conv.Partition(C, 1, 1, M, 1, 1, 0, N, Cw, 1, 1)
    assert (fp.I, fp.P, fp.O) == (p.I, p.P, p.O)
    assert np.array_equal(layers.pack_fc_input(x, fp), conv.pack_input(x.reshape(C, 1, 1), p))
    assert np.array_equal(layers.pack_fc_weights(Wm, fp), conv.pack_weights(Wm.reshape(M, C, 1, 1), p))


def test_canonical_fc_partition():
    # C = 512, M = 10, N = 4096: one input poly (Cw = 512, up to 8 rows each) and
    # two outputs; No = 5 ties No = 8 on every count and is the smaller
    fp = layers.canonical_fc_partition(512, 10, 4096)
    assert (fp.Cw, fp.No, fp.G, fp.Mp, fp.cost()) == (512, 5, 1, 2, 8)
    for C, M, N in ((37, 23, 128), (100, 9, 256), (7, 40, 64)):
        fp = layers.canonical_fc_partition(C, M, N)
        assert fp.Cw * fp.No <= N
        best = min(layers.FcPartition(C, M, N, cw, no).cost()
                   for cw in range(1, min(C, N) + 1) for no in range(1, min(M, N // cw) + 1))
        assert fp.cost() == best
    # ResNet-50's classifier 2048 -> 1000 at N = 16384 needs 126 products (1000 with one row per poly)
    fp = layers.canonical_fc_partition(2048, 1000, 16384)
    assert (fp.Cw, fp.No, fp.G, fp.Mp, fp.P) == (114, 143, 18, 7, 126)


def test_fc_server_step_end_to_end():
    C, M, N = 45, 23, 256
    s = Stream(49, 0)
    params = bfv.Params(N, CANONICAL_PRIMES[:2], T_PLAIN)
    sk = s.ternary(N)
    fp = layers.FcPartition(C, M, N, 20, 9)                   # 3 input chunks (ragged), 3 outputs (ragged)
    assert (fp.G, fp.Mp) == (3, 3)
    x_c = s.below(T_PLAIN, C).astype(np.int64)
    x_s = s.below(T_PLAIN, C).astype(np.int64)
    Wm = s.int8(M * C).astype(np.int64).reshape(M, C)
    r = s.below(T_PLAIN, M).astype(np.int64)
    ct = _encrypt_all(s, params, sk, layers.pack_fc_input(x_c, fp))
    ct1 = layers.fc_share_add(ct, x_s, fp, params.moduli, T_PLAIN)
    out = conv.conv_ct_pt(ct1, layers.pack_fc_weights(Wm, fp), fp, params.moduli)
    slots = layers.fc_extract_masked(out, r, fp, params.moduli, T_PLAIN)
    assert slots.shape == (fp.Mp, 2, fp.No)
    y = layers.fc_mod_t((x_c + x_s) % T_PLAIN, Wm, T_PLAIN)
    for m in range(M):
        mp, k = layers.fc_output_coeff(fp, m)
        c = out[mp].copy()
        c[0, :, k] = slots[mp, :, m - mp * fp.No]
        assert int(bfv.decrypt_at(params, sk, c, [k])[0]) == (int(y[m]) - int(r[m])) % T_PLAIN, m
    assert not slots[fp.Mp - 1, :, M - (fp.Mp - 1) * fp.No:].any()   # rows past M are zero
