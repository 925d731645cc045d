"""Pins of the oracle's Z_P convolution layer (oracle/zp.py, SecONNds-P's
convolutions over Z_P^N as the multiply-accumulate-rotate iteration, Sec. 6.1
and Sec. 2.3).  The packing is pinned on slot vectors against a direct
convolution loop, which is itself pinned against a library convolution; the
weight plaintexts against their two-term closed form; and the whole layer
through BFV encryption, rotations by key switching and decryption against the
plain convolution mod P."""
import numpy as np
import pytest

from oracle import bfv, core, zp
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, Stream

N = 4096
L = 2
P = zp.plaintext_prime(N, 17)
KP = zp.KsParams(N, tuple(CANONICAL_PRIMES[:L]), CANONICAL_PRIMES[L])

SHAPES = [  # (C, H, W, M, kh, kw, pad)
    (3, 5, 6, 3, 3, 3, 1),
    (2, 4, 4, 4, 1, 1, 0),
    (2, 5, 4, 1, 2, 3, 0),
    (4, 7, 3, 5, 3, 1, 1),
    (2, 3, 6, 3, 1, 3, 0),
]


def test_direct_convolution_against_a_library_convolution():
    torch = pytest.importorskip("torch")
    s = Stream(90, 0)
    x = s.below(50, 3 * 6 * 5).astype(np.int64).reshape(3, 6, 5)
    K = s.int8(4 * 3 * 9).astype(np.int64).reshape(4, 3, 3, 3)
    want = torch.nn.functional.conv2d(torch.from_numpy(x[None].astype(np.float64)),
                                      torch.from_numpy(K.astype(np.float64)), padding=1)[0].numpy()
    # every value is an exact small integer in float64; mod P afterwards
    assert np.array_equal(zp.conv2d_mod(x, K, 1, P), np.mod(want.astype(np.int64), P))


@pytest.mark.parametrize("shape", SHAPES)
def test_slot_packing_gives_the_convolution(shape):
    """sum_i rot^(delta_i)(sum_c x_c * w_{y,i,c}) on plain slot vectors equals the
    convolution mod P at every output slot, for odd M (a half-empty last output
    ciphertext), 1x1, rectangular and one-column kernels."""
    C, H, W, M, kh, kw, pad = shape
    sh = zp.ConvShape(C, H, W, M, kh, kw, pad, N)
    assert sh.fits()
    s = Stream(91, sum(shape))
    x = s.below(P, C * H * W).astype(np.int64).reshape(C, H, W)
    K = s.below(P, M * C * kh * kw).astype(np.int64).reshape(M, C, kh, kw)
    got = zp.conv_output(zp.slot_conv(zp.conv_input_slots(x, sh, P), zp.conv_weight_slots(K, sh, P), sh, P), sh)
    assert np.array_equal(got, zp.conv2d_mod(x, K, pad, P))
    # the rotation steps are 1 within a kernel row and Wp - kw + 1 to the next row
    assert set(sh.steps) <= {1, sh.Wp - kw + 1}
    assert sum(sh.steps) == sh.offsets[-1]


def test_weight_plaintexts_have_the_two_term_closed_form():
    """A slot vector constant a in row 0 and b in row 1 encodes to alpha + beta X^(N/2)
    with alpha = (a + b)/2 and beta = (a - b)/(2 iota), iota = zeta^(N/2) (X^(N/2) has
    slot value iota in row 0 and -iota in row 1)."""
    zeta = core.min_psi(P, N)
    iota = pow(zeta, N // 2, P)
    inv2 = pow(2, -1, P)
    for a, b in ((3, 3), (5, P - 7), (0, 11), (P - 1, 1)):
        m = np.zeros((2, N // 2), dtype=np.int64)
        m[0], m[1] = a, b
        p = zp.encode(m, N, P)
        want = np.zeros(N, dtype=np.uint64)
        want[0] = (a + b) * inv2 % P
        want[N // 2] = (a - b) * inv2 * pow(iota, -1, P) % P
        assert np.array_equal(p, want), (a, b)
        assert np.array_equal(zp.decode(p, N, P), m)


def _keygen(s, sk, steps):
    keys = {}
    for st in sorted(set(steps)):
        a = np.stack([np.stack([s.below(q, N) for q in KP.qp]) for _ in range(L)])
        e = np.stack([s.rounded_gaussian(N) for _ in range(L)])
        keys[st] = zp.galois_key(KP, sk, zp.galois_step(st, N), a, e)
    return keys


@pytest.mark.parametrize("shape", [(2, 4, 4, 2, 3, 3, 1), (3, 3, 5, 3, 2, 2, 0)])
def test_convolution_through_encryption(shape):
    """Encrypt the packed input channels, run the layer on ciphertexts (products,
    key-switched rotations by 1 and by Wp - kw + 1), decrypt and decode: the output
    slots equal the plain convolution mod P."""
    C, H, W, M, kh, kw, pad = shape
    sh = zp.ConvShape(C, H, W, M, kh, kw, pad, N)
    s = Stream(92, sum(shape))
    sk = s.ternary(N)
    params = zp.bfv_params(N, KP.moduli, P)
    x = s.below(P, C * H * W).astype(np.int64).reshape(C, H, W)
    K = s.below(P, M * C * kh * kw).astype(np.int64).reshape(M, C, kh, kw)
    cts = []
    for xs in zp.conv_input_slots(x, sh, P):
        a = np.stack([s.below(q, N) for q in KP.moduli])
        cts.append(bfv.encrypt(params, sk, zp.encode(xs, N, P), a, s.rounded_gaussian(N)))
    ws = zp.conv_weight_slots(K, sh, P)
    w_polys = [[[zp.encode(ws[y, i, c], N, P) for c in range(C)] for i in range(kh * kw)] for y in range(sh.Y)]
    keys = _keygen(s, sk, sh.steps)
    out = zp.conv_mac_rotate(np.stack(cts), w_polys, keys, sh, KP, P)
    dec = [zp.decode(bfv.decrypt_at(params, sk, out[y], list(range(N))).astype(np.uint64), N, P) for y in range(sh.Y)]
    assert np.array_equal(zp.conv_output(dec, sh), zp.conv2d_mod(x, K, pad, P))
