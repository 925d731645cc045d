"""GPU parity of the Z_P convolution layer (hc_zp_conv_preprocess, hc_zp_conv:
SecONNds-P's convolutions over Z_P^N as the multiply-accumulate-rotate
iteration, Sec. 6.1 and Sec. 2.3): the resident weight plaintexts equal the
oracle's encodings lifted and transformed, every residue of every output
ciphertext equals the oracle's layer (oracle/zp.py) on the same BFV
ciphertexts and Galois keys, and the outputs decrypt to the convolution mod P,
up to a full SqueezeNet-1.1 layer (fire2 expand 3x3, 16 -> 64 channels at
55 x 55) at N = 8192 with a 37-bit P."""
import numpy as np
import pytest

from gpu_util import to_dev, to_host
from oracle import bfv, core, zp
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, Stream

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_11586_gb300 import _lib
    from paper_2506_11586_gb300.build import build
    build()
    return _lib


class Layer:
    """Keys, encrypted packed inputs and the library's handles for one Z_P convolution."""

    def __init__(self, L, shape, N, nl, pbits, seed, x=None, K=None):
        C, H, W, M, kh, kw, pad = shape
        self.sh = zp.ConvShape(C, H, W, M, kh, kw, pad, N)
        assert self.sh.fits()
        self.kp = zp.KsParams(N, tuple(CANONICAL_PRIMES[:nl]), CANONICAL_PRIMES[nl])
        self.P = P = zp.plaintext_prime(N, pbits)
        s = Stream(seed, 0)
        self.sk = s.ternary(N)
        self.params = zp.bfv_params(N, self.kp.moduli, P)
        self.x = x if x is not None else s.below(P, C * H * W).astype(np.int64).reshape(C, H, W)
        self.K = K if K is not None else s.below(P, M * C * kh * kw).astype(np.int64).reshape(M, C, kh, kw)
        self.cts = []
        for xs in zp.conv_input_slots(self.x, self.sh, P):
            a = np.stack([s.below(q, N) for q in self.kp.moduli])
            self.cts.append(bfv.encrypt(self.params, self.sk, zp.encode(xs, N, P), a, s.rounded_gaussian(N)))
        self.cts = np.stack(self.cts)
        self.gks = {}
        for st in sorted(set(self.sh.steps)):
            a = np.stack([np.stack([s.below(q, N) for q in self.kp.qp]) for _ in range(nl)])
            e = np.stack([s.rounded_gaussian(N) for _ in range(nl)])
            self.gks[st] = zp.galois_key(self.kp, self.sk, zp.galois_step(st, N), a, e)
        self.ctx = L.hc_ctx_create(N, self.kp.moduli, P)
        self.ctx_p = L.hc_ctx_create(N, [P], P)
        self.desc = L.make_desc(C, H, W, M, kh, kw, pad=pad)
        self.key_1 = (L.hc_galois_key_create(self.ctx, self.kp.special, 5, self.gks[1])
                      if kw > 1 else None)
        srow = self.sh.Wp - kw + 1
        self.key_row = (L.hc_galois_key_create(self.ctx, self.kp.special, zp.galois_step(srow, N), self.gks[srow])
                        if kh > 1 else None)
        self.n_plain = self.sh.Y * kh * kw * C
        self.w = torch.empty(self.n_plain * nl * N, dtype=torch.int64, device="cuda")
        L.hc_zp_conv_preprocess(self.ctx, self.ctx_p, self.desc, self.K % P, self.w)

    def run(self, L):
        sh, nl = self.sh, self.kp.L
        out = torch.full((sh.Y * 2 * nl * sh.N,), -1, dtype=torch.int64, device="cuda")
        L.hc_zp_conv(self.ctx, self.desc, self.key_1, self.key_row, self.w, to_dev(self.cts), out)
        L.hc_ctx_device_status(self.ctx)
        return to_host(out).reshape(sh.Y, 2, nl, sh.N)

    def decrypt(self, out):
        N = self.sh.N
        dec = [zp.decode(bfv.decrypt_at(self.params, self.sk, out[y], list(range(N))).astype(np.uint64), N, self.P)
               for y in range(self.sh.Y)]
        return zp.conv_output(dec, self.sh)

    def oracle(self):
        sh, P = self.sh, self.P
        ws = zp.conv_weight_slots(self.K, sh, P)
        w_polys = [[[zp.encode(ws[y, i, c], sh.N, P) for c in range(sh.C)] for i in range(sh.kh * sh.kw)]
                   for y in range(sh.Y)]
        return zp.conv_mac_rotate(self.cts, w_polys, self.gks, sh, self.kp, P)


# N = 4096 with three 50-bit primes: a 37-bit P needs Q of about 2^150 (the plaintext
# product's term (Q mod P) * floor(m w / P) reaches about 2^75)
SMALL = [  # (C, H, W, M, kh, kw, pad)
    (3, 5, 6, 3, 3, 3, 1),
    (2, 4, 4, 4, 1, 1, 0),
    (2, 5, 4, 1, 2, 3, 0),
    (4, 7, 3, 5, 3, 1, 1),
    (2, 3, 6, 3, 1, 3, 0),
]


@pytest.mark.parametrize("shape", SMALL)
def test_zp_conv_matches_oracle_and_decrypts(L, shape):
    ly = Layer(L, shape, 4096, 3, 37, 300 + sum(shape))
    got = ly.run(L)
    assert np.array_equal(got, ly.oracle())                     # every residue of every output
    assert np.array_equal(ly.decrypt(got), zp.conv2d_mod(ly.x, ly.K, shape[6], ly.P))


def test_zp_conv_weight_plaintexts_match_oracle(L):
    """Resident weights: plaintext (y, i, c) is NTT(centered lift(encode(w_{y,i,c}))) per limb."""
    ly = Layer(L, (3, 5, 6, 3, 3, 3, 1), 4096, 3, 37, 310)
    sh, kp, P, N = ly.sh, ly.kp, ly.P, 4096
    ws = zp.conv_weight_slots(ly.K, sh, P)
    got = to_host(ly.w).reshape(sh.Y, sh.kh * sh.kw, sh.C, kp.L, N)
    for (y, i, c) in ((0, 0, 0), (1, 8, 2), (0, 4, 1)):
        lift = zp.lift_plain(zp.encode(ws[y, i, c], N, P), P, kp.moduli)
        for li, q in enumerate(kp.moduli):
            assert np.array_equal(got[y, i, c, li], core.ntt(lift[li], q, core.min_psi(q, N))), (y, i, c, li)


def test_zp_conv_squeezenet_fire_shape_bit_exact(L):
    """A 13 x 13, 3 x 3, pad 1 layer (the shape of SqueezeNet-1.1's fire6-fire9 expand
    convolutions, fewer channels) at N = 8192, three 50-bit primes, 37-bit P."""
    shape = (4, 13, 13, 2, 3, 3, 1)
    ly = Layer(L, shape, 8192, 3, 37, 320)
    got = ly.run(L)
    assert np.array_equal(got, ly.oracle())
    assert np.array_equal(ly.decrypt(got), zp.conv2d_mod(ly.x, ly.K, 1, ly.P))


def test_zp_conv_fire2_expand3x3_decrypts(L):
    """SqueezeNet-1.1's fire2 expand 3 x 3 layer in full (16 -> 64 channels, 55 x 55, pad 1)
    at N = 8192 with a 37-bit P: int8 weights, activations below 2^20, every output pixel
    of the 64 channels decrypts to the convolution mod P (the exact integer convolution is
    below 2^53, so torch's float64 conv2d on the CPU computes it exactly)."""
    s = Stream(330, 1)
    x = s.below(1 << 20, 16 * 55 * 55).astype(np.int64).reshape(16, 55, 55)
    K = s.int8(64 * 16 * 9).astype(np.int64).reshape(64, 16, 3, 3)
    ly = Layer(L, (16, 55, 55, 64, 3, 3, 1), 8192, 3, 37, 331, x=x, K=K)
    got = ly.run(L)
    want = torch.nn.functional.conv2d(torch.from_numpy(x[None].astype(np.float64)),
                                      torch.from_numpy(K.astype(np.float64)), padding=1)[0].numpy()
    assert np.array_equal(ly.decrypt(got), np.mod(want.astype(np.int64), ly.P))


def test_zp_conv_rejects_bad_arguments(L):
    ly = Layer(L, (2, 4, 4, 2, 3, 3, 1), 4096, 3, 37, 340)
    out = torch.empty(ly.sh.Y * 2 * ly.kp.L * 4096, dtype=torch.int64, device="cuda")
    with pytest.raises(L.HcError) as e:          # the keys swapped
        L.hc_zp_conv(ly.ctx, ly.desc, ly.key_row, ly.key_1, ly.w, to_dev(ly.cts), out)
    assert e.value.status == L.HC_ERR_INVALID_ARG
    big = L.make_desc(2, 60, 60, 2, 3, 3, pad=1)  # 62 x 62 slots do not fit one row of 2048
    with pytest.raises(L.HcError) as e:
        L.hc_zp_conv(ly.ctx, big, ly.key_1, ly.key_row, ly.w, to_dev(ly.cts), out)
    assert e.value.status == L.HC_ERR_INVALID_ARG
    strided = L.make_desc(2, 4, 4, 2, 3, 3, pad=1, stride=2)
    with pytest.raises(L.HcError) as e:
        L.hc_zp_conv(ly.ctx, strided, ly.key_1, ly.key_row, ly.w, to_dev(ly.cts), out)
    assert e.value.status == L.HC_ERR_UNSUPPORTED
