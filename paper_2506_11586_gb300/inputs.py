"""Seeded synthetic inputs and workload shapes for the HE-convolution hot path.

This module holds random-number generation, parameter constants and layer
shapes only -- none of the method's arithmetic.  It is the one module that
both the GPU library's tests/benchmark and the CPU oracle's tests draw inputs
from; neither side's arithmetic lives here.

Random numbers come from a counter-based splitmix64 generator (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", 2014): value i of a
stream is mix64(base + (i + 1) * 0x9E3779B97F4A7C15), so every draw is a pure
function of (seed, stream, counter) on any platform.

The paper (arXiv 2506.11586) evaluates on ImageNet with a trained 37-bit
SqueezeNet-1.1 / ResNet-50 (Sec. 8).  Neither dataset nor weights are used:
the hot path is exact modular arithmetic whose cost does not depend on the
values, so seeded uniform activations mod t = 2^37 and uniform int8 weights at
the paper's layer shapes stand in for them.
"""
from dataclasses import dataclass

import numpy as np

# Canonical RNS primes: the largest primes q < 2^50 with q = 1 (mod 2^15), in
# descending order.  q = 1 mod 2^15 makes every N <= 16384 NTT-friendly
# (q = 1 mod 2N), so mixed-N batches share them.  The paper fixes neither N
# nor Q; the oracle's tests re-derive this list.
CANONICAL_PRIMES = (
    1125899904679937,
    1125899903991809,
    1125899903827969,
    1125899903795201,
    1125899903500289,
    1125899903107073,
)

# Plaintext modulus: secret shares live in Z_{2^37} (Sec. 8: 37-bit fixed point).
T_PLAIN = 1 << 37

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based splitmix64 stream identified by (seed, stream id)."""

    def __init__(self, seed: int, stream: int = 0):
        with np.errstate(over="ignore"):
            s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GAMMA + np.uint64(stream & 0xFFFFFFFF)
        self.base = _mix64(np.array([s], dtype=np.uint64))[0]
        self.ctr = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.ctr + 1, self.ctr + 1 + n, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            return _mix64(self.base + idx * _GAMMA)

    def below(self, bound: int, n: int) -> np.ndarray:
        """n uniform integers in [0, bound), by rejection on the top bits."""
        bits = int(bound - 1).bit_length() if bound > 1 else 1
        out = np.empty(0, dtype=np.uint64)
        while out.size < n:
            need = n - out.size
            cand = self.u64(need + need // 2 + 16) >> np.uint64(64 - bits)
            out = np.concatenate([out, cand[cand < np.uint64(bound)]])
        return out[:n]

    def int8(self, n: int) -> np.ndarray:
        """n uniform values in {-128..127}."""
        return ((self.u64(n) >> np.uint64(56)).astype(np.int64) - 128).astype(np.int8)

    def ternary(self, n: int) -> np.ndarray:
        """n values uniform in {-1, 0, 1}."""
        v = self.below(3, n).astype(np.int64)
        return v - 1

    def rounded_gaussian(self, n: int, sigma: float = 3.2, tail: float = 6.0) -> np.ndarray:
        """n rounded zero-mean Gaussian integers (Box-Muller), |e| <= tail*sigma."""
        out = np.empty(0, dtype=np.int64)
        lim = int(np.floor(tail * sigma))
        while out.size < n:
            m = (n - out.size) + 16
            u1 = ((self.u64(m) >> np.uint64(11)).astype(np.float64) + 1.0) / 9007199254740992.0
            u2 = (self.u64(m) >> np.uint64(11)).astype(np.float64) / 9007199254740992.0
            z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2) * sigma
            e = np.rint(z).astype(np.int64)
            out = np.concatenate([out, e[np.abs(e) <= lim]])
        return out[:n]


def uniform_residues(stream: Stream, moduli, shape_before_limb, N) -> np.ndarray:
    """Array of shape (*shape_before_limb, L, N) with limb l uniform in [0, moduli[l])."""
    L = len(moduli)
    count = int(np.prod(shape_before_limb)) if len(shape_before_limb) else 1
    out = np.empty((count, L, N), dtype=np.uint64)
    for li, q in enumerate(moduli):
        out[:, li, :] = stream.below(q, count * N).reshape(count, N)
    return out.reshape(*shape_before_limb, L, N)


# ---- layer shapes -----------------------------------------------------------

@dataclass(frozen=True)
class ConvShape:
    """Stride-1 convolution: C input channels of H x W, M output channels, kh x kw kernel."""
    name: str
    C: int
    H: int
    W: int
    M: int
    kh: int
    kw: int
    pad: int


def _fire(idx, C, sq, e, hw):
    return [
        ConvShape(f"fire{idx}.squeeze", C, hw, hw, sq, 1, 1, 0),
        ConvShape(f"fire{idx}.expand1x1", sq, hw, hw, e, 1, 1, 0),
        ConvShape(f"fire{idx}.expand3x3", sq, hw, hw, e, 3, 3, 1),
    ]


# SqueezeNet-1.1 at a 224x224x3 input: every stride-1 convolution (all fire
# squeeze/expand convolutions and the final 1x1 classifier conv10).  conv1
# (3x3, stride 2) is not stride-1 and is not part of this list.
SQUEEZENET_1_1 = (
    _fire(2, 64, 16, 64, 55) + _fire(3, 128, 16, 64, 55)
    + _fire(4, 128, 32, 128, 27) + _fire(5, 256, 32, 128, 27)
    + _fire(6, 256, 48, 192, 13) + _fire(7, 384, 48, 192, 13)
    + _fire(8, 384, 64, 256, 13) + _fire(9, 512, 64, 256, 13)
    + [ConvShape("conv10", 512, 13, 13, 1000, 1, 1, 0)]
)

# Distinct stride-1 3x3 / 1x1 convolutions of ResNet-50 (v1.5 layout) at a
# 224x224 input.
RESNET50_STRIDE1 = (
    ConvShape("res2.conv1_in64", 64, 56, 56, 64, 1, 1, 0),
    ConvShape("res2.conv2", 64, 56, 56, 64, 3, 3, 1),
    ConvShape("res2.conv3", 64, 56, 56, 256, 1, 1, 0),
    ConvShape("res2.conv1", 256, 56, 56, 64, 1, 1, 0),
    ConvShape("res3.conv1_in256", 256, 56, 56, 128, 1, 1, 0),
    ConvShape("res3.conv2", 128, 28, 28, 128, 3, 3, 1),
    ConvShape("res3.conv3", 128, 28, 28, 512, 1, 1, 0),
    ConvShape("res3.conv1", 512, 28, 28, 128, 1, 1, 0),
    ConvShape("res4.conv1_in512", 512, 28, 28, 256, 1, 1, 0),
    ConvShape("res4.conv2", 256, 14, 14, 256, 3, 3, 1),
    ConvShape("res4.conv3", 256, 14, 14, 1024, 1, 1, 0),
    ConvShape("res4.conv1", 1024, 14, 14, 256, 1, 1, 0),
    ConvShape("res5.conv1_in1024", 1024, 14, 14, 512, 1, 1, 0),
    ConvShape("res5.conv2", 512, 7, 7, 512, 3, 3, 1),
    ConvShape("res5.conv3", 512, 7, 7, 2048, 1, 1, 0),
    ConvShape("res5.conv1", 2048, 7, 7, 512, 1, 1, 0),
)

@dataclass(frozen=True)
class StridedShape:
    """Convolution with stride: C input channels of H x W, M output channels,
    kh x kw kernel, zero padding pad on every side."""
    name: str
    C: int
    H: int
    W: int
    M: int
    kh: int
    kw: int
    stride: int
    pad: int


# SqueezeNet-1.1's first convolution (3x3, stride 2, no padding, 224 -> 111).
SQUEEZENET_CONV1 = StridedShape("conv1", 3, 224, 224, 64, 3, 3, 2, 0)

# The strided convolutions of ResNet-50 (v1.5 layout: the stride sits on the
# 3x3 convolution of each stage's first block, and the projection shortcut of
# stages 3-5 is a 1x1 stride-2 convolution), at a 224x224 input.
RESNET50_STRIDED = (
    StridedShape("conv1", 3, 224, 224, 64, 7, 7, 2, 3),
    StridedShape("res3.conv2_s2", 128, 56, 56, 128, 3, 3, 2, 1),
    StridedShape("res3.proj", 256, 56, 56, 512, 1, 1, 2, 0),
    StridedShape("res4.conv2_s2", 256, 28, 28, 256, 3, 3, 2, 1),
    StridedShape("res4.proj", 512, 28, 28, 1024, 1, 1, 2, 0),
    StridedShape("res5.conv2_s2", 512, 14, 14, 512, 3, 3, 2, 1),
    StridedShape("res5.proj", 1024, 14, 14, 2048, 1, 1, 2, 0),
)

# ResNet-50's fully connected classifier: 2048 inputs, 1000 outputs.
RESNET50_FC = (2048, 1000)

# The single-layer benchmark workload: 56x56x64 activations, 3x3 weights,
# 64 output channels, stride 1, pad 1, N = 8192 with three 50-bit primes.
CONV_56x56x64 = ConvShape("conv3x3_56x56x64_to64", 64, 56, 56, 64, 3, 3, 1)


def conv_tensors(shape: ConvShape, seed: int):
    """Seeded activations x ~ U[0, 2^37)^(C,H,W) and weights K ~ U{-128..127}^(M,C,kh,kw)."""
    s = Stream(seed, 1)
    x = s.below(T_PLAIN, shape.C * shape.H * shape.W).astype(np.int64)
    x = x.reshape(shape.C, shape.H, shape.W)
    K = s.int8(shape.M * shape.C * shape.kh * shape.kw).reshape(shape.M, shape.C, shape.kh, shape.kw)
    return x, K


# ---- uneven ct x pt batch ------------------------------------------------------

# (N, L) classes and their shares of the mixed batch: 40 % / 40 % / 20 %.
UNEVEN_CLASSES = ((4096, 2, 0.4), (8192, 3, 0.4), (16384, 4, 0.2))


def uneven_mix(n_products: int, seed: int):
    """Seeded shuffle of class labels (0, 1, 2) in the 40/40/20 proportions."""
    counts = [int(round(n_products * f)) for (_, _, f) in UNEVEN_CLASSES]
    counts[-1] = n_products - sum(counts[:-1])
    labels = np.concatenate([np.full(c, i, dtype=np.int64) for i, c in enumerate(counts)])
    keys = Stream(seed, 7).u64(n_products)
    return labels[np.argsort(keys, kind="stable")]


# ---- serving workload ------------------------------------------------------------

# How many times each distinct stride-1 ResNet-50 (v1.5) convolution shape
# occurs in the network (the 3x3 stride-2 convolutions and stride-2
# projection shortcuts of the first block of stages 3-5 are not stride-1; the
# stride-1 projection shortcut 64 -> 256 of stage 2 has res2.conv3's shape).
# Each occurrence has its own weights: about 47 GB of NTT-domain weights at
# N = 16384 with four 50-bit primes.
RESNET50_MULTIPLICITY = {
    "res2.conv1_in64": 1, "res2.conv2": 3, "res2.conv3": 4, "res2.conv1": 2,
    "res3.conv1_in256": 1, "res3.conv2": 3, "res3.conv3": 4, "res3.conv1": 3,
    "res4.conv1_in512": 1, "res4.conv2": 5, "res4.conv3": 6, "res4.conv1": 5,
    "res5.conv1_in1024": 1, "res5.conv2": 2, "res5.conv3": 3, "res5.conv1": 2,
}


def resnet50_instances():
    """Every stride-1 convolution instance of ResNet-50: list of (ConvShape, occurrence)."""
    return [(sh, k) for sh in RESNET50_STRIDE1 for k in range(RESNET50_MULTIPLICITY[sh.name])]


@dataclass(frozen=True)
class ServingTrace:
    """Request arrivals: times in seconds from the start, and for each request
    its family (0 = SqueezeNet-1.1 at N = 8192, 1 = ResNet-50 at N = 16384)
    and its layer index within that family."""
    t: np.ndarray
    family: np.ndarray
    layer: np.ndarray


def serving_trace(n_requests: int, rate: float, seed: int, n_layers=None) -> ServingTrace:
    """Poisson arrivals at `rate` requests/s (exponential gaps by inversion),
    each request a fair coin between the two families and then a uniform
    layer of that family."""
    if n_layers is None:
        n_layers = (len(SQUEEZENET_1_1), len(resnet50_instances()))
    s = Stream(seed, 11)
    u = (s.u64(n_requests) >> np.uint64(11)).astype(np.float64) / 9007199254740992.0
    t = np.cumsum(-np.log1p(-u) / rate)
    fam = (s.u64(n_requests) >> np.uint64(63)).astype(np.int64)
    r = (s.u64(n_requests) >> np.uint64(11)).astype(np.float64) / 9007199254740992.0
    sizes = np.where(fam == 0, n_layers[0], n_layers[1])
    layer = np.minimum((r * sizes).astype(np.int64), sizes - 1)
    return ServingTrace(t, fam, layer)
