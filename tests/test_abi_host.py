"""Host-only checks of libhconv: it loads, exports every symbol include/*.h
declares, validates context parameters without touching a GPU, and resolves
the same canonical convolution partition as the oracle."""
import glob
import os
import re

import pytest

from oracle import conv
from paper_2506_11586_gb300 import _lib as L
from paper_2506_11586_gb300.build import build
from paper_2506_11586_gb300.inputs import (CANONICAL_PRIMES, CONV_56x56x64, RESNET50_STRIDE1, SQUEEZENET_1_1,
                                           T_PLAIN, Stream)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build()


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w ]*?[\s*]+(hc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol():
    names = _declared_symbols()
    assert "hc_conv_ct_pt" in names and "hc_ntt_fwd" in names and len(names) >= 15
    lib = L.lib()
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_status_strings():
    for code, name in L.STATUS_NAMES.items():
        assert L.hc_status_str(code) == name


def test_ctx_validate():
    q = CANONICAL_PRIMES
    assert L.hc_ctx_validate(8192, q[:3], T_PLAIN) == L.HC_OK
    assert L.hc_ctx_validate(16384, q[:4], T_PLAIN) == L.HC_OK
    assert L.hc_ctx_validate(4096, q[:1], 2) == L.HC_OK
    assert L.hc_ctx_validate(2048, q[:2], T_PLAIN) == L.HC_ERR_INVALID_ARG      # unsupported N
    assert L.hc_ctx_validate(8192, [], T_PLAIN) == L.HC_ERR_INVALID_ARG         # L = 0
    assert L.hc_ctx_validate(8192, list(q) + list(q)[:3], T_PLAIN) == L.HC_ERR_INVALID_ARG  # L = 9
    assert L.hc_ctx_validate(8192, q[:2], 1) == L.HC_ERR_INVALID_ARG            # t < 2
    assert L.hc_ctx_validate(8192, [q[0], q[0]], T_PLAIN) == L.HC_ERR_BAD_MODULUS  # duplicate
    assert "duplicates" in L.hc_last_error()
    big = (1 << 50) + 1 + 0  # >= 2^50
    assert L.hc_ctx_validate(8192, [big], T_PLAIN) == L.HC_ERR_BAD_MODULUS
    assert L.hc_ctx_validate(8192, [q[0] + 2 * 16384], T_PLAIN) in (L.HC_OK, L.HC_ERR_BAD_MODULUS)
    comp = q[0] + 2 * 16384 * 3  # = 1 mod 2N; composite or prime, decided below
    import sympy
    assert (L.hc_ctx_validate(8192, [comp], T_PLAIN) == L.HC_OK) == sympy.isprime(comp)
    assert L.hc_ctx_validate(8192, [97], T_PLAIN) == L.HC_ERR_BAD_MODULUS       # not 1 mod 2N
    assert L.hc_ctx_validate(4096, [40961], T_PLAIN) == L.HC_ERR_BAD_MODULUS    # prime, = 1 mod 2N, < 2^32
    assert L.hc_ctx_validate(8192, [1 + 16384 * 5], T_PLAIN) == L.HC_ERR_BAD_MODULUS  # 81921 = 3 * 27307


def test_ctx_validate_matches_sympy_on_candidates():
    import sympy
    N = 4096
    s = Stream(31, 0)
    for k in s.below(1 << 36, 300):
        cand = int(k) * 2 * N + 1
        if cand >= (1 << 50):
            continue
        want = L.HC_OK if (sympy.isprime(cand) and cand > (1 << 32)) else L.HC_ERR_BAD_MODULUS
        assert L.hc_ctx_validate(N, [cand], T_PLAIN) == want, cand


def _lib_partition(sh, N):
    d = L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad)
    res, i, p, o = L.hc_conv_partition(d, N)
    return (res.Cw, res.Hw, res.Ww, i, p, o)


def _oracle_partition(sh, N):
    p = conv.canonical_partition(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, sh.pad, N)
    return (p.Cw, p.Hw, p.Ww, p.I, p.P, p.O)


def test_partition_parity_squeezenet_and_conv():
    for sh in list(SQUEEZENET_1_1) + [CONV_56x56x64]:
        assert _lib_partition(sh, 8192) == _oracle_partition(sh, 8192), sh.name


def test_partition_parity_resnet():
    for sh in RESNET50_STRIDE1[:6]:
        assert _lib_partition(sh, 16384) == _oracle_partition(sh, 16384), sh.name


def test_partition_parity_random_shapes():
    from paper_2506_11586_gb300.inputs import ConvShape
    s = Stream(17, 0)
    for i in range(25):
        C_, H, W, M = (int(v) for v in (s.below(40, 1)[0] + 1, s.below(20, 1)[0] + 3,
                                         s.below(20, 1)[0] + 3, s.below(9, 1)[0] + 1))
        k = int(s.below(3, 1)[0])
        kh = kw = (1, 3, 5)[k]
        pad = kh // 2 if int(s.below(2, 1)[0]) else 0
        if kh > H + 2 * pad or kw > W + 2 * pad:
            continue
        sh = ConvShape("r%d" % i, C_, H, W, M, kh, kw, pad)
        N = (4096, 8192)[i % 2]
        assert _lib_partition(sh, N) == _oracle_partition(sh, N), sh


def test_partition_errors():
    d = L.make_desc(8, 8, 8, 4, 3, 3, pad=1, stride=0)
    with pytest.raises(L.HcError) as e:
        L.hc_conv_partition(d, 4096)
    assert e.value.status == L.HC_ERR_INVALID_ARG
    d = L.make_desc(8, 8, 8, 4, 3, 3, pad=1, Cw=8, Hw=30, Ww=30)   # 8*30*30 > 4096
    with pytest.raises(L.HcError) as e:
        L.hc_conv_partition(d, 4096)
    assert e.value.status == L.HC_ERR_INVALID_ARG
    d = L.make_desc(8, 2, 2, 4, 3, 3, pad=0)                       # kernel larger than input
    with pytest.raises(L.HcError):
        L.hc_conv_partition(d, 4096)
    d = L.make_desc(8, 8, 8, 4, 3, 3, pad=1, Cw=4, Hw=6, Ww=6)     # explicit, valid
    res, i, p, o = L.hc_conv_partition(d, 4096)
    op = conv.Partition(8, 8, 8, 4, 3, 3, 1, 4096, 4, 6, 6)
    assert (res.Cw, res.Hw, res.Ww, i, p, o) == (4, 6, 6, op.I, op.P, op.O)


STRIDED = [  # (C, H, W, M, kh, kw, stride, pad, N): the networks' strided layers and odd cases
    (3, 224, 224, 64, 3, 3, 2, 0, 8192),      # SqueezeNet-1.1 conv1
    (3, 224, 224, 64, 7, 7, 2, 3, 16384),     # ResNet-50 conv1
    (128, 56, 56, 128, 3, 3, 2, 1, 16384),    # ResNet-50 layer2 downsampling 3x3
    (256, 56, 56, 512, 1, 1, 2, 0, 16384),    # ResNet-50 layer2 projection 1x1
    (5, 13, 11, 3, 4, 2, 3, 1, 4096),
    (2, 9, 9, 2, 2, 3, 2, 2, 4096),
]


def test_strided_partition_parity():
    from oracle import layers
    for C_, H, W, M, kh, kw, st, pad, N in STRIDED:
        res, i, p, o = L.hc_conv_partition(L.make_desc(C_, H, W, M, kh, kw, pad=pad, stride=st), N)
        ph, op = layers.strided_partition(C_, H, W, M, kh, kw, st, pad, N)
        assert (res.C, res.H, res.W, res.M, res.kh, res.kw, res.stride, res.pad) == \
            (ph.C1, ph.H1, ph.W1, M, ph.kh1, ph.kw1, 1, 0)
        assert (res.Cw, res.Hw, res.Ww, i, p, o) == (op.Cw, op.Hw, op.Ww, op.I, op.P, op.O)
    # stride 1 is left as given
    res, *_ = L.hc_conv_partition(L.make_desc(4, 9, 9, 2, 3, 3, pad=1), 4096)
    assert (res.C, res.H, res.pad, res.stride) == (4, 9, 1, 1)


def test_fc_partition_parity():
    from oracle import layers
    s = Stream(18, 0)
    cases = [(2048, 1000, 16384), (2048, 1000, 8192), (512, 10, 4096), (4096, 4096, 8192)]
    for _ in range(12):
        cases.append((int(s.below(3000, 1)[0]) + 1, int(s.below(300, 1)[0]) + 1, (1024, 4096)[int(s.below(2, 1)[0])]))
    for C_, M, N in cases:
        res, i, p, o = L.hc_fc_partition(L.make_fc_desc(C_, M), N)
        fp = layers.canonical_fc_partition(C_, M, N)
        assert (res.Cw, res.No, i, p, o) == (fp.Cw, fp.No, fp.I, fp.P, fp.O), (C_, M, N)
    res, i, p, o = L.hc_fc_partition(L.make_fc_desc(45, 23, Cw=20, No=9), 256)
    assert (res.Cw, res.No, i, p, o) == (20, 9, 3, 9, 3)


def test_fc_partition_errors():
    for d, N in ((L.make_fc_desc(0, 5), 4096), (L.make_fc_desc(10, 5, Cw=11, No=1), 4096),
                 (L.make_fc_desc(10, 5, Cw=10, No=6), 4096), (L.make_fc_desc(100, 50, Cw=100, No=50), 4096),
                 (L.make_fc_desc(10, 5, Cw=10, No=0), 4096)):
        with pytest.raises(L.HcError) as e:
            L.hc_fc_partition(d, N)
        assert e.value.status == L.HC_ERR_INVALID_ARG
