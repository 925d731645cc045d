"""Host-side accounting of bench.py (no GPU): the algorithmic bytes and
integer-pipe work it divides by, and the plaintext prime of its Z_P section,
against independent statements of the same quantities."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from oracle import core, zp  # noqa: E402


def test_layer_bytes_and_integer_work():
    # the 56x56x64 layer: I = 32, P = 512, O = 256, 2048 products, N = 8192, L = 3
    geo = dict(I=32, P=512, O=256, products=2048)
    N, L = 8192, 3
    assert bench.alg_bytes(geo, N, L) == 8 * N * L * (2 * 32 + 512 + 2 * 256) == 213909504
    bfly = 4096 * 13                                  # (N/2) log2 N butterflies per limb
    fwd = 2 * 32 * L * bfly * 14
    mac = 2048 * 2 * L * N * 8 + 256 * 2 * L * N * 19
    inv = 2 * 256 * L * bfly * 14
    assert bench.conv_imad_eq(32, 256, 2048, N, L) == fwd + mac + inv
    assert bench.kernel_work("k_ntt_inv/N8192", geo, N, L) == {"bytes": 2 * 8 * N * L * 2 * 256, "imad_eq": inv}
    assert bench.kernel_work("k_ntt_fwd/N8192", geo, N, L)["imad_eq"] == fwd
    assert bench.kernel_work("k_mac_conv", geo, N, L)["imad_eq"] == mac
    # one standalone product: NTT and INTT of both components plus the pointwise product
    assert bench.product_imad_eq(4096, 2) == 2 * 2 * (2 * 2048 * 12 * 14 + 4096 * 14)


def test_roofline_fractions():
    r = bench.roofline_fracs(213909504, 2.3325e9, 0.25)
    peak, _ = bench.measured_peaks()
    assert r["hbm_frac"] == pytest.approx(213909504 / 0.25e-3 / 1e9 / peak)
    assert r["alu_frac"] == pytest.approx(2.3325e9 / 0.25e-3 / 1e12 / bench.alu_peak_imad_eq())
    assert r["bound"] == ("alu" if r["alu_frac"] >= r["hbm_frac"] else "hbm")


@pytest.mark.parametrize("N", [4096, 8192, 16384])
def test_zp_plain_prime_matches_the_oracle(N):
    P = bench.zp_plain_prime(N)
    assert P == zp.plaintext_prime(N, 37)
    assert core.is_prime(P) and P % (2 * N) == 1 and (1 << 36) < P < (1 << 37)
