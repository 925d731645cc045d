"""Pins of the oracle's server step around the convolution (Sec. 7: the server
adds its activation share to the client's ciphertexts, runs the convolution
with NTT-preprocessed weights and applies a random mask; Sec. 6.2: only the
output coefficients go back).  Pinned end to end through BFV: the client's
decryption of every returned slot equals conv(x_c + x_s) - r mod t, computed
by the plaintext convolution."""
import numpy as np

from oracle import bfv, conv
from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream


def _setup(C_, H, W, M, kh, kw, pad, N, nl, seed, part=None):
    s = Stream(seed, 31)
    p = conv.Partition(C_, H, W, M, kh, kw, pad, N, *part) if part else \
        conv.canonical_partition(C_, H, W, M, kh, kw, pad, N)
    params = bfv.Params(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    sk = s.ternary(N)
    x_c = s.below(T_PLAIN, C_ * H * W).astype(np.int64).reshape(C_, H, W)
    x_s = s.below(T_PLAIN, C_ * H * W).astype(np.int64).reshape(C_, H, W)
    K = s.int8(M * C_ * kh * kw).astype(np.int64).reshape(M, C_, kh, kw)
    r = s.below(T_PLAIN, M * p.Ho * p.Wo).astype(np.int64).reshape(M, p.Ho, p.Wo)
    packed = conv.pack_input(x_c, p)
    ct = np.zeros((p.I, 2, nl, N), dtype=np.uint64)
    for i in range(p.I):
        a = np.stack([s.below(q, N) for q in params.moduli])
        ct[i] = bfv.encrypt(params, sk, packed[i], a, s.rounded_gaussian(N))
    return p, params, sk, x_c, x_s, K, r, ct


def test_delta_residues_match_bfv_scale():
    for nl in (1, 2, 3, 4):
        params = bfv.Params(4096, CANONICAL_PRIMES[:nl], T_PLAIN)
        assert conv.delta_residues(params.moduli, T_PLAIN) == [params.delta % q for q in params.moduli]


def test_share_add_adds_the_share_to_the_plaintext():
    p, params, sk, x_c, x_s, K, r, ct = _setup(5, 7, 6, 3, 3, 3, 1, 4096, 2, 1)
    ct1 = conv.share_add(ct, x_s, p, params.moduli, T_PLAIN)
    assert np.array_equal(ct1[:, 1], ct[:, 1])                   # c1 untouched
    want = conv.pack_input((x_c + x_s) % T_PLAIN, p)
    ks = np.arange(p.Cw * p.Hw * p.Ww)
    for i in range(p.I):
        assert np.array_equal(bfv.decrypt_at(params, sk, ct1[i], ks), want[i][ks] % T_PLAIN)


def test_server_step_decrypts_to_masked_convolution():
    # explicit partition Cw = 3, Hw = 6, Ww = 5: two channel groups (one ragged)
    # and 2 x 2 spatial blocks whose last row of blocks is ragged
    p, params, sk, x_c, x_s, K, r, ct = _setup(5, 7, 6, 3, 3, 3, 1, 4096, 2, 2, part=(3, 6, 5))
    assert (p.G, p.Bh, p.Bw) == (2, 2, 2) and p.Ho % p.oh != 0
    ct1 = conv.share_add(ct, x_s, p, params.moduli, T_PLAIN)
    out = conv.conv_ct_pt(ct1, conv.pack_weights(K, p), p, params.moduli)
    slots = conv.extract_masked(out, r, p, params.moduli, T_PLAIN)
    assert slots.shape == (p.O, 2, conv.slot_count(p))
    y = conv.conv2d_mod_t((x_c + x_s) % T_PLAIN, K, p.pad, T_PLAIN)
    checked = 0
    for m in range(p.M):
        for b in range(p.B):
            o = m * p.B + b
            for k, row, col in conv.output_slots(p, b):
                rel = k - p.offset
                s_idx = (rel // p.Ww) * p.ow + rel % p.Ww
                c = out[o].copy()
                c[0, :, k] = slots[o, :, s_idx]                      # the returned c0 slot, with c1
                got = int(bfv.decrypt_at(params, sk, c, [k])[0])
                assert got == (int(y[m, row, col]) - int(r[m, row, col])) % T_PLAIN, (m, b, k)
                checked += 1
    assert checked == p.M * p.Ho * p.Wo
    # slots of edge blocks that fall outside the output map are zero
    n_zero_slots = 0
    for b in range(p.B):
        valid = {((k - p.offset) // p.Ww) * p.ow + (k - p.offset) % p.Ww for k, _, _ in conv.output_slots(p, b)}
        for s_idx in set(range(conv.slot_count(p))) - valid:
            assert not slots[b::p.B, :, s_idx].any()
            n_zero_slots += 1
    assert n_zero_slots > 0                                          # this shape has ragged edge blocks
