// hc_direct.cu -- the convolution without NTT preprocessing (the "no NTT" form
// the paper lists beside offline and online NTT preprocessing, Sec. 9):
// every output ciphertext component is computed directly in the coefficient
// domain as the negacyclic product sum
//   y(m',b)[k] = sum_r sum_g sum_{c,l,l'} K[m'*No+r, g*Cw+c, l, l'] * x(g,b)[k - pos]   (mod q),
// pos = r*Cw*Hw*Ww + offset - c*Hw*Ww - l*Ww - l' the coefficient of that
// weight in the packed weight polynomial (No output channels per output
// polynomial; 1 for convolutions), a term whose index wraps below 0 taking x[k - pos + N]
// with the opposite sign (X^N = -1, Sec. 2.1).  Weights stay small signed
// integers; nothing is transformed.  Cost grows with N * C*kh*kw per output
// coefficient instead of log N: a comparison form, not the fast path.
#include "hc_arith.cuh"
#include "hc_internal.h"

namespace hc {
namespace {

struct DirectGeom {
    uint32_t C, Cw, Hw, Ww, kh, kw, G, B, M, offset, No, span;
};

constexpr int kDirectThreads = 256;

// one CTA: 256 consecutive output coefficients of one (output ct, component, limb)
__global__ void __launch_bounds__(kDirectThreads)
k_conv_direct(const uint64_t *__restrict__ x, const int8_t *__restrict__ K, uint64_t *__restrict__ y,
              const LimbConst *__restrict__ limbs, uint32_t L, uint32_t N, DirectGeom g)
{
    const uint32_t tiles = N / kDirectThreads;
    const uint32_t tile = blockIdx.x % tiles;
    const uint32_t rest = blockIdx.x / tiles;
    const uint32_t limb = rest % L, comp = (rest / L) % 2, o = rest / (2 * L);
    const uint32_t mp = o / g.B, b = o % g.B;
    const uint32_t k = tile * kDirectThreads + threadIdx.x;
    const LimbConst &lc = limbs[limb];
    const uint64_t q = lc.q, nq = 0ull - q;
    const uint32_t ones = (uint32_t)lc.one_s;
    const size_t LN = (size_t)L * N;
    uint64_t acc_p = 0, acc_n = 0;  // terms of either sign, each < 2^57; reduced every 64 terms
    uint32_t n_terms = 0;
    const uint32_t area = g.Hw * g.Ww;
    // output channels m'*No + r share this output polynomial, channel r at shift r*span
    for (uint32_t r = 0; r < g.No; ++r) {
        const uint32_t m = mp * g.No + r;
        if (m >= g.M) break;
        for (uint32_t gi = 0; gi < g.G; ++gi) {
            const uint64_t *xr = x + (((size_t)(gi * g.B + b) * 2 + comp) * L + limb) * N;
            for (uint32_t c = 0; c < g.Cw; ++c) {
                const uint32_t ch = gi * g.Cw + c;
                if (ch >= g.C) break;
                const int8_t *kr = K + (((size_t)m * g.C + ch) * g.kh) * g.kw;
                for (uint32_t l = 0; l < g.kh; ++l)
                    for (uint32_t l2 = 0; l2 < g.kw; ++l2) {
                        const int w = __ldg(kr + l * g.kw + l2);
                        const uint32_t pos = r * g.span + g.offset - c * area - l * g.Ww - l2;
                        const bool wrap = k < pos;
                        const uint64_t xv = __ldg(xr + (wrap ? k + N - pos : k - pos));
                        const bool neg = (w < 0) != wrap;
                        const uint64_t t = xv * (uint64_t)(w < 0 ? -w : w);
                        if (neg)
                            acc_n += t;
                        else
                            acc_p += t;
                        if (++n_terms == 64) {
                            acc_p = reduce_lazy(acc_p, ones, nq);
                            acc_n = reduce_lazy(acc_n, ones, nq);
                            n_terms = 0;
                        }
                    }
            }
        }
    }
    const uint64_t p = canon3(reduce_lazy(acc_p, ones, nq), q), n = canon3(reduce_lazy(acc_n, ones, nq), q);
    y[((size_t)o * 2 + comp) * LN + (size_t)limb * N + k] = p >= n ? p - n : p + q - n;
}

}  // namespace

hc_status launch_conv_direct(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_in, uint64_t *d_out,
                             cudaStream_t s)
{
    const hc_conv_desc &d = w->desc;
    DirectGeom g{d.C, d.Cw, d.Hw, d.Ww, d.kh, d.kw, w->G, w->B, d.M,
                 (d.Cw - 1) * d.Hw * d.Ww + (d.kh - 1) * d.Ww + (d.kw - 1), w->No, d.Cw * d.Hw * d.Ww};
    const size_t blocks = (size_t)w->O * 2 * ctx->L * (ctx->N / kDirectThreads);
    if (blocks == 0) return HC_OK;
    if (blocks > 0x7fffffffu) return set_error(HC_ERR_INVALID_ARG, "layer too large");
    ProfileScope ps("k_conv_direct", s);
    k_conv_direct<<<(unsigned)blocks, kDirectThreads, 0, s>>>(d_in, w->d_k, d_out, ctx->d_limbs, ctx->L, ctx->N, g);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HC_OK : cuda_error(e, "launch k_conv_direct");
}

}  // namespace hc
