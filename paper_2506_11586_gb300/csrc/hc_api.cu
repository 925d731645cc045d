// hc_api.cu -- the C ABI of libhconv (include/hconv.h).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "hc_internal.h"

namespace hc {
const char *last_error();
void set_allocator(hc_alloc_fn a, hc_free_fn f, void *user);
}  // namespace hc

using namespace hc;

namespace {

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool ctx_ok(const hc_ctx *c) { return c && c->magic == kMagicCtx; }
inline bool weights_ok(const hc_weights *w) { return w && w->magic == kMagicWeights; }

uint32_t log2_exact(uint32_t n)
{
    uint32_t l = 0;
    while ((1u << l) < n) ++l;
    return ((1u << l) == n) ? l : 0xffffffffu;
}

// ---- partition of a stride-1 convolution --------------------------------------
struct Geom {
    uint32_t Cw, Hw, Ww, G, Bh, Bw, B, Mp, I, P, O;
    uint64_t cost;
};

// No output channels share one output polynomial (1 for convolutions)
Geom geom_of(const hc_conv_desc &d, uint32_t Cw, uint32_t Hw, uint32_t Ww, uint32_t No = 1)
{
    Geom g{};
    g.Cw = Cw;
    g.Hw = Hw;
    g.Ww = Ww;
    const uint32_t Ho = d.H + 2 * d.pad - d.kh + 1, Wo = d.W + 2 * d.pad - d.kw + 1;
    g.G = (d.C + Cw - 1) / Cw;
    const uint32_t oh = Hw - d.kh + 1, ow = Ww - d.kw + 1;
    g.Bh = (Ho + oh - 1) / oh;
    g.Bw = (Wo + ow - 1) / ow;
    g.B = g.Bh * g.Bw;
    g.Mp = (d.M + No - 1) / No;
    g.I = g.G * g.B;
    g.P = g.Mp * g.G;
    g.O = g.Mp * g.B;
    g.cost = 2ull * g.I + g.P + 2ull * g.O;
    return g;
}

// Phases of a strided convolution.  A stride-s convolution with zero padding p,
// y[m][r][c] = sum x~[ch][s*r+l][s*c+l'] K[m][ch][l][l'] (x~ the padded input),
// equals the stride-1 convolution without padding of the phase-split input
//   x'[(a*pb + b)*C + ch][i][j] = x~[ch][s*i + a][s*j + b]     (0 past x~'s edge)
// with the phase-split kernel
//   K'[m][(a*pb + b)*C + ch][u][v] = K[m][ch][s*u + a][s*v + b]  (0 past kh, kw),
// phases a < pa = min(s, kh), b < pb = min(s, kw), kernel ceil(kh/s) x ceil(kw/s)
// and x' of (Ho + kh' - 1) x (Wo + kw' - 1) for the strided output Ho x Wo
// (l = s*u + a gives s*r + l = s*(r + u) + a).  Phases a >= kh meet no weight
// and are left out.
struct Phases {
    uint32_t s, pa, pb;
};

hc_status effective_desc(const hc_conv_desc &d, hc_conv_desc *eff, Phases *ph)
{
    if (!d.C || !d.H || !d.W || !d.M || !d.kh || !d.kw)
        return set_error(HC_ERR_INVALID_ARG, "zero dimension in convolution descriptor");
    if (!d.stride) return set_error(HC_ERR_INVALID_ARG, "stride 0");
    const uint64_t Hp = (uint64_t)d.H + 2ull * d.pad, Wp = (uint64_t)d.W + 2ull * d.pad;
    if (Hp > 0xffffffffu || Wp > 0xffffffffu) return set_error(HC_ERR_INVALID_ARG, "padded input too large");
    if (d.kh > Hp || d.kw > Wp) return set_error(HC_ERR_INVALID_ARG, "kernel larger than padded input");
    *eff = d;
    *ph = Phases{1, 1, 1};
    if (d.stride == 1) return HC_OK;
    const uint32_t s = d.stride;
    const uint32_t Ho = (uint32_t)((Hp - d.kh) / s + 1), Wo = (uint32_t)((Wp - d.kw) / s + 1);
    const uint32_t kh1 = (d.kh + s - 1) / s, kw1 = (d.kw + s - 1) / s;
    ph->s = s;
    ph->pa = std::min(s, d.kh);
    ph->pb = std::min(s, d.kw);
    const uint64_t C1 = (uint64_t)ph->pa * ph->pb * d.C;
    if (C1 > 0xffffffffu) return set_error(HC_ERR_INVALID_ARG, "too many phase-split channels");
    eff->C = (uint32_t)C1;
    eff->H = Ho + kh1 - 1;
    eff->W = Wo + kw1 - 1;
    eff->kh = kh1;
    eff->kw = kw1;
    eff->stride = 1;
    eff->pad = 0;
    return HC_OK;
}

// K (int8 [M][C][kh][kw]) -> K' ([M][pa*pb*C][kh'][kw']) as above
void polyphase_kernel(const hc_conv_desc &d, const hc_conv_desc &eff, const Phases &ph, const int8_t *K,
                      std::vector<int8_t> &out)
{
    out.assign((size_t)eff.M * eff.C * eff.kh * eff.kw, 0);
    for (uint32_t m = 0; m < d.M; ++m)
        for (uint32_t a = 0; a < ph.pa; ++a)
            for (uint32_t b = 0; b < ph.pb; ++b)
                for (uint32_t ch = 0; ch < d.C; ++ch) {
                    const uint32_t c1 = (a * ph.pb + b) * d.C + ch;
                    for (uint32_t u = 0; u < eff.kh; ++u)
                        for (uint32_t v = 0; v < eff.kw; ++v) {
                            const uint32_t l = ph.s * u + a, l2 = ph.s * v + b;
                            if (l < d.kh && l2 < d.kw)
                                out[(((size_t)m * eff.C + c1) * eff.kh + u) * eff.kw + v] =
                                    K[(((size_t)m * d.C + ch) * d.kh + l) * d.kw + l2];
                        }
                }
}

// partition of the stride-1 layer `eff` (explicit, or the canonical search)
hc_status partition_of(const hc_conv_desc &d, uint32_t N, hc_conv_desc *res, Geom *geo)
{
    const uint32_t Hp = d.H + 2 * d.pad, Wp = d.W + 2 * d.pad;
    if ((uint64_t)d.kh * d.kw > N) return set_error(HC_ERR_INVALID_ARG, "kernel does not fit in N");
    Geom best{};
    bool have = false;
    if (d.Cw || d.Hw || d.Ww) {
        if (!d.Cw || !d.Hw || !d.Ww || d.Cw > d.C || d.Hw < d.kh || d.Ww < d.kw || d.Hw > Hp || d.Ww > Wp ||
            (uint64_t)d.Cw * d.Hw * d.Ww > N)
            return set_error(HC_ERR_INVALID_ARG, "invalid explicit partition Cw=%u Hw=%u Ww=%u", d.Cw, d.Hw, d.Ww);
        best = geom_of(d, d.Cw, d.Hw, d.Ww);
        have = true;
    } else {
        // exhaustive search: minimal 2I + P + 2O, then larger Hw*Ww, larger Cw, larger Ww
        for (uint32_t Cw = 1; Cw <= d.C && (uint64_t)Cw * d.kh * d.kw <= N; ++Cw) {
            for (uint32_t Hw = d.kh; Hw <= Hp && (uint64_t)Cw * Hw * d.kw <= N; ++Hw) {
                const uint32_t wmax = std::min<uint64_t>(Wp, N / ((uint64_t)Cw * Hw));
                for (uint32_t Ww = d.kw; Ww <= wmax; ++Ww) {
                    const Geom g = geom_of(d, Cw, Hw, Ww);
                    bool better;
                    if (!have) {
                        better = true;
                    } else if (g.cost != best.cost) {
                        better = g.cost < best.cost;
                    } else if (g.Hw * g.Ww != best.Hw * best.Ww) {
                        better = g.Hw * g.Ww > best.Hw * best.Ww;
                    } else if (g.Cw != best.Cw) {
                        better = g.Cw > best.Cw;
                    } else {
                        better = g.Ww > best.Ww;
                    }
                    if (better) {
                        best = g;
                        have = true;
                    }
                }
            }
        }
    }
    if (!have) return set_error(HC_ERR_INVALID_ARG, "no partition fits N = %u", N);
    *res = d;
    res->Cw = best.Cw;
    res->Hw = best.Hw;
    res->Ww = best.Ww;
    if (geo) *geo = best;
    return HC_OK;
}

// any convolution: *res is the stride-1 layer computed, with its partition
hc_status resolve_partition(const hc_conv_desc *desc, uint32_t N, hc_conv_desc *res, Geom *geo, Phases *ph = nullptr)
{
    if (!desc || !res) return set_error(HC_ERR_INVALID_ARG, "null descriptor");
    hc_conv_desc eff{};
    Phases p{};
    hc_status st = effective_desc(*desc, &eff, &p);
    if (st != HC_OK) return st;
    if (ph) *ph = p;
    return partition_of(eff, N, res, geo);
}

// A fully connected layer y = W x (W: M x C) is the 1x1 convolution on a 1x1
// image {C, 1, 1, M, 1, 1} with partition (Cw, 1, 1) and No output rows per
// output polynomial (matrix-vector packing):
//   input poly g : coeff [c] = x[g*Cw + c]
//   weight poly m'*G + g : coeff [r*Cw + Cw-1 - c] = W[m'*No + r][g*Cw + c]
//   output poly m' : coeff [r*Cw + Cw-1] holds y[m'*No + r]
// No*Cw <= N.  A term lands at r*Cw + Cw-1 + (c_in - c), |c_in - c| < Cw, so no
// other row's term reaches an extracted coefficient, and a term past X^N wraps
// below Cw - 1.  Canonical: minimal 2I + P + 2O, then fewer P, larger Cw,
// smaller No.
hc_conv_desc fc_conv(uint32_t C, uint32_t M, uint32_t Cw)
{
    hc_conv_desc d{};
    d.C = C;
    d.H = d.W = 1;
    d.M = M;
    d.kh = d.kw = 1;
    d.stride = 1;
    d.pad = 0;
    d.Cw = Cw;
    d.Hw = d.Ww = 1;
    return d;
}

hc_status resolve_fc(const hc_fc_desc *desc, uint32_t N, hc_fc_desc *res, hc_conv_desc *eff, Geom *geo)
{
    if (!desc) return set_error(HC_ERR_INVALID_ARG, "null descriptor");
    const hc_fc_desc d = *desc;
    if (!d.C || !d.M) return set_error(HC_ERR_INVALID_ARG, "zero dimension in fully connected descriptor");
    Geom best{};
    uint32_t best_no = 0;
    if (d.Cw || d.No) {
        if (!d.Cw || !d.No || d.Cw > d.C || d.No > d.M || (uint64_t)d.Cw * d.No > N)
            return set_error(HC_ERR_INVALID_ARG, "invalid explicit partition Cw=%u No=%u", d.Cw, d.No);
        best = geom_of(fc_conv(d.C, d.M, d.Cw), d.Cw, 1, 1, d.No);
        best_no = d.No;
    } else {
        const uint32_t cmax = std::min(d.C, N);
        for (uint32_t Cw = 1; Cw <= cmax; ++Cw) {
            const hc_conv_desc c = fc_conv(d.C, d.M, Cw);
            const uint32_t nmax = std::min(d.M, N / Cw);
            for (uint32_t No = 1; No <= nmax; ++No) {
                const Geom g = geom_of(c, Cw, 1, 1, No);
                bool better;
                if (!best_no) {
                    better = true;
                } else if (g.cost != best.cost) {
                    better = g.cost < best.cost;
                } else if (g.P != best.P) {
                    better = g.P < best.P;
                } else if (g.Cw != best.Cw) {
                    better = g.Cw > best.Cw;
                } else {
                    better = No < best_no;
                }
                if (better) {
                    best = g;
                    best_no = No;
                }
            }
        }
    }
    if (res) {
        *res = d;
        res->Cw = best.Cw;
        res->No = best_no;
    }
    if (eff) *eff = fc_conv(d.C, d.M, best.Cw);
    if (geo) *geo = best;
    return HC_OK;
}

// Pack int8 weights [M][C][kh][kw] of the stride-1 layer d into P = Mp*G
// polynomials of N int8 coefficients: poly (m', g) coefficient
// r*S + O - c*Hw*Ww - l*Ww - l' = K[m'*No + r][g*Cw + c][l][l'], S = Cw*Hw*Ww.
void pack_weights(const hc_conv_desc &d, const Geom &g, uint32_t No, uint32_t N, const int8_t *K,
                  std::vector<int8_t> &out)
{
    out.assign((size_t)g.P * N, 0);
    const uint32_t HW = g.Hw * g.Ww, S = g.Cw * HW;
    const uint32_t off = (g.Cw - 1) * HW + (d.kh - 1) * g.Ww + (d.kw - 1);
    for (uint32_t mp = 0; mp < g.Mp; ++mp)
        for (uint32_t gi = 0; gi < g.G; ++gi) {
            int8_t *poly = out.data() + ((size_t)mp * g.G + gi) * N;
            for (uint32_t r = 0; r < No; ++r) {
                const uint32_t m = mp * No + r;
                if (m >= d.M) break;
                for (uint32_t c = 0; c < g.Cw; ++c) {
                    const uint32_t ch = gi * g.Cw + c;
                    if (ch >= d.C) break;
                    for (uint32_t l = 0; l < d.kh; ++l)
                        for (uint32_t l2 = 0; l2 < d.kw; ++l2)
                            poly[r * S + off - c * HW - l * g.Ww - l2] =
                                K[(((size_t)m * d.C + ch) * d.kh + l) * d.kw + l2];
                }
            }
        }
}

// output-channel blocks of the pipelined host-buffer convolution
constexpr uint32_t kHostChunks = 8;

// per host thread and device: a copy stream and its events (made once, kept)
struct CopyLane {
    cudaStream_t st = nullptr;
    cudaEvent_t ev[kHostChunks + 1] = {};
};

hc_status copy_lane(CopyLane **out)
{
    static thread_local CopyLane lanes[32];
    int dev = 0;
    HC_CUDA_TRY(cudaGetDevice(&dev));
    CopyLane &l = lanes[dev & 31];
    if (!l.st) {
        HC_CUDA_TRY(cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking));
        for (auto &e : l.ev) HC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    *out = &l;
    return HC_OK;
}

struct ScratchGuard {
    void *p = nullptr;
    cudaStream_t s;
    explicit ScratchGuard(cudaStream_t st) : s(st) {}
    ~ScratchGuard() { dev_free(p, s); }
};

}  // namespace

namespace hc {
// Per-call scratch comes from the device's default stream-ordered pool.  With
// the pool's default release threshold (0) every synchronisation hands freed
// scratch back to the driver and the next call maps it again, which costs
// more than a small layer's kernels; keep freed scratch cached instead (once
// per device, and only if nobody has set a threshold).  cudaMemPoolTrimTo
// releases it.
void keep_scratch_cached(int device)
{
    static std::atomic<uint32_t> done{0};
    const uint32_t bit = 1u << (device & 31);
    if (done.fetch_or(bit) & bit) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    uint64_t cur = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur == 0) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
}

size_t conv_scratch_words(const hc_ctx *ctx, const hc_weights *w)
{
    // NTT-domain inputs, then dependency counters of the fused form (two per 64-bit word)
    return (size_t)w->I * 2 * ctx->L * ctx->N + (conv_counter_bound(ctx, w) + 1) / 2;
}

size_t conv_counter_bound(const hc_ctx *ctx, const hc_weights *w)
{
    return 1 + (size_t)ctx->L * (1 + w->Mp);
}

hc_status conv_layer(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_in, uint64_t *d_out,
                     uint64_t *scratch, size_t scratch_words, cudaStream_t s, const uint64_t *wpt)
{
    const size_t ntt_words = (size_t)w->I * 2 * ctx->L * ctx->N;
    const ConvJob job{ctx, w, d_in, d_out, scratch, conv_job_blocked(ctx, w), wpt};
    uint32_t *ctr = scratch_words > ntt_words ? reinterpret_cast<uint32_t *>(scratch + ntt_words) : nullptr;
    return launch_conv_jobs(&job, 1, s, ctr, ctr ? 2 * (scratch_words - ntt_words) : 0);
}

// one layer in the weights' preprocessing mode, scratch from the allocator
hc_status conv_any(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_in, uint64_t *d_out, cudaStream_t s)
{
    if (w->mode == HC_WEIGHTS_NO_NTT) return launch_conv_direct(ctx, w, d_in, d_out, s);
    const size_t words = conv_scratch_words(ctx, w);
    // the online weights start on a 256-byte boundary: the transforms store 16-byte
    // pairs and the MAC reads them with TMA bulk copies (16-byte aligned addresses)
    const size_t woff = (words + 31) & ~(size_t)31;
    const size_t wwords = w->mode == HC_WEIGHTS_NTT_ONLINE ? (size_t)w->P * ctx->L * ctx->N : 0;
    ScratchGuard scratch(s);
    scratch.p = dev_alloc((wwords ? woff + wwords : words) * sizeof(uint64_t), s);
    if (!scratch.p) return set_error(HC_ERR_OOM, "scratch allocation failed");
    uint64_t *base = (uint64_t *)scratch.p;
    if (!wwords) return conv_layer(ctx, w, d_in, d_out, base, words, s);
    // online NTT preprocessing: transform this query's weights first
    hc_status st = launch_ntt_fwd(ctx, w->d_pt, base + woff, w->P, s);
    if (st != HC_OK) return st;
    return conv_layer(ctx, w, d_in, d_out, base, words, s, base + woff);
}

// checked mode: HC_ERR_RANGE if any residue of [n][L][N] is >= its q_i (synchronises s)
hc_status check_inputs(const hc_ctx *ctx, const uint64_t *p, size_t n_polys, cudaStream_t s)
{
    if (!(ctx->flags & HC_CTX_CHECKED) || n_polys == 0) return HC_OK;
    HC_CUDA_TRY(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
    hc_status st = launch_range_check(ctx, p, n_polys, ctx->d_flag, s);
    if (st != HC_OK) return st;
    int h = 0;
    HC_CUDA_TRY(cudaMemcpyAsync(&h, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    HC_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) return set_error(HC_ERR_RANGE, "input residue out of range [0, q_i)");
    return HC_OK;
}
}  // namespace hc

namespace {
// Weights of the stride-1 layer `eff` (resolved partition, geometry g, No output
// rows per output polynomial) from its int8 kernel K [M][C][kh][kw].
hc_status build_weights(const hc_ctx *ctx, const hc_conv_desc &eff, const Geom &g, uint32_t No, uint32_t kind,
                        const hc_conv_desc &user, uint32_t pa, uint32_t pb, const int8_t *K, uint32_t mode,
                        hc_weights **out, cudaStream_t s)
{
    DeviceGuard guard(ctx->device);
    const uint32_t N = ctx->N, L = ctx->L;
    hc_status st = HC_OK;

    std::vector<int8_t> packed;
    // CSR of output terms: output o = m'*B + b sums g < G of (ct g*B + b, pt m'*G + g)
    std::vector<uint32_t> term_ptr((size_t)g.O + 1), terms((size_t)2 * g.O * g.G);
    for (uint32_t m = 0; m < g.Mp; ++m)
        for (uint32_t b = 0; b < g.B; ++b) {
            const uint32_t o = m * g.B + b;
            term_ptr[o] = o * g.G;
            for (uint32_t gi = 0; gi < g.G; ++gi) {
                terms[2 * ((size_t)o * g.G + gi)] = gi * g.B + b;
                terms[2 * ((size_t)o * g.G + gi) + 1] = m * g.G + gi;
            }
        }
    term_ptr[g.O] = g.O * g.G;

    hc_weights *w = new (std::nothrow) hc_weights();
    if (!w) return set_error(HC_ERR_OOM, "host allocation failed");
    w->magic = kMagicWeights;
    w->ctx = ctx;
    w->device = ctx->device;
    w->desc = eff;
    w->user = user;
    w->user.Cw = eff.Cw;
    w->user.Hw = eff.Hw;
    w->user.Ww = eff.Ww;
    w->kind = kind;
    w->No = No;
    w->Mp = g.Mp;
    w->pa = pa;
    w->pb = pb;
    w->G = g.G;
    w->B = g.B;
    w->I = g.I;
    w->P = g.P;
    w->O = g.O;
    w->mode = mode;
    st = build_slot_table(w);
    if (st != HC_OK) {
        hc_free(w);
        return st;
    }
    if (mode == HC_WEIGHTS_NO_NTT) {
        // keep the small signed weights of the stride-1 layer; nothing is packed, lifted or transformed
        const size_t kbytes = (size_t)eff.M * eff.C * eff.kh * eff.kw;
        w->d_k = (int8_t *)dev_alloc_persistent(kbytes);
        cudaError_t e = w->d_k ? cudaMemcpy(w->d_k, K, kbytes, cudaMemcpyHostToDevice) : cudaErrorMemoryAllocation;
        if (e != cudaSuccess) {
            hc_free(w);
            return e == cudaErrorMemoryAllocation ? set_error(HC_ERR_OOM, "device allocation of weights failed")
                                                  : cuda_error(e, "uploading weights");
        }
        *out = w;
        return HC_OK;
    }
    pack_weights(eff, g, No, N, K, packed);
    w->d_pt = (uint64_t *)dev_alloc_persistent((size_t)g.P * L * N * sizeof(uint64_t));
    w->d_term_ptr = (uint32_t *)dev_alloc_persistent(term_ptr.size() * sizeof(uint32_t));
    w->d_terms = (uint32_t *)dev_alloc_persistent(terms.size() * sizeof(uint32_t));
    int8_t *d_packed = (int8_t *)dev_alloc(packed.size(), s);
    auto fail = [&](hc_status e) {
        dev_free(d_packed, s);
        cudaStreamSynchronize(s);
        hc_free(w);
        return e;
    };
    if (!w->d_pt || !w->d_term_ptr || !w->d_terms || !d_packed)
        return fail(set_error(HC_ERR_OOM, "device allocation of weights failed"));
    cudaError_t e = cudaMemcpyAsync(d_packed, packed.data(), packed.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w->d_term_ptr, term_ptr.data(), term_ptr.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w->d_terms, terms.data(), terms.size() * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(cuda_error(e, "uploading weights"));
    st = launch_lift_int8(ctx, d_packed, w->d_pt, g.P, s);
    if (st == HC_OK && mode == HC_WEIGHTS_NTT_OFFLINE) st = launch_ntt_fwd(ctx, w->d_pt, w->d_pt, g.P, s);
    if (st != HC_OK) return fail(st);
    // the host copy must outlive the asynchronous upload
    e = cudaStreamSynchronize(s);
    dev_free(d_packed, s);
    d_packed = nullptr;
    if (e != cudaSuccess) return fail(cuda_error(e, "weights preprocessing"));
    *out = w;
    return HC_OK;
}

// weights of a convolution (any stride) or of a fully connected layer, from the
// caller's descriptor and int8 kernel
hc_status make_conv_weights(const hc_ctx *ctx, const hc_conv_desc *desc, const int8_t *h_K, uint32_t mode,
                            hc_weights **out, cudaStream_t s)
{
    hc_conv_desc res{};
    Geom g{};
    Phases ph{};
    hc_status st = resolve_partition(desc, ctx->N, &res, &g, &ph);
    if (st != HC_OK) return st;
    if (ph.s == 1) return build_weights(ctx, res, g, 1, LAYER_CONV, *desc, 1, 1, h_K, mode, out, s);
    std::vector<int8_t> k1;
    polyphase_kernel(*desc, res, ph, h_K, k1);
    return build_weights(ctx, res, g, 1, LAYER_CONV, *desc, ph.pa, ph.pb, k1.data(), mode, out, s);
}

hc_status make_fc_weights(const hc_ctx *ctx, const hc_fc_desc *desc, const int8_t *h_W, uint32_t mode,
                          hc_weights **out, cudaStream_t s)
{
    hc_fc_desc res{};
    hc_conv_desc eff{};
    Geom g{};
    hc_status st = resolve_fc(desc, ctx->N, &res, &eff, &g);
    if (st != HC_OK) return st;
    // W [M][C] is the kernel [M][C][1][1] of the 1x1 convolution
    return build_weights(ctx, eff, g, res.No, LAYER_FC, eff, 1, 1, h_W, mode, out, s);
}
}  // namespace

namespace hc {
hc_status layer_geometry(const hc_conv_desc &user, uint32_t kind, uint32_t No, uint32_t N, LayerGeom *out)
{
    Geom g{};
    LayerGeom lg{};
    if (kind == LAYER_FC) {
        if (user.H != 1 || user.W != 1 || user.kh != 1 || user.kw != 1 || user.stride != 1 || user.pad != 0)
            return set_error(HC_ERR_INVALID_ARG, "not a fully connected layer");
        const hc_fc_desc d{user.C, user.M, user.Cw, No};
        hc_status st = resolve_fc(&d, N, nullptr, &lg.eff, &g);
        if (st != HC_OK) return st;
        lg.No = No;
        lg.pa = lg.pb = 1;
    } else if (kind == LAYER_CONV) {
        if (No != 1) return set_error(HC_ERR_INVALID_ARG, "convolutions have one output channel per ciphertext");
        Phases ph{};
        hc_status st = resolve_partition(&user, N, &lg.eff, &g, &ph);
        if (st != HC_OK) return st;
        lg.No = 1;
        lg.pa = ph.pa;
        lg.pb = ph.pb;
    } else {
        return set_error(HC_ERR_INVALID_ARG, "unknown layer kind %u", kind);
    }
    lg.Mp = g.Mp;
    lg.G = g.G;
    lg.B = g.B;
    lg.I = g.I;
    lg.P = g.P;
    lg.O = g.O;
    *out = lg;
    return HC_OK;
}
}  // namespace hc

// =============================================================================
extern "C" {

const char *hc_version(void) { return "hconv 0.1 (sm_103a)"; }

const char *hc_status_str(hc_status s)
{
    switch (s) {
    case HC_OK: return "HC_OK";
    case HC_ERR_INVALID_ARG: return "HC_ERR_INVALID_ARG";
    case HC_ERR_BAD_MODULUS: return "HC_ERR_BAD_MODULUS";
    case HC_ERR_RANGE: return "HC_ERR_RANGE";
    case HC_ERR_OOM: return "HC_ERR_OOM";
    case HC_ERR_BUDGET: return "HC_ERR_BUDGET";
    case HC_ERR_TIMEOUT: return "HC_ERR_TIMEOUT";
    case HC_ERR_CUDA: return "HC_ERR_CUDA";
    case HC_ERR_UNSUPPORTED: return "HC_ERR_UNSUPPORTED";
    }
    return "HC_ERR_UNKNOWN";
}

const char *hc_last_error(void) { return hc::last_error(); }

void hc_set_allocator(hc_alloc_fn alloc, hc_free_fn free_fn, void *user) { hc::set_allocator(alloc, free_fn, user); }

hc_status hc_ctx_validate(uint32_t N, const uint64_t *moduli, uint32_t L, uint64_t t)
{
    if (!moduli) return set_error(HC_ERR_INVALID_ARG, "moduli is NULL");
    if (N != 4096 && N != 8192 && N != 16384) return set_error(HC_ERR_INVALID_ARG, "unsupported N = %u", N);
    if (L == 0 || L > kMaxLimbs) return set_error(HC_ERR_INVALID_ARG, "L = %u outside [1, %u]", L, kMaxLimbs);
    if (t < 2) return set_error(HC_ERR_INVALID_ARG, "plaintext modulus t < 2");
    for (uint32_t i = 0; i < L; ++i) {
        const uint64_t q = moduli[i];
        if (q >= (1ull << 50)) return set_error(HC_ERR_BAD_MODULUS, "q[%u] = %llu >= 2^50", i, (unsigned long long)q);
        if (q <= (1ull << 32)) return set_error(HC_ERR_BAD_MODULUS, "q[%u] = %llu <= 2^32", i, (unsigned long long)q);
        if (q % (2ull * N) != 1)
            return set_error(HC_ERR_BAD_MODULUS, "q[%u] = %llu is not 1 mod 2N", i, (unsigned long long)q);
        if (!is_prime_u64(q)) return set_error(HC_ERR_BAD_MODULUS, "q[%u] = %llu is not prime", i, (unsigned long long)q);
        for (uint32_t j = 0; j < i; ++j)
            if (moduli[j] == q) return set_error(HC_ERR_BAD_MODULUS, "q[%u] duplicates q[%u]", i, j);
    }
    return HC_OK;
}

hc_status hc_ctx_create_ex(uint32_t N, const uint64_t *moduli, uint32_t L, uint64_t t, uint32_t flags,
                           hc_ctx **out)
{
    if (!out) return set_error(HC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    hc_status st = hc_ctx_validate(N, moduli, L, t);
    if (st != HC_OK) return st;

    hc_ctx *c = new (std::nothrow) hc_ctx();
    if (!c) return set_error(HC_ERR_OOM, "host allocation failed");
    c->magic = kMagicCtx;
    c->N = N;
    c->logN = log2_exact(N);
    c->L = L;
    c->t = t;
    c->flags = flags;
    for (int k = 0; k < KK_COUNT; ++k) c->variant[k] = (uint8_t)default_variant(k, c->logN);
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        cudaGetLastError();
        return set_error(HC_ERR_CUDA, "no CUDA device");
    }
    {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms <= 0) {
            delete c;
            cudaGetLastError();
            return set_error(HC_ERR_CUDA, "cannot read the SM count of device %d", c->device);
        }
        c->sms = (uint32_t)sms;
    }
    keep_scratch_cached(c->device);

    // host tables: per limb, forward and inverse twiddles with Shoup companions
    // per limb: forward, inverse, then the rearranged tables (inverse first round,
    // forward last round) for LOGC = 3, 4, 5
    constexpr uint32_t kTablesPerLimb = 8;
    std::vector<ulonglong2> tw((size_t)kTablesPerLimb * L * N);
    std::vector<LimbConst> lcs(L);
    std::vector<uint64_t> delta(L);
    delta_residues(moduli, L, t, delta.data());
    for (uint32_t i = 0; i < L; ++i) {
        const uint64_t q = moduli[i];
        const uint64_t psi = min_primitive_2n_root(q, N);
        if (!psi) {
            delete c;
            return set_error(HC_ERR_BAD_MODULUS, "no primitive 2N-th root mod q[%u]", i);
        }
        const uint64_t psi_inv = powmod_u64(psi, q - 2, q);
        c->q[i] = q;
        c->psi[i] = psi;
        ulonglong2 *f = tw.data() + (size_t)(kTablesPerLimb * i) * N;
        ulonglong2 *b = tw.data() + (size_t)(kTablesPerLimb * i + 1) * N;
        // powers psi^j and psi^-j in natural order, then scattered to bit-reversed slots
        uint64_t pf = 1, pb = 1;
        for (uint32_t j = 0; j < N; ++j) {
            const uint32_t k = bit_reverse(j, c->logN);
            f[k].x = pf;
            f[k].y = shoup_companion(pf, q);
            b[k].x = pb;
            b[k].y = shoup_companion(pb, q);
            pf = mulmod_u64(pf, psi, q);
            pb = mulmod_u64(pb, psi_inv, q);
        }
        // first inverse register round with 2^lc residues per thread (thread t, stage s,
        // group g uses b[(N >> (s+1)) + t*2^(lc-1-s) + g]), rearranged for coalesced reads
        for (uint32_t lcg = 3; lcg <= 5 && lcg < c->logN; ++lcg) {
            ulonglong2 *r0 = tw.data() + (size_t)(kTablesPerLimb * i + 2 + (lcg - 3)) * N;
            const uint32_t T = N >> lcg;
            for (uint32_t st = 0; st < lcg; ++st) {
                const uint32_t ngrp = 1u << (lcg - 1 - st), off = N - (N >> st);
                for (uint32_t g = 0; g < ngrp; ++g)
                    for (uint32_t tt = 0; tt < T; ++tt) r0[off + g * T + tt] = b[(N >> (st + 1)) + tt * ngrp + g];
            }
            // last forward register round (stages S0 .. log2 N - 1, SUBS sub-transforms per
            // thread): thread t, sub-transform v, stage S0 + sig, group lam uses
            // f[2^(S0+sig) + (t*SUBS + v)*2^sig + lam]
            ulonglong2 *rl = tw.data() + (size_t)(kTablesPerLimb * i + 5 + (lcg - 3)) * N;
            const uint32_t nr = (c->logN + lcg - 1) / lcg, S0 = (nr - 1) * lcg, K = c->logN - S0;
            const uint32_t subs = 1u << (lcg - K);
            for (uint32_t sig = 0; sig < K; ++sig) {
                const uint32_t st = S0 + sig, off = (1u << st) - (1u << S0);
                for (uint32_t v = 0; v < subs; ++v)
                    for (uint32_t lam = 0; lam < (1u << sig); ++lam)
                        for (uint32_t tt = 0; tt < T; ++tt)
                            rl[off + ((v << sig) + lam) * T + tt] = f[(1u << st) + ((tt * subs + v) << sig) + lam];
            }
        }
        LimbConst &lc = lcs[i];
        memset(&lc, 0, sizeof(lc));
        lc.q = q;
        lc.r64 = (uint64_t)(((unsigned __int128)1 << 64) % q);
        lc.r64_s = shoup_companion(lc.r64, q);
        lc.one_s = shoup_companion(1, q);
        lc.ninv = powmod_u64(N, q - 2, q);
        lc.ninv_s = shoup_companion(lc.ninv, q);
        lc.ninvw = mulmod_u64(lc.ninv, b[1].x, q);
        lc.ninvw_s = shoup_companion(lc.ninvw, q);
        lc.delta = delta[i];
        lc.delta_s = shoup_companion(delta[i], q);
        const uint64_t c50 = (1ull << 50) - q;
        lc.special_c = c50 > 0 && c50 < (1ull << 22) ? c50 : 0;
    }

    c->table_bytes = tw.size() * sizeof(ulonglong2);
    c->d_tables = dev_alloc_persistent(c->table_bytes);
    c->d_limbs = (LimbConst *)dev_alloc_persistent(sizeof(LimbConst) * L);
    c->d_flag = (int *)dev_alloc_persistent(sizeof(int) * 4);
    if (!c->d_tables || !c->d_limbs || !c->d_flag) {
        dev_free_persistent(c->d_tables);
        dev_free_persistent(c->d_limbs);
        dev_free_persistent(c->d_flag);
        delete c;
        return set_error(HC_ERR_OOM, "device allocation of context tables failed");
    }
    for (uint32_t i = 0; i < L; ++i) {
        lcs[i].tw_f = (const ulonglong2 *)c->d_tables + (size_t)(kTablesPerLimb * i) * N;
        lcs[i].tw_i = (const ulonglong2 *)c->d_tables + (size_t)(kTablesPerLimb * i + 1) * N;
        lcs[i].tw_r = (const ulonglong2 *)c->d_tables + (size_t)(kTablesPerLimb * i + 2) * N;
    }
    cudaError_t e = cudaMemcpy(c->d_tables, tw.data(), c->table_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_limbs, lcs.data(), sizeof(LimbConst) * L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->d_flag, 0, sizeof(int) * 4);
    if (e != cudaSuccess) {
        hc_status s2 = cuda_error(e, "uploading context tables");
        dev_free_persistent(c->d_tables);
        dev_free_persistent(c->d_limbs);
        dev_free_persistent(c->d_flag);
        delete c;
        return s2;
    }
    *out = c;
    return HC_OK;
}

hc_status hc_ctx_create(uint32_t N, const uint64_t *moduli, uint32_t L, uint64_t t, hc_ctx **out)
{
    return hc_ctx_create_ex(N, moduli, L, t, 0, out);
}

hc_status hc_ctx_device_status(const hc_ctx *ctx, void *cuda_stream)
{
    if (!ctx_ok(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    DeviceGuard g(ctx->device);
    cudaStream_t s = as_stream(cuda_stream);
    int h = 0;
    HC_CUDA_TRY(cudaMemcpyAsync(&h, ctx->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    HC_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) {
        HC_CUDA_TRY(cudaMemsetAsync(ctx->d_flag + 1, 0, sizeof(int), s));
        HC_CUDA_TRY(cudaStreamSynchronize(s));
        return set_error(HC_ERR_TIMEOUT, "a bounded device-side wait expired (code %d)", h);
    }
    return HC_OK;
}

hc_status hc_selftest_wait_timeout(const hc_ctx *ctx, uint32_t limit, void *cuda_stream)
{
    if (!ctx_ok(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (limit == 0 || limit > (1u << 20)) return set_error(HC_ERR_INVALID_ARG, "limit must be in [1, 2^20]");
    DeviceGuard g(ctx->device);
    return launch_wait_selftest(ctx, limit, as_stream(cuda_stream));
}

hc_status hc_ctx_set_variant(hc_ctx *ctx, uint32_t kind, uint32_t variant)
{
    if (!ctx_ok(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (kind >= (uint32_t)KK_COUNT) return set_error(HC_ERR_INVALID_ARG, "kernel kind %u out of range", kind);
    if (variant >= (uint32_t)kind_variants((int)kind))
        return set_error(HC_ERR_INVALID_ARG, "variant %u out of range", variant);
    ctx->variant[kind] = (uint8_t)variant;
    return HC_OK;
}

hc_status hc_ctx_get_variant(const hc_ctx *ctx, uint32_t kind, uint32_t *variant)
{
    if (!ctx_ok(ctx) || !variant) return set_error(HC_ERR_INVALID_ARG, "invalid context or output");
    if (kind >= (uint32_t)KK_COUNT) return set_error(HC_ERR_INVALID_ARG, "kernel kind %u out of range", kind);
    *variant = ctx->variant[kind];
    return HC_OK;
}

hc_status hc_ctx_info(const hc_ctx *ctx, uint32_t *N, uint32_t *L, uint64_t *t, uint64_t *moduli_out,
                      uint64_t *psi_out)
{
    if (!ctx_ok(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (N) *N = ctx->N;
    if (L) *L = ctx->L;
    if (t) *t = ctx->t;
    for (uint32_t i = 0; i < ctx->L; ++i) {
        if (moduli_out) moduli_out[i] = ctx->q[i];
        if (psi_out) psi_out[i] = ctx->psi[i];
    }
    return HC_OK;
}

hc_status hc_ntt_fwd(const hc_ctx *ctx, uint64_t *d_polys, size_t n_polys, void *cuda_stream)
{
    if (!ctx_ok(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (n_polys == 0) return HC_OK;
    if (!d_polys) return set_error(HC_ERR_INVALID_ARG, "d_polys is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t s = as_stream(cuda_stream);
    hc_status st = check_inputs(ctx, d_polys, n_polys, s);
    if (st != HC_OK) return st;
    return launch_ntt_fwd(ctx, d_polys, d_polys, n_polys, s);
}

hc_status hc_ntt_inv(const hc_ctx *ctx, uint64_t *d_polys, size_t n_polys, void *cuda_stream)
{
    if (!ctx_ok(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (n_polys == 0) return HC_OK;
    if (!d_polys) return set_error(HC_ERR_INVALID_ARG, "d_polys is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t s = as_stream(cuda_stream);
    hc_status st = check_inputs(ctx, d_polys, n_polys, s);
    if (st != HC_OK) return st;
    return launch_ntt_inv(ctx, d_polys, d_polys, n_polys, s);
}

hc_status hc_conv_partition(const hc_conv_desc *desc, uint32_t N, hc_conv_desc *resolved, uint32_t *n_in_ct,
                            uint32_t *n_pt, uint32_t *n_out_ct)
{
    Geom g{};
    hc_status st = resolve_partition(desc, N, resolved, &g);
    if (st != HC_OK) return st;
    if (n_in_ct) *n_in_ct = g.I;
    if (n_pt) *n_pt = g.P;
    if (n_out_ct) *n_out_ct = g.O;
    return HC_OK;
}

hc_status hc_fc_partition(const hc_fc_desc *desc, uint32_t N, hc_fc_desc *resolved, uint32_t *n_in_ct,
                          uint32_t *n_pt, uint32_t *n_out_ct)
{
    if (!resolved) return set_error(HC_ERR_INVALID_ARG, "resolved is NULL");
    Geom g{};
    hc_status st = resolve_fc(desc, N, resolved, nullptr, &g);
    if (st != HC_OK) return st;
    if (n_in_ct) *n_in_ct = g.I;
    if (n_pt) *n_pt = g.P;
    if (n_out_ct) *n_out_ct = g.O;
    return HC_OK;
}

hc_status hc_weights_preprocess(const hc_ctx *ctx, const hc_conv_desc *desc, const int8_t *h_K, hc_weights **out,
                                void *cuda_stream)
{
    return hc_weights_preprocess_ex(ctx, desc, h_K, HC_WEIGHTS_NTT_OFFLINE, out, cuda_stream);
}


hc_status hc_weights_preprocess_range(const hc_ctx *ctx, const hc_conv_desc *desc, const int8_t *h_K,
                                      uint32_t m0, uint32_t m1, hc_weights **out, void *cuda_stream)
{
    if (!out) return set_error(HC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx_ok(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (!desc || !h_K) return set_error(HC_ERR_INVALID_ARG, "null descriptor or kernel");
    if (!(m0 < m1 && m1 <= desc->M))
        return set_error(HC_ERR_INVALID_ARG, "channel range [%u, %u) not inside [0, %u)", m0, m1, desc->M);
    // the whole layer's partition, forced on the shard: same input blocks, same packing
    hc_conv_desc res{};
    uint32_t I = 0, P = 0, O = 0;
    hc_status st = hc_conv_partition(desc, ctx->N, &res, &I, &P, &O);
    if (st != HC_OK) return st;
    hc_conv_desc sub = *desc;
    sub.M = m1 - m0;
    sub.Cw = res.Cw;
    sub.Hw = res.Hw;
    sub.Ww = res.Ww;
    const size_t per = (size_t)desc->C * desc->kh * desc->kw;
    return hc_weights_preprocess_ex(ctx, &sub, h_K + (size_t)m0 * per, HC_WEIGHTS_NTT_OFFLINE, out, cuda_stream);
}

hc_status hc_weights_preprocess_ex(const hc_ctx *ctx, const hc_conv_desc *desc, const int8_t *h_K, uint32_t mode,
                                   hc_weights **out, void *cuda_stream)
{
    if (!out) return set_error(HC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx_ok(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (!h_K) return set_error(HC_ERR_INVALID_ARG, "h_K is NULL");
    if (mode > HC_WEIGHTS_NO_NTT) return set_error(HC_ERR_INVALID_ARG, "unknown weights mode %u", mode);
    return make_conv_weights(ctx, desc, h_K, mode, out, as_stream(cuda_stream));
}

hc_status hc_weights_preprocess_fc(const hc_ctx *ctx, const hc_fc_desc *desc, const int8_t *h_W, uint32_t mode,
                                   hc_weights **out, void *cuda_stream)
{
    if (!out) return set_error(HC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx_ok(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (!h_W) return set_error(HC_ERR_INVALID_ARG, "h_W is NULL");
    if (mode > HC_WEIGHTS_NO_NTT) return set_error(HC_ERR_INVALID_ARG, "unknown weights mode %u", mode);
    return make_fc_weights(ctx, desc, h_W, mode, out, as_stream(cuda_stream));
}

hc_status hc_weights_layout(const hc_weights *w, hc_conv_desc *computed, uint32_t *kind, uint32_t *No,
                            uint32_t *n_slots)
{
    if (!weights_ok(w)) return set_error(HC_ERR_INVALID_ARG, "invalid weights handle");
    if (computed) *computed = w->desc;
    if (kind) *kind = w->kind;
    if (No) *No = w->No;
    if (n_slots) *n_slots = w->No * (w->desc.Hw - w->desc.kh + 1) * (w->desc.Ww - w->desc.kw + 1);
    return HC_OK;
}

hc_status hc_conv_geometry(const hc_weights *w, uint32_t *n_in_ct, uint32_t *n_out_ct, uint32_t *Cw, uint32_t *Hw,
                           uint32_t *Ww)
{
    if (!weights_ok(w)) return set_error(HC_ERR_INVALID_ARG, "invalid weights handle");
    if (n_in_ct) *n_in_ct = w->I;
    if (n_out_ct) *n_out_ct = w->O;
    if (Cw) *Cw = w->desc.Cw;
    if (Hw) *Hw = w->desc.Hw;
    if (Ww) *Ww = w->desc.Ww;
    return HC_OK;
}

hc_status hc_weights_data(const hc_weights *w, const uint64_t **d_pt_ntt, size_t *n_pt)
{
    if (!weights_ok(w)) return set_error(HC_ERR_INVALID_ARG, "invalid weights handle");
    if (w->mode == HC_WEIGHTS_NO_NTT) return set_error(HC_ERR_UNSUPPORTED, "weights kept without NTT have no plaintexts");
    if (d_pt_ntt) *d_pt_ntt = w->d_pt;
    if (n_pt) *n_pt = w->P;
    return HC_OK;
}

hc_status hc_weights_export(const hc_weights *w, uint64_t *d_dst, void *cuda_stream)
{
    if (!weights_ok(w)) return set_error(HC_ERR_INVALID_ARG, "invalid weights handle");
    if (!d_dst) return set_error(HC_ERR_INVALID_ARG, "d_dst is NULL");
    if (w->mode == HC_WEIGHTS_NO_NTT) return set_error(HC_ERR_UNSUPPORTED, "weights kept without NTT have no plaintexts");
    DeviceGuard g(w->device);
    const size_t bytes = (size_t)w->P * w->ctx->L * w->ctx->N * sizeof(uint64_t);
    HC_CUDA_TRY(cudaMemcpyAsync(d_dst, w->d_pt, bytes, cudaMemcpyDeviceToDevice, as_stream(cuda_stream)));
    return HC_OK;
}

hc_status hc_conv_ct_pt(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_ct_in, uint64_t *d_ct_out,
                        void *cuda_stream)
{
    if (!ctx_ok(ctx) || !weights_ok(w)) return set_error(HC_ERR_INVALID_ARG, "invalid context or weights");
    if (w->ctx != ctx) return set_error(HC_ERR_INVALID_ARG, "weights were preprocessed for another context");
    if (!d_ct_in || !d_ct_out) return set_error(HC_ERR_INVALID_ARG, "null ciphertext buffer");
    DeviceGuard g(ctx->device);
    cudaStream_t s = as_stream(cuda_stream);
    hc_status st = check_inputs(ctx, d_ct_in, (size_t)2 * w->I, s);
    if (st != HC_OK) return st;
    return conv_any(ctx, w, d_ct_in, d_ct_out, s);
}

hc_status hc_conv_ct_pt_plain(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_ct_in, uint64_t *d_ct_out,
                              void *cuda_stream)
{
    if (!ctx_ok(ctx) || !weights_ok(w)) return set_error(HC_ERR_INVALID_ARG, "invalid context or weights");
    if (w->ctx != ctx) return set_error(HC_ERR_INVALID_ARG, "weights were preprocessed for another context");
    if (!d_ct_in || !d_ct_out) return set_error(HC_ERR_INVALID_ARG, "null ciphertext buffer");
    if (w->mode != HC_WEIGHTS_NTT_OFFLINE)
        return set_error(HC_ERR_UNSUPPORTED, "the plain form needs NTT-preprocessed (offline) weights");
    DeviceGuard g(ctx->device);
    cudaStream_t s = as_stream(cuda_stream);
    hc_status st = check_inputs(ctx, d_ct_in, (size_t)2 * w->I, s);
    if (st != HC_OK) return st;
    const size_t ct_words = (size_t)2 * ctx->L * ctx->N, pt_words = (size_t)ctx->L * ctx->N;
    HC_CUDA_TRY(cudaMemsetAsync(d_ct_out, 0, (size_t)w->O * ct_words * sizeof(uint64_t), s));
    const uint32_t M = w->Mp;
    for (uint32_t m = 0; m < M; ++m)
        for (uint32_t gi = 0; gi < w->G; ++gi)
            for (uint32_t b = 0; b < w->B; ++b) {
                st = launch_product(ctx, d_ct_in + (size_t)(gi * w->B + b) * ct_words,
                                    w->d_pt + (size_t)(m * w->G + gi) * pt_words, nullptr,
                                    d_ct_out + (size_t)(m * w->B + b) * ct_words, 1, true, s);
                if (st != HC_OK) return st;
            }
    return HC_OK;
}

hc_status hc_conv_ct_pt_host(const hc_ctx *ctx, const hc_weights *w, const uint64_t *h_ct_in, uint64_t *h_ct_out,
                             void *cuda_stream)
{
    if (!ctx_ok(ctx) || !weights_ok(w)) return set_error(HC_ERR_INVALID_ARG, "invalid context or weights");
    if (w->ctx != ctx) return set_error(HC_ERR_INVALID_ARG, "weights were preprocessed for another context");
    if (!h_ct_in || !h_ct_out) return set_error(HC_ERR_INVALID_ARG, "null ciphertext buffer");
    DeviceGuard g(ctx->device);
    cudaStream_t s = as_stream(cuda_stream);
    const size_t ct_words = (size_t)2 * ctx->L * ctx->N, ct_bytes = ct_words * sizeof(uint64_t);
    ScratchGuard din(s), dout(s), dntt(s);
    din.p = dev_alloc(w->I * ct_bytes, s);
    dout.p = dev_alloc(w->O * ct_bytes, s);
    if (!din.p || !dout.p) return set_error(HC_ERR_OOM, "device buffer allocation failed");
    HC_CUDA_TRY(cudaMemcpyAsync(din.p, h_ct_in, w->I * ct_bytes, cudaMemcpyHostToDevice, s));
    const uint32_t K = std::min<uint32_t>(kHostChunks, w->Mp);
    if (w->mode != HC_WEIGHTS_NTT_OFFLINE || !conv_job_blocked(ctx, w) || K < 2) {
        hc_status st = hc_conv_ct_pt(ctx, w, (const uint64_t *)din.p, (uint64_t *)dout.p, cuda_stream);
        if (st != HC_OK) return st;
        HC_CUDA_TRY(cudaMemcpyAsync(h_ct_out, dout.p, w->O * ct_bytes, cudaMemcpyDeviceToHost, s));
        return hc_ctx_device_status(ctx, cuda_stream);
    }
    // Pipelined: the outputs of a block of output channels (contiguous in the output
    // and in the weights) go back to the host while the next block is computed.
    hc_status st = check_inputs(ctx, (const uint64_t *)din.p, (size_t)2 * w->I, s);
    if (st != HC_OK) return st;
    CopyLane *lane = nullptr;
    st = copy_lane(&lane);
    if (st != HC_OK) return st;
    dntt.p = dev_alloc(w->I * ct_bytes, s);
    if (!dntt.p) return set_error(HC_ERR_OOM, "device buffer allocation failed");
    uint64_t *x = (uint64_t *)dntt.p, *y = (uint64_t *)dout.p;
    st = launch_ntt_fwd_ct(ctx, (const uint64_t *)din.p, x, w->I, s);
    if (st != HC_OK) return st;
    const size_t LN = (size_t)ctx->L * ctx->N;
    const uint32_t per = (w->Mp + K - 1) / K;
    uint32_t used = 0;
    for (uint32_t j = 0; j < K; ++j) {
        const uint32_t m0 = j * per, m1 = std::min(w->Mp, m0 + per);
        if (m0 >= m1) break;
        const size_t o0 = (size_t)m0 * w->B, no = (size_t)(m1 - m0) * w->B;
        st = launch_mac_conv(ctx, x, w->d_pt + (size_t)m0 * w->G * LN, y + o0 * ct_words, w->G, w->B, m1 - m0, s);
        if (st == HC_OK) st = launch_ntt_inv_ct(ctx, y + o0 * ct_words, y + o0 * ct_words, no, s);
        if (st != HC_OK) return st;
        HC_CUDA_TRY(cudaEventRecord(lane->ev[j], s));
        HC_CUDA_TRY(cudaStreamWaitEvent(lane->st, lane->ev[j], 0));
        HC_CUDA_TRY(cudaMemcpyAsync(h_ct_out + o0 * ct_words, y + o0 * ct_words, no * ct_bytes,
                                    cudaMemcpyDeviceToHost, lane->st));
        used = j + 1;
    }
    HC_CUDA_TRY(cudaEventRecord(lane->ev[used], lane->st));
    HC_CUDA_TRY(cudaStreamWaitEvent(s, lane->ev[used], 0));  // scratch is freed after the copies
    return hc_ctx_device_status(ctx, cuda_stream);
}

hc_status hc_ctpt_mac(const hc_ctx *ctx, const uint64_t *d_ct, const uint64_t *d_pt_ntt, const uint32_t *h_slot,
                      size_t n, uint64_t *d_out, size_t n_out, void *cuda_stream)
{
    if (!ctx_ok(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (n_out == 0) return HC_OK;
    if (!d_out) return set_error(HC_ERR_INVALID_ARG, "d_out is NULL");
    if (n > 0 && (!d_ct || !d_pt_ntt || !h_slot)) return set_error(HC_ERR_INVALID_ARG, "null input");
    if (n > 0xffffffffull || n_out > 0xffffffffull) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    std::vector<uint32_t> count(n_out, 0);
    for (size_t j = 0; j < n; ++j) {
        if (h_slot[j] >= n_out) return set_error(HC_ERR_INVALID_ARG, "slot[%zu] = %u >= n_out", j, h_slot[j]);
        ++count[h_slot[j]];
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = as_stream(cuda_stream);
    hc_status st = check_inputs(ctx, d_ct, 2 * n, s);
    if (st == HC_OK) st = check_inputs(ctx, d_pt_ntt, n, s);
    if (st != HC_OK) return st;
    const size_t ct_words = (size_t)2 * ctx->L * ctx->N;
    const bool single = std::all_of(count.begin(), count.end(), [](uint32_t c) { return c <= 1; });

    if (single) {
        // every slot has at most one product: fused NTT -> product -> INTT per product
        if (n < n_out) HC_CUDA_TRY(cudaMemsetAsync(d_out, 0, n_out * ct_words * sizeof(uint64_t), s));
        ScratchGuard idx(s);
        idx.p = dev_alloc(n * sizeof(uint32_t), s);
        if (!idx.p) return set_error(HC_ERR_OOM, "slot list allocation failed");
        if (n) HC_CUDA_TRY(cudaMemcpyAsync(idx.p, h_slot, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        return launch_product(ctx, d_ct, d_pt_ntt, (const uint32_t *)idx.p, d_out, n, false, s);
    }

    // general case: NTT all ciphertexts once, then per slot MAC + INTT
    std::vector<uint32_t> term_ptr(n_out + 1, 0), terms(2 * n);
    for (size_t o = 0; o < n_out; ++o) term_ptr[o + 1] = term_ptr[o] + count[o];
    std::vector<uint32_t> fill(term_ptr.begin(), term_ptr.end() - 1);
    for (size_t j = 0; j < n; ++j) {
        const uint32_t t = fill[h_slot[j]]++;
        terms[2 * t] = (uint32_t)j;
        terms[2 * t + 1] = (uint32_t)j;
    }
    ScratchGuard ctn(s), tp(s), tm(s);
    ctn.p = dev_alloc(n * ct_words * sizeof(uint64_t), s);
    tp.p = dev_alloc(term_ptr.size() * 4, s);
    tm.p = dev_alloc(terms.size() * 4, s);
    if (!ctn.p || !tp.p || !tm.p) return set_error(HC_ERR_OOM, "scratch allocation failed");
    HC_CUDA_TRY(cudaMemcpyAsync(tp.p, term_ptr.data(), term_ptr.size() * 4, cudaMemcpyHostToDevice, s));
    HC_CUDA_TRY(cudaMemcpyAsync(tm.p, terms.data(), terms.size() * 4, cudaMemcpyHostToDevice, s));
    st = launch_ntt_fwd_ct(ctx, d_ct, (uint64_t *)ctn.p, n, s);
    if (st != HC_OK) return st;
    return launch_mac_intt(ctx, (const uint64_t *)ctn.p, d_pt_ntt,
                           MacTerms{(const uint32_t *)tp.p, (const uint32_t *)tm.p}, d_out, n_out, s);
}

void hc_free(void *handle)
{
    if (!handle) return;
    const uint32_t magic = *(const uint32_t *)handle;
    if (magic == kMagicCtx) {
        hc_ctx *c = (hc_ctx *)handle;
        DeviceGuard g(c->device);
        dev_free_persistent(c->d_tables);
        dev_free_persistent(c->d_limbs);
        dev_free_persistent(c->d_flag);
        c->magic = kMagicDead;
        delete c;
    } else if (magic == kMagicPlan) {
        plan_destroy((hc_plan *)handle);
    } else if (magic == kMagicServer) {
        server_destroy((hc_server *)handle);
    } else if (magic == kMagicGaloisKey) {
        galois_key_destroy((hc_galois_key *)handle);
    } else if (magic == kMagicWeights) {
        hc_weights *w = (hc_weights *)handle;
        DeviceGuard g(w->device);
        dev_free_persistent(w->d_pt);
        dev_free_persistent(w->d_k);
        dev_free_persistent(w->d_term_ptr);
        dev_free_persistent(w->d_terms);
        dev_free_persistent(w->d_slot_table);
        w->magic = kMagicDead;
        delete w;
    }
}

}  // extern "C"
