// hc_launch.cu -- dispatch of the public launchers to the per-N kernel
// instantiations and the launch variant recorded in the context, plus the
// small elementwise kernels (weight lifting, range checks) and the blocked
// convolution MAC.
#include <atomic>
#include <vector>

#include "hc_arith.cuh"
#include "hc_async.cuh"
#include "hc_internal.h"
#include "hc_mac.cuh"

namespace hc {

static hc_status after_launch_status(const char *what)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HC_OK : cuda_error(e, what);
}

// ---------------------------------------------------------------------------
__global__ void k_lift_int8(const int8_t *__restrict__ packed, uint64_t *__restrict__ out,
                            const LimbConst *__restrict__ limbs, uint32_t L, uint32_t N, size_t n_polys)
{
    const size_t total = n_polys * L * N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t k = i % N;
        const size_t l = (i / N) % L;
        const size_t p = i / ((size_t)N * L);
        const int v = packed[p * N + k];
        const uint64_t q = limbs[l].q;
        out[i] = v >= 0 ? (uint64_t)v : q - (uint64_t)(-v);
    }
}

__global__ void k_range_check(const uint64_t *__restrict__ p, const LimbConst *__restrict__ limbs,
                              uint32_t L, uint32_t N, size_t n_polys, int *flag)
{
    const size_t total = n_polys * L * N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t l = (i / N) % L;
        if (p[i] >= limbs[l].q) {
            *flag = 1;
            return;
        }
    }
}


// Launch shapes a context starts with (the autotuner may change them).  Measured
// on GB300: at N >= 8192 the forward transforms run fastest as two-CTA clusters
// and the inverse ones as the persistent prefetching kernel (variant 2 of both),
// for a few polynomials (latency) and for a layer's hundreds (throughput) alike.
int default_variant(int kind, uint32_t logn)
{
    if (logn >= 13 && (kind == KK_FWD || kind == KK_FWDCT || kind == KK_INV || kind == KK_INVCT)) return 2;
    return 0;
}

// ---------------------------------------------------------------------------
// Blocked convolution MAC (the task in hc_mac.cuh): one task per CTA; the
// CTAs of a launch cover the (chunk, limb, channel group) tasks of every
// segment (layer) of the table.
constexpr int kMacThreads = 256;

template <int KC, int NS>
__global__ void __launch_bounds__(kMacThreads)
k_mac_conv(const __grid_constant__ MacSegsT<NS> segs, int *err)
{
    __shared__ __align__(8) uint64_t bars[1 + kMacStages];
    extern __shared__ __align__(16) uint64_t dsm[];
    uint32_t si = 0;
    while (si + 1 < segs.n && blockIdx.x >= segs.s[si + 1].cta_begin) ++si;
    const MacSeg &sg = segs.s[si];
    const uint32_t local = blockIdx.x - sg.cta_begin;
    const uint32_t chunk = local % sg.chunks, rest = local / sg.chunks;
    const uint32_t lc = seg_limbs(sg);
    const uint32_t limb = sg.limb0 + rest % lc;
    const uint32_t m0 = (rest / lc) * sg.MB, m1 = min(sg.M, m0 + sg.MB);
    if (threadIdx.x == 0) {
        for (int i = 0; i < 1 + kMacStages; ++i) mbar_init(&bars[i], 1);
        mbar_fence_init();
    }
    __syncthreads();
    MacRing ring{0, 0};
    mac_task<KC, kMacThreads>(sg, chunk, limb, m0, m1, dsm, bars, ring, err);
}

// launch variants of the blocked MAC: (slots per chunk, weight rows per stage)
constexpr uint32_t kMacVariantKC[kNumVariants] = {64, 64, 64};
constexpr uint32_t kMacStageRows[kNumVariants] = {8, 16, 32};
constexpr size_t kMacSmemCap = 200 * 1024;

static size_t mac_smem(uint32_t G, uint32_t B, uint32_t MS, uint32_t kc)
{
    return ((size_t)G * 2 * B + (size_t)kMacStages * MS * G) * kc * sizeof(uint64_t);
}

// channels per stage: about the variant's stage rows, within the shared-memory cap
static uint32_t mac_stage_channels(uint32_t G, uint32_t B, uint32_t M, int variant, uint32_t kc)
{
    uint32_t ms = kMacStageRows[variant] / G;
    if (ms < 1) ms = 1;
    if (ms > M) ms = M;
    while (ms > 1 && mac_smem(G, B, ms, kc) > kMacSmemCap / 2) --ms;  // keep two CTAs per SM where possible
    return ms;
}

// fill the launch geometry of one segment: enough CTAs for about `waves` waves of
// the layer's full work (all L limbs)
MacSeg make_mac_seg(const hc_ctx *ctx, const uint64_t *x, const uint64_t *w, uint64_t *y, uint32_t G, uint32_t B,
                    uint32_t M, uint32_t kc, uint32_t waves)
{
    int v = ctx->variant[KK_MACB];
    if (v >= kNumVariants) v = 1;  // shapes the tensor-core MAC does not take: stages of 16 rows
    if (kc == 0) kc = kMacVariantKC[v];
    MacSeg sg{};
    sg.X = x;
    sg.W = w;
    sg.Y = y;
    sg.limbs = ctx->d_limbs;
    sg.N = ctx->N;
    sg.L = ctx->L;
    sg.G = G;
    sg.B = B;
    sg.M = M;
    sg.KC = kc;
    sg.MS = mac_stage_channels(G, B, M, v, kc);
    const size_t smem = mac_smem(G, B, sg.MS, kc);
    const uint32_t per_sm = (uint32_t)(kMacSmemCap / smem) < 4 ? (uint32_t)(kMacSmemCap / smem) : 4;
    sg.chunks = ctx->N / kc;
    const uint32_t target = ctx->sms * (per_sm ? per_sm : 1) * waves;
    const uint32_t want = (target + sg.chunks * ctx->L - 1) / (sg.chunks * ctx->L);
    const uint32_t groups = want < 1 ? 1 : (want > M ? M : want);
    sg.MB = (M + groups - 1) / groups;
    sg.MB = (sg.MB + sg.MS - 1) / sg.MS * sg.MS;  // whole stages per CTA
    sg.groups = (M + sg.MB - 1) / sg.MB;
    return sg;
}

template <int KC, int NS>
static hc_status run_mac_segs_kc(MacSegsT<NS> &segs, size_t smem, int *err, cudaStream_t s)
{
    static std::atomic<uint32_t> attr_done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(attr_done.load() & (1u << (dev & 31)))) {
        cudaError_t e = cudaFuncSetAttribute(k_mac_conv<KC, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kMacSmemCap);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(k_mac_conv)");
        attr_done.fetch_or(1u << (dev & 31));
    }
    uint32_t begin = 0;
    for (uint32_t i = 0; i < segs.n; ++i) {
        segs.s[i].cta_begin = begin;
        begin += segs.s[i].chunks * seg_limbs(segs.s[i]) * segs.s[i].groups;
    }
    if (begin == 0) return HC_OK;
    ProfileScope ps("k_mac_conv", s);
    k_mac_conv<KC, NS><<<begin, kMacThreads, smem, s>>>(segs, err);
    return after_launch_status("k_mac_conv");
}

// every segment of one launch has the same chunk width
template <int NS>
static hc_status run_mac_segs(MacSegsT<NS> &segs, size_t smem, int *err, cudaStream_t s)
{
    return segs.s[0].KC == 32 ? run_mac_segs_kc<32, NS>(segs, smem, err, s)
                              : run_mac_segs_kc<64, NS>(segs, smem, err, s);
}

size_t mac_seg_smem(const MacSeg &sg)
{
    return mac_smem(sg.G, sg.B, sg.MS, sg.KC);
}

bool mac_conv_fits(uint32_t G, uint32_t B)
{
    return mac_smem(G, B, 1, 64) <= kMacSmemCap;
}

hc_status launch_mac_conv(const hc_ctx *ctx, const uint64_t *x_ntt, const uint64_t *w_ntt, uint64_t *y, uint32_t G,
                          uint32_t B, uint32_t M, cudaStream_t s)
{
    if (ctx->variant[KK_MACB] == kMacTcVariant && mac_tc_fits(G, B))
        return launch_mac_tc(ctx, x_ntt, w_ntt, y, G, B, M, 0, 0, s);
    if (!mac_conv_fits(G, B) || ctx->N % 64) return set_error(HC_ERR_UNSUPPORTED, "blocked MAC does not fit");
    MacSegs1 segs{};
    segs.n = 1;
    segs.s[0] = make_mac_seg(ctx, x_ntt, w_ntt, y, G, B, M);
    return run_mac_segs(segs, mac_seg_smem(segs.s[0]), timeout_flag(ctx), s);
}

static bool use_tc(const hc_ctx *ctx, const MacLayer &ly)
{
    return ctx->variant[KK_MACB] == kMacTcVariant && mac_tc_fits(ly.G, ly.B);
}

hc_status launch_mac_conv_layers(const hc_ctx *const *ctxs, const MacLayer *layers, size_t n, cudaStream_t s)
{
    // layers the tensor-core MAC takes: one launch each; the others share blocked launches
    std::vector<size_t> rest;
    for (size_t i = 0; i < n; ++i) {
        if (!use_tc(ctxs[i], layers[i])) {
            rest.push_back(i);
            continue;
        }
        const MacLayer &ly = layers[i];
        hc_status st = launch_mac_tc(ctxs[i], ly.x, ly.w, ly.y, ly.G, ly.B, ly.M, ly.limb0, ly.Lc, s);
        if (st != HC_OK) return st;
    }
    for (size_t r0 = 0; r0 < rest.size(); r0 += kMaxSegs) {
        MacSegs segs{};
        size_t smem = 0;
        const size_t r1 = r0 + kMaxSegs < rest.size() ? r0 + kMaxSegs : rest.size();
        const size_t i0 = rest[r0];
        const int v0 = ctxs[i0]->variant[KK_MACB];
        const uint32_t kc = kMacVariantKC[v0 < kNumVariants ? v0 : 1];  // one chunk width per launch
        for (size_t ri = r0; ri < r1; ++ri) {
            const size_t i = rest[ri];
            const MacLayer &ly = layers[i];
            if (!mac_conv_fits(ly.G, ly.B)) return set_error(HC_ERR_UNSUPPORTED, "blocked MAC does not fit");
            // one limb's launch of the per-limb chains runs beside the other limbs' MACs:
            // fewer, longer CTAs (each loads its input chunk once for more channels)
            // measured faster there (2 waves: 0.240 vs 0.250 ms on the 56x56x64 layer)
            segs.s[segs.n] = make_mac_seg(ctxs[i], ly.x, ly.w, ly.y, ly.G, ly.B, ly.M, kc, ly.Lc ? 2 : 4);
            segs.s[segs.n].Lc = ly.Lc;
            segs.s[segs.n].limb0 = ly.limb0;
            const size_t sm = mac_seg_smem(segs.s[segs.n++]);
            if (sm > smem) smem = sm;
        }
        hc_status st = run_mac_segs(segs, smem, timeout_flag(ctxs[i0]), s);
        if (st != HC_OK) return st;
    }
    return HC_OK;
}

// Self-test of the bounded-wait error path: one CTA waits on an mbarrier that
// nothing ever arrives at, gives up after `limit` attempts, records the
// timeout in the context's device flag and returns.
__global__ void k_wait_selftest(uint32_t limit, int *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, limit);
    if (!ok && threadIdx.x == 0) atomicExch(err, 3);
}

hc_status launch_wait_selftest(const hc_ctx *ctx, uint32_t limit, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(limit, timeout_flag(ctx));
    return after_launch_status("k_wait_selftest");
}

namespace {

hc_status after(const char *what)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HC_OK : cuda_error(e, what);
}

hc_status dispatch(const hc_ctx *ctx, int kind, const LaunchArgs &a, cudaStream_t s)
{
    const int v = kind == KK_FWDCT_SEGS    ? ctx->variant[KK_FWDCT]
                  : kind == KK_INVCT_SEGS  ? ctx->variant[KK_INVCT]
                  : kind == KK_INV_EXTRACT ? ctx->variant[KK_INVCT]
                                           : ctx->variant[kind];
    switch (ctx->logN) {
    case 12: return launch_n<12>(ctx, kind, v, a, s);
    case 13: return launch_n<13>(ctx, kind, v, a, s);
    case 14: return launch_n<14>(ctx, kind, v, a, s);
    default: return set_error(HC_ERR_UNSUPPORTED, "unsupported N = %u", ctx->N);
    }
}

}  // namespace

hc_status launch_ntt_fwd(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_polys, cudaStream_t s)
{
    LaunchArgs a{};
    a.in = in;
    a.out = out;
    a.n = n_polys;
    return dispatch(ctx, KK_FWD, a, s);
}

hc_status launch_ntt_inv(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_polys, cudaStream_t s)
{
    LaunchArgs a{};
    a.in = in;
    a.out = out;
    a.n = n_polys;
    return dispatch(ctx, KK_INV, a, s);
}

hc_status launch_inv_extract(const hc_ctx *ctx, const ExtractArgs &ex, cudaStream_t s)
{
    LaunchArgs a{};
    a.ex = &ex;
    return dispatch(ctx, KK_INV_EXTRACT, a, s);
}

hc_status launch_ntt_fwd_ct(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_ct, cudaStream_t s)
{
    LaunchArgs a{};
    a.in = in;
    a.out = out;
    a.n = n_ct;
    return dispatch(ctx, KK_FWDCT, a, s);
}

hc_status launch_ntt_inv_ct(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_ct, cudaStream_t s)
{
    LaunchArgs a{};
    a.in = in;
    a.out = out;
    a.n = n_ct;
    return dispatch(ctx, KK_INVCT, a, s);
}

hc_status launch_ntt_ct_segs(const hc_ctx *ctx, const NttSegs &segs, bool inverse, cudaStream_t s)
{
    LaunchArgs a{};
    a.segs = &segs;
    return dispatch(ctx, inverse ? KK_INVCT_SEGS : KK_FWDCT_SEGS, a, s);
}

hc_status launch_mac_intt(const hc_ctx *ctx, const uint64_t *ct_ntt, const uint64_t *pt_ntt, MacTerms terms,
                          uint64_t *out, size_t n_out, cudaStream_t s)
{
    LaunchArgs a{};
    a.in = ct_ntt;
    a.pt = pt_ntt;
    a.terms = terms;
    a.out = out;
    a.n = n_out;
    return dispatch(ctx, KK_MAC, a, s);
}

hc_status launch_product(const hc_ctx *ctx, const uint64_t *ct, const uint64_t *pt_ntt, const uint32_t *out_index,
                         uint64_t *out, size_t n, bool accumulate, cudaStream_t s)
{
    LaunchArgs a{};
    a.in = ct;
    a.pt = pt_ntt;
    a.out_index = out_index;
    a.out = out;
    a.n = n;
    a.accumulate = accumulate;
    return dispatch(ctx, KK_PROD, a, s);
}

hc_status launch_lift_int8(const hc_ctx *ctx, const int8_t *packed, uint64_t *out, size_t n_polys, cudaStream_t s)
{
    if (n_polys == 0) return HC_OK;
    const size_t total = n_polys * ctx->L * ctx->N;
    const size_t cap = (size_t)ctx->sms * 32;
    const unsigned blocks = (unsigned)((total + 255) / 256 < cap ? (total + 255) / 256 : cap);
    ProfileScope ps("k_lift_int8", s);
    k_lift_int8<<<blocks, 256, 0, s>>>(packed, out, ctx->d_limbs, ctx->L, ctx->N, n_polys);
    return after("k_lift_int8");
}

hc_status launch_range_check(const hc_ctx *ctx, const uint64_t *p, size_t n_polys, int *flag, cudaStream_t s)
{
    if (n_polys == 0) return HC_OK;
    const size_t total = n_polys * ctx->L * ctx->N;
    const size_t cap = (size_t)ctx->sms * 16;
    const unsigned blocks = (unsigned)((total + 255) / 256 < cap ? (total + 255) / 256 : cap);
    ProfileScope ps("k_range_check", s);
    k_range_check<<<blocks, 256, 0, s>>>(p, ctx->d_limbs, ctx->L, ctx->N, n_polys, flag);
    return after("k_range_check");
}

}  // namespace hc
