// hc_plan.cu -- plans: one batched launch sequence over many conv layers and
// standalone products of any supported ring degree, captured into a CUDA
// graph and replayed; the plain one-launch-per-product form of the same work;
// and the plan autotuner (launch-shape variants timed on the plan itself).
//
// The arithmetic is the one of Sec. 6.2 / App. C.1 (NTT -> NTT-domain MAC ->
// INTT); batching only changes how many launches carry it.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hc_internal.h"

using namespace hc;

namespace {

using PlanConv = ConvJob;

struct PlanProd {
    const hc_ctx *ctx;
    const uint64_t *ct;
    const uint64_t *pt;
    uint64_t *out;
    size_t n;
};

}  // namespace

struct hc_plan {
    uint32_t magic;
    int device;
    std::vector<PlanConv> convs;
    std::vector<PlanProd> prods;
    std::vector<const hc_ctx *> ctxs;   // distinct contexts, first-use order
    void *d_scratch = nullptr;          // conv NTT'd inputs
    uint32_t *d_ctr = nullptr;          // dependency counters of the fused form
    size_t ctr_words = 0;
    void *d_mix = nullptr;              // MixItem[] | units[] | counter
    MixItem *d_items = nullptr;
    uint32_t *d_units = nullptr;
    uint32_t *d_next = nullptr;
    uint32_t n_units = 0;
    uint64_t n_products = 0, alg_bytes = 0;
    uint32_t n_launches = 0;
    uint32_t runs = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
inline bool ctx_ok(const hc_ctx *c) { return c && c->magic == kMagicCtx; }
inline bool weights_ok(const hc_weights *w) { return w && w->magic == kMagicWeights; }
inline bool plan_ok(const hc_plan *p) { return p && p->magic == kMagicPlan; }

size_t ct_words(const hc_ctx *c) { return (size_t)2 * c->L * c->N; }

// ---- overlap check ----------------------------------------------------------
struct Span {
    uintptr_t b, e;
    size_t item;
    int role;  // 0 input ct, 1 input pt, 2 output
};

hc_status check_overlaps(const std::vector<hc_work_item> &items)
{
    std::vector<Span> sp;
    for (size_t i = 0; i < items.size(); ++i) {
        const hc_work_item &it = items[i];
        const size_t cw = ct_words(it.ctx) * 8;
        size_t nin, nout;
        if (it.kind == HC_WORK_CONV) {
            nin = it.weights->I;
            nout = it.weights->O;
        } else {
            nin = nout = it.n;
            const uintptr_t pb = (uintptr_t)it.d_pt_ntt;
            sp.push_back(Span{pb, pb + it.n * (size_t)it.ctx->L * it.ctx->N * 8, i, 1});
        }
        const uintptr_t ib = (uintptr_t)it.d_ct_in, ob = (uintptr_t)it.d_ct_out;
        sp.push_back(Span{ib, ib + nin * cw, i, 0});
        sp.push_back(Span{ob, ob + nout * cw, i, 2});
    }
    std::sort(sp.begin(), sp.end(), [](const Span &a, const Span &b) { return a.b < b.b; });
    std::vector<Span> active;
    for (const Span &cur : sp) {
        active.erase(std::remove_if(active.begin(), active.end(), [&](const Span &a) { return a.e <= cur.b; }),
                     active.end());
        for (const Span &a : active) {
            if (a.role != 2 && cur.role != 2) continue;  // inputs may be shared
            if (a.item != cur.item)
                return set_error(HC_ERR_INVALID_ARG, "items %zu and %zu overlap (an output is involved)", a.item,
                                 cur.item);
            const hc_work_item &it = items[a.item];
            const bool in_out = (a.role == 0 && cur.role == 2) || (a.role == 2 && cur.role == 0);
            if (it.kind == HC_WORK_CONV && in_out) continue;  // all inputs are read before any output is written
            if (it.kind == HC_WORK_PRODUCTS && in_out && a.b == cur.b) continue;  // exactly in place
            return set_error(HC_ERR_INVALID_ARG, "item %zu: output partially overlaps its inputs", a.item);
        }
        active.push_back(cur);
    }
    return HC_OK;
}

// ---- the batched launch sequence ---------------------------------------------
hc_status run_batched(hc_plan *p, cudaStream_t s)
{
    hc_status st = launch_conv_jobs(p->convs.data(), p->convs.size(), s, p->d_ctr, p->ctr_words);
    if (st != HC_OK) return st;
    // every standalone product, one persistent launch
    if (p->n_units) {
        HC_CUDA_TRY(cudaMemsetAsync(p->d_next, 0, sizeof(uint32_t), s));
        st = launch_product_mixed(p->d_items, p->d_units, p->n_units, p->d_next, s);
        if (st != HC_OK) return st;
    }
    return HC_OK;
}

// kernels one batched run launches (the fused form counts one per degree)
uint32_t count_launches(const hc_plan *p)
{
    uint32_t n = 0, fit = 0;
    uint32_t per_n[3] = {0, 0, 0}, per_n_fit[3] = {0, 0, 0};
    bool fused[3] = {false, false, false};
    for (int d = 0; d < 3; ++d) {
        uint32_t cnt = 0;
        const PlanConv *first = nullptr;
        for (const PlanConv &c : p->convs)
            if (c.ctx->logN == (uint32_t)(12 + d) && c.blocked) {
                if (!first) first = &c;
                ++cnt;
            }
        fused[d] = first && first->ctx->variant[KK_CONV] == 1 && cnt <= (uint32_t)kFusedMaxLayers && p->d_ctr;
        if (fused[d]) ++n;
        if (first && first->ctx->variant[KK_CONV] == 2 && !fused[d]) {
            uint32_t maxl = 0;
            for (const PlanConv &c : p->convs)
                if (c.ctx->logN == (uint32_t)(12 + d) && c.blocked && c.ctx->L > maxl) maxl = c.ctx->L;
            n += 3 * maxl * ((cnt + kMaxSegs - 1) / kMaxSegs);
            fused[d] = true;  // counted here, not below
        }
    }
    for (const PlanConv &c : p->convs) {
        if (c.blocked && fused[c.ctx->logN - 12]) continue;
        ++per_n[c.ctx->logN - 12];
        if (c.blocked) {
            ++per_n_fit[c.ctx->logN - 12];
            ++fit;
        } else {
            ++n;  // fused MAC + INTT
        }
    }
    for (int i = 0; i < 3; ++i) n += (per_n[i] + kMaxSegs - 1) / kMaxSegs + (per_n_fit[i] + kMaxSegs - 1) / kMaxSegs;
    n += (fit + kMaxSegs - 1) / kMaxSegs;
    if (p->n_units) ++n;
    return n;
}

hc_status check_plan_inputs(hc_plan *p, cudaStream_t s)
{
    for (const PlanConv &c : p->convs) {
        hc_status st = check_inputs(c.ctx, c.in, (size_t)2 * c.w->I, s);
        if (st != HC_OK) return st;
    }
    for (const PlanProd &q : p->prods) {
        hc_status st = check_inputs(q.ctx, q.ct, 2 * q.n, s);
        if (st == HC_OK) st = check_inputs(q.ctx, q.pt, q.n, s);
        if (st != HC_OK) return st;
    }
    return HC_OK;
}

void drop_graph(hc_plan *p)
{
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
}

hc_status capture(hc_plan *p)
{
    if (!p->cap_stream) HC_CUDA_TRY(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    HC_CUDA_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    hc_status st = run_batched(p, p->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
    if (st != HC_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&p->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        p->exec = nullptr;
        return cuda_error(e, "cudaGraphInstantiate");
    }
    p->graph = g;
    return HC_OK;
}

// ---- autotuner ------------------------------------------------------------------
// signature of the work a plan runs (shapes only, not addresses): tuned
// choices depend on the layer mix, so they are cached per signature
uint64_t plan_signature(const hc_plan *p)
{
    uint64_t h = 1469598103934665603ull;  // FNV-1a
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (v >> (8 * i)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    for (const PlanConv &c : p->convs) {
        mix(c.ctx->N);
        mix(c.ctx->L);
        mix(c.w->G);
        mix(c.w->B);
        mix(c.w->Mp);
        mix(c.w->I);
        mix(c.w->O);
    }
    for (const PlanProd &q : p->prods) {
        mix(q.ctx->N | (uint64_t)q.ctx->L << 32);
        mix(q.n);
    }
    return h;
}

std::string tune_key(const hc_ctx *c, int kind, const char *gpu, int sms, uint64_t sig)
{
    std::string k = gpu;
    for (char &ch : k)
        if (ch == ' ' || ch == '\t') ch = '_';
    char buf[64];
    snprintf(buf, sizeof buf, "|sm%d|N%u|L%u", sms, c->N, c->L);
    k += buf;
    for (uint32_t i = 0; i < c->L; ++i) {
        snprintf(buf, sizeof buf, "|%llx", (unsigned long long)c->q[i]);
        k += buf;
    }
    snprintf(buf, sizeof buf, "|work%016llx|kind%d", (unsigned long long)sig, kind);
    return k + buf;
}

// median device time (ms) of `reps` batched runs on s
hc_status time_batched(hc_plan *p, cudaStream_t s, int reps, float *ms)
{
    cudaEvent_t a = nullptr, b = nullptr;
    HC_CUDA_TRY(cudaEventCreate(&a));
    cudaError_t e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return cuda_error(e, "cudaEventCreate");
    }
    std::vector<float> t;
    hc_status st = run_batched(p, s);  // warm-up with this variant
    for (int r = 0; st == HC_OK && r < reps; ++r) {
        cudaEventRecord(a, s);
        st = run_batched(p, s);
        cudaEventRecord(b, s);
        if (st != HC_OK) break;
        e = cudaEventSynchronize(b);
        float x = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&x, a, b);
        if (e != cudaSuccess) st = cuda_error(e, "autotune timing");
        t.push_back(x);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != HC_OK) return st;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return HC_OK;
}

}  // namespace

namespace hc {
bool conv_job_blocked(const hc_ctx *c, const hc_weights *w) { return mac_conv_fits(w->G, w->B) && c->N % 64 == 0; }

namespace {
thread_local int *t_flag = nullptr;
thread_local SidePool *t_side = nullptr;
}  // namespace

int *timeout_flag(const hc_ctx *ctx) { return t_flag ? t_flag : ctx->d_flag + 1; }
SidePool *side_override() { return t_side; }

LaunchScope::LaunchScope(int *flag, SidePool *side) : prev_flag_(t_flag), prev_side_(t_side)
{
    if (flag) t_flag = flag;
    if (side) t_side = side;
}

LaunchScope::~LaunchScope()
{
    t_flag = prev_flag_;
    t_side = prev_side_;
}

// side streams and events for fork / join: the LaunchScope's pool if one is set,
// else one per host thread and device (made once, kept); grown to `need` streams
hc_status side_pool(uint32_t need, SidePool **out)
{
    static thread_local SidePool pools[32];
    int dev = 0;
    HC_CUDA_TRY(cudaGetDevice(&dev));
    SidePool &p = t_side ? *t_side : pools[dev & 31];
    if (p.ev.empty()) {
        cudaEvent_t e = nullptr;
        HC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p.ev.push_back(e);
    }
    while (p.st.size() < need) {
        cudaStream_t st = nullptr;
        cudaEvent_t e = nullptr;
        HC_CUDA_TRY(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, p.priority));
        p.st.push_back(st);
        HC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p.ev.push_back(e);
    }
    *out = &p;
    return HC_OK;
}

// Limbs are independent through all three phases, so the blocked jobs of one
// degree split into one forward -> MAC -> inverse chain per limb; the chains run
// on parallel streams (parallel branches under graph capture), and the tail
// of one chain's kernel overlaps the next kernels of the others.
hc_status launch_limb_chains(const ConvJob *jobs, size_t n, uint32_t logN, cudaStream_t s)
{
    uint32_t maxl = 0;
    for (size_t i = 0; i < n; ++i)
        if (jobs[i].ctx->logN == logN && jobs[i].blocked && jobs[i].ctx->L > maxl) maxl = jobs[i].ctx->L;
    if (!maxl) return HC_OK;
    SidePool *pool = nullptr;
    hc_status st = side_pool(maxl - 1, &pool);
    if (st != HC_OK) return st;
    HC_CUDA_TRY(cudaEventRecord(pool->ev[0], s));
    for (uint32_t l = 1; l < maxl; ++l) HC_CUDA_TRY(cudaStreamWaitEvent(pool->st[l - 1], pool->ev[0], 0));
    for (uint32_t l = 0; l < maxl; ++l) {
        cudaStream_t sl = l == 0 ? s : pool->st[l - 1];
        for (size_t i0 = 0; i0 < n;) {  // at most kMaxSegs jobs per launch
            const size_t i0_begin = i0;
            NttSegs fwd{}, inv{};
            std::vector<const hc_ctx *> mctx;
            std::vector<MacLayer> layers;
            const hc_ctx *first = nullptr;
            size_t i = i0;
            for (; i < n && fwd.n < (uint32_t)kMaxSegs; ++i) {
                const ConvJob &c = jobs[i];
                if (c.ctx->logN != logN || !c.blocked || c.ctx->L <= l) continue;
                if (!first) first = c.ctx;
                NttSeg f{c.in, c.ntt, c.ctx->d_limbs, c.ctx->L, c.w->I, 0};
                f.Lc = 1;
                f.limb0 = l;
                fwd.s[fwd.n++] = f;
                if (!c.ex) {
                    NttSeg v{c.out, c.out, c.ctx->d_limbs, c.ctx->L, c.w->O, 0};
                    v.Lc = 1;
                    v.limb0 = l;
                    inv.s[inv.n++] = v;
                }
                MacLayer ly{c.ntt, job_weights(c), c.out, c.w->G, c.w->B, c.w->Mp};
                ly.Lc = 1;
                ly.limb0 = l;
                mctx.push_back(c.ctx);
                layers.push_back(ly);
            }
            i0 = i;
            if (!first) continue;
            st = launch_ntt_ct_segs(first, fwd, false, sl);
            if (st == HC_OK) st = launch_mac_conv_layers(mctx.data(), layers.data(), layers.size(), sl);
            if (st == HC_OK && inv.n) st = launch_ntt_ct_segs(first, inv, true, sl);
            for (size_t j = i0_begin; st == HC_OK && j < i; ++j) {  // the server step's epilogue, per job
                const ConvJob &c = jobs[j];
                if (!c.ex || c.ctx->logN != logN || !c.blocked || c.ctx->L <= l) continue;
                ExtractArgs ex = *c.ex;
                ex.limb0 = l;
                ex.Lc = 1;
                st = launch_inv_extract(c.ctx, ex, sl);
            }
            if (st != HC_OK) return st;
        }
        if (l > 0) HC_CUDA_TRY(cudaEventRecord(pool->ev[l], sl));
    }
    for (uint32_t l = 1; l < maxl; ++l) HC_CUDA_TRY(cudaStreamWaitEvent(s, pool->ev[l], 0));
    return HC_OK;
}

size_t conv_jobs_counter_words(const ConvJob *jobs, size_t n)
{
    size_t w = 0;
    for (uint32_t logN = 12; logN <= 14; ++logN) {
        const size_t x = fused_counter_words(jobs, n, logN);
        if (x > w) w = x;
    }
    return w;
}

// the batched launch sequence of n conv jobs (all degrees), in stream order on s
hc_status launch_conv_jobs(const ConvJob *jobs, size_t n, cudaStream_t s, uint32_t *ctr, size_t ctr_words)
{
    // degrees whose blocked jobs run as one fused persistent launch
    bool fused[3] = {false, false, false};
    for (uint32_t logN = 12; logN <= 14; ++logN) {
        const ConvJob *first = nullptr;
        size_t count = 0;
        for (size_t i = 0; i < n; ++i)
            if (jobs[i].ctx->logN == logN && jobs[i].blocked) {
                if (!first) first = &jobs[i];
                ++count;
            }
        if (!first) continue;
        if (first->ctx->variant[KK_CONV] == 2) {
            hc_status st = launch_limb_chains(jobs, n, logN, s);
            if (st != HC_OK) return st;
            fused[logN - 12] = true;
            continue;
        }
        if (first->ctx->variant[KK_CONV] != 1 || count > (size_t)kFusedMaxLayers || !ctr) continue;
        const size_t words = fused_counter_words(jobs, n, logN);
        if (words > ctr_words) continue;
        hc_status st = launch_conv_fused(jobs, n, logN, ctr, s);
        if (st != HC_OK) return st;
        fused[logN - 12] = true;
    }
    if (n == 1 && !fused[jobs[0].ctx->logN - 12] && jobs[0].ctx->variant[KK_CONV] != 2) {
        // one layer: the single-segment launchers (small parameter blocks, no host tables)
        const ConvJob &c = jobs[0];
        hc_status st = launch_ntt_fwd_ct(c.ctx, c.in, c.ntt, c.w->I, s);
        if (st != HC_OK) return st;
        if (!c.blocked)
            return launch_mac_intt(c.ctx, c.ntt, job_weights(c), MacTerms{c.w->d_term_ptr, c.w->d_terms}, c.out, c.w->O,
                                   s);
        st = launch_mac_conv(c.ctx, c.ntt, job_weights(c), c.out, c.w->G, c.w->B, c.w->Mp, s);
        if (st != HC_OK) return st;
        return launch_ntt_inv_ct(c.ctx, c.out, c.out, c.w->O, s);
    }
    auto done = [&](const ConvJob &c) { return c.blocked && fused[c.ctx->logN - 12]; };
    // forward NTT of every other conv input, one launch per ring degree (per kMaxSegs jobs)
    for (uint32_t logN = 12; logN <= 14; ++logN) {
        NttSegs segs{};
        const hc_ctx *first = nullptr;
        for (size_t i = 0; i <= n; ++i) {
            if (i < n) {
                const ConvJob &c = jobs[i];
                if (c.ctx->logN != logN || done(c)) continue;
                if (!first) first = c.ctx;
                segs.s[segs.n++] = NttSeg{c.in, c.ntt, c.ctx->d_limbs, c.ctx->L, c.w->I, 0};
            }
            if (segs.n && (segs.n == kMaxSegs || i == n)) {
                hc_status st = launch_ntt_ct_segs(first, segs, false, s);
                if (st != HC_OK) return st;
                segs.n = 0;
                first = nullptr;
            }
        }
    }
    // NTT-domain MAC of every job with a blocked MAC, one launch (per kMaxSegs jobs)
    std::vector<const hc_ctx *> mctx;
    std::vector<MacLayer> layers;
    for (size_t i = 0; i < n; ++i) {
        const ConvJob &c = jobs[i];
        if (done(c)) continue;
        if (c.blocked) {
            mctx.push_back(c.ctx);
            layers.push_back(MacLayer{c.ntt, job_weights(c), c.out, c.w->G, c.w->B, c.w->Mp});
        } else {
            hc_status st = launch_mac_intt(c.ctx, c.ntt, job_weights(c), MacTerms{c.w->d_term_ptr, c.w->d_terms}, c.out,
                                           c.w->O, s);
            if (st != HC_OK) return st;
        }
    }
    if (!layers.empty()) {
        hc_status st = launch_mac_conv_layers(mctx.data(), layers.data(), layers.size(), s);
        if (st != HC_OK) return st;
    }
    // inverse NTT of every blocked-MAC output, in place, one launch per ring degree
    for (uint32_t logN = 12; logN <= 14; ++logN) {
        NttSegs segs{};
        const hc_ctx *first = nullptr;
        for (size_t i = 0; i <= n; ++i) {
            if (i < n) {
                const ConvJob &c = jobs[i];
                if (c.ctx->logN != logN || !c.blocked || done(c)) continue;
                if (!first) first = c.ctx;
                segs.s[segs.n++] = NttSeg{c.out, c.out, c.ctx->d_limbs, c.ctx->L, c.w->O, 0};
            }
            if (segs.n && (segs.n == kMaxSegs || i == n)) {
                hc_status st = launch_ntt_ct_segs(first, segs, true, s);
                if (st != HC_OK) return st;
                segs.n = 0;
                first = nullptr;
            }
        }
    }
    return HC_OK;
}

void plan_destroy(hc_plan *p)
{
    DeviceGuard g(p->device);
    drop_graph(p);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    dev_free_persistent(p->d_scratch);
    dev_free_persistent(p->d_mix);
    dev_free_persistent(p->d_ctr);
    p->magic = kMagicDead;
    delete p;
}
}  // namespace hc

// =============================================================================
extern "C" {

hc_status hc_plan_create(const hc_work_item *items, size_t n, hc_plan **out)
{
    if (!out) return set_error(HC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n > 0 && !items) return set_error(HC_ERR_INVALID_ARG, "items is NULL");
    int dev = 0;
    HC_CUDA_TRY(cudaGetDevice(&dev));
    std::vector<hc_work_item> its(items, items + n);
    for (size_t i = 0; i < n; ++i) {
        const hc_work_item &it = its[i];
        if (!ctx_ok(it.ctx)) return set_error(HC_ERR_INVALID_ARG, "item %zu: invalid context", i);
        if (it.ctx->device != dev) return set_error(HC_ERR_INVALID_ARG, "item %zu: context on another device", i);
        if (!it.d_ct_in || !it.d_ct_out) return set_error(HC_ERR_INVALID_ARG, "item %zu: null buffer", i);
        if (it.kind == HC_WORK_CONV) {
            if (!weights_ok(it.weights) || it.weights->ctx != it.ctx)
                return set_error(HC_ERR_INVALID_ARG, "item %zu: weights invalid or of another context", i);
            if (it.weights->mode != HC_WEIGHTS_NTT_OFFLINE)
                return set_error(HC_ERR_UNSUPPORTED, "item %zu: plans need NTT-preprocessed (offline) weights", i);
        } else if (it.kind == HC_WORK_PRODUCTS) {
            if (it.n == 0 || !it.d_pt_ntt) return set_error(HC_ERR_INVALID_ARG, "item %zu: empty product list", i);
        } else {
            return set_error(HC_ERR_INVALID_ARG, "item %zu: unknown kind %u", i, it.kind);
        }
    }
    hc_status st = check_overlaps(its);
    if (st != HC_OK) return st;

    hc_plan *p = new (std::nothrow) hc_plan();
    if (!p) return set_error(HC_ERR_OOM, "host allocation failed");
    p->magic = kMagicPlan;
    p->device = dev;
    size_t scratch_words = 0;
    std::vector<MixItem> mix;
    for (const hc_work_item &it : its) {
        const hc_ctx *c = it.ctx;
        if (std::find(p->ctxs.begin(), p->ctxs.end(), c) == p->ctxs.end()) p->ctxs.push_back(c);
        const uint64_t nl = (uint64_t)c->N * c->L * 8;
        if (it.kind == HC_WORK_CONV) {
            const hc_weights *w = it.weights;
            p->convs.push_back(PlanConv{c, w, it.d_ct_in, it.d_ct_out, nullptr, conv_job_blocked(c, w)});
            scratch_words += (size_t)w->I * ct_words(c);
            p->n_products += (uint64_t)w->Mp * w->G * w->B;
            p->alg_bytes += nl * (2ull * w->I + w->P + 2ull * w->O);
        } else {
            p->prods.push_back(PlanProd{c, it.d_ct_in, it.d_pt_ntt, it.d_ct_out, it.n});
            for (size_t j = 0; j < it.n; ++j)
                mix.push_back(MixItem{it.d_ct_in + j * ct_words(c), it.d_pt_ntt + j * (size_t)c->L * c->N,
                                      it.d_ct_out + j * ct_words(c), c->d_limbs, c->L, c->logN});
            p->n_products += it.n;
            p->alg_bytes += nl * 5ull * it.n;
        }
    }
    if (mix.size() >= (1u << 28)) {
        hc_free(p);
        return set_error(HC_ERR_INVALID_ARG, "more than 2^28 standalone products");
    }
    // units in cost order: larger ring degree first (stable: item order within a degree)
    std::vector<uint32_t> units;
    for (uint32_t logN = 14; logN >= 12; --logN)
        for (uint32_t j = 0; j < mix.size(); ++j) {
            if (mix[j].logN != logN) continue;
            const uint32_t step = mix_comps_per_unit(logN);
            for (uint32_t limb = 0; limb < mix[j].L; ++limb)
                for (uint32_t comp = 0; comp < 2; comp += step) units.push_back(mix_unit(j, limb, comp));
        }
    p->n_units = (uint32_t)units.size();

    for (const PlanConv &c : p->convs) p->ctr_words += conv_counter_bound(c.ctx, c.w);
    if (p->ctr_words) {
        p->d_ctr = (uint32_t *)dev_alloc_persistent(p->ctr_words * sizeof(uint32_t));
        if (!p->d_ctr) {
            hc_free(p);
            return set_error(HC_ERR_OOM, "plan counter allocation failed");
        }
    }
    if (scratch_words) {
        p->d_scratch = dev_alloc_persistent(scratch_words * sizeof(uint64_t));
        if (!p->d_scratch) {
            hc_free(p);
            return set_error(HC_ERR_OOM, "plan scratch allocation failed (%zu bytes)", scratch_words * 8);
        }
        uint64_t *q = (uint64_t *)p->d_scratch;
        for (PlanConv &c : p->convs) {
            c.ntt = q;
            q += (size_t)c.w->I * ct_words(c.ctx);
        }
    }
    if (!mix.empty()) {
        const size_t items_b = (mix.size() * sizeof(MixItem) + 255) & ~(size_t)255;
        const size_t units_b = (units.size() * sizeof(uint32_t) + 255) & ~(size_t)255;
        p->d_mix = dev_alloc_persistent(items_b + units_b + 256);
        if (!p->d_mix) {
            hc_free(p);
            return set_error(HC_ERR_OOM, "plan work-table allocation failed");
        }
        p->d_items = (MixItem *)p->d_mix;
        p->d_units = (uint32_t *)((char *)p->d_mix + items_b);
        p->d_next = (uint32_t *)((char *)p->d_mix + items_b + units_b);
        cudaError_t e = cudaMemcpy(p->d_items, mix.data(), mix.size() * sizeof(MixItem), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_units, units.data(), units.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            hc_free(p);
            return cuda_error(e, "plan work-table upload");
        }
    }
    p->n_launches = count_launches(p);
    *out = p;
    return HC_OK;
}

hc_status hc_plan_run(hc_plan *p, void *cuda_stream)
{
    if (!plan_ok(p)) return set_error(HC_ERR_INVALID_ARG, "invalid plan");
    DeviceGuard g(p->device);
    cudaStream_t s = as_stream(cuda_stream);
    hc_status st = check_plan_inputs(p, s);
    if (st != HC_OK) return st;
    // the first run (and any run while tracing) issues the launches directly;
    // the launch sequence is then captured once and replayed
    if (profile_enabled() || (!p->exec && p->runs == 0)) {
        st = run_batched(p, s);
        if (st == HC_OK) ++p->runs;
        return st;
    }
    if (!p->exec) {
        st = capture(p);
        if (st != HC_OK) return st;
    }
    HC_CUDA_TRY(cudaGraphLaunch(p->exec, s));
    ++p->runs;
    return HC_OK;
}

hc_status hc_plan_run_plain(hc_plan *p, void *cuda_stream)
{
    if (!plan_ok(p)) return set_error(HC_ERR_INVALID_ARG, "invalid plan");
    DeviceGuard g(p->device);
    for (const PlanConv &c : p->convs) {
        hc_status st = hc_conv_ct_pt_plain(c.ctx, c.w, c.in, c.out, cuda_stream);
        if (st != HC_OK) return st;
    }
    cudaStream_t s = as_stream(cuda_stream);
    for (const PlanProd &q : p->prods) {
        hc_status st = check_inputs(q.ctx, q.ct, 2 * q.n, s);
        if (st == HC_OK) st = check_inputs(q.ctx, q.pt, q.n, s);
        if (st != HC_OK) return st;
        const size_t cw = ct_words(q.ctx), pw = (size_t)q.ctx->L * q.ctx->N;
        for (size_t j = 0; j < q.n; ++j) {
            st = launch_product(q.ctx, q.ct + j * cw, q.pt + j * pw, nullptr, q.out + j * cw, 1, false, s);
            if (st != HC_OK) return st;
        }
    }
    return HC_OK;
}

hc_status hc_plan_autotune(hc_plan *p, const char *cache_path, void *cuda_stream)
{
    if (!plan_ok(p)) return set_error(HC_ERR_INVALID_ARG, "invalid plan");
    DeviceGuard g(p->device);
    cudaStream_t s = as_stream(cuda_stream);
    cudaDeviceProp prop;
    HC_CUDA_TRY(cudaGetDeviceProperties(&prop, p->device));

    // knobs: the kernel families this plan launches, per context
    struct Knob {
        hc_ctx *ctx;
        int kind;
    };
    std::vector<Knob> knobs;
    for (const hc_ctx *c : p->ctxs) {
        bool any = false, blocked = false, fused = false;
        for (const PlanConv &cv : p->convs)
            if (cv.ctx == c) {
                any = true;
                (cv.blocked ? blocked : fused) = true;
            }
        hc_ctx *mc = const_cast<hc_ctx *>(c);  // variants are a documented mutable hint
        if (any) knobs.push_back(Knob{mc, KK_FWDCT});
        if (blocked) knobs.push_back(Knob{mc, KK_MACB});
        if (blocked) knobs.push_back(Knob{mc, KK_INVCT});
        if (fused) knobs.push_back(Knob{mc, KK_MAC});
        if (blocked) knobs.push_back(Knob{mc, KK_CONV});  // last: the form, with the tuned kernels
    }

    const uint64_t sig = plan_signature(p);
    std::vector<std::pair<std::string, int>> cache;
    if (cache_path) {
        if (FILE *f = fopen(cache_path, "r")) {
            char line[1024];
            while (fgets(line, sizeof line, f)) {
                char key[960];
                int v = -1;
                if (sscanf(line, "%959s %d", key, &v) == 2 && v >= 0 && v <= kNumVariants) cache.emplace_back(key, v);
            }
            fclose(f);
        }
    }
    std::vector<size_t> pending;
    for (size_t i = 0; i < knobs.size(); ++i) {
        const std::string k = tune_key(knobs[i].ctx, knobs[i].kind, prop.name, prop.multiProcessorCount, sig);
        int v = -1;
        for (const auto &e : cache)
            if (e.first == k) v = e.second;  // last entry wins
        if (v >= 0 && v < kind_variants(knobs[i].kind))
            knobs[i].ctx->variant[knobs[i].kind] = (uint8_t)v;
        else
            pending.push_back(i);
    }
    drop_graph(p);  // captured launches carry the old variants
    if (pending.empty()) return HC_OK;

    FILE *out = cache_path ? fopen(cache_path, "a") : nullptr;
    hc_status st = HC_OK;
    for (size_t i : pending) {
        Knob &kb = knobs[i];
        int best = kb.ctx->variant[kb.kind];
        float best_ms = -1.f;
        for (int v = 0; v < kind_variants(kb.kind) && st == HC_OK; ++v) {
            kb.ctx->variant[kb.kind] = (uint8_t)v;
            float ms = 0.f;
            st = time_batched(p, s, 5, &ms);
            if (st == HC_OK && (best_ms < 0.f || ms < best_ms)) {
                best_ms = ms;
                best = v;
            }
        }
        kb.ctx->variant[kb.kind] = (uint8_t)best;
        if (st != HC_OK) break;
        if (out)
            fprintf(out, "%s %d\n", tune_key(kb.ctx, kb.kind, prop.name, prop.multiProcessorCount, sig).c_str(), best);
    }
    if (out) fclose(out);
    return st;
}

hc_status hc_plan_info(const hc_plan *p, uint64_t *n_products, uint64_t *alg_bytes, uint32_t *n_launches)
{
    if (!plan_ok(p)) return set_error(HC_ERR_INVALID_ARG, "invalid plan");
    if (n_products) *n_products = p->n_products;
    if (alg_bytes) *alg_bytes = p->alg_bytes;
    if (n_launches) *n_launches = count_launches(p);
    return HC_OK;
}

}  // extern "C"
