// hc_fused.cu -- the whole online convolution of many layers of one ring
// degree (Sec. 6.2: NTT of the inputs, NTT-domain MAC, INTT of the outputs)
// in ONE persistent launch.
//
// Tasks, numbered over the launch:  all forward-NTT tasks (one input
// polynomial limb each, limb-major), then all MAC tasks (one 64-slot chunk
// of one limb for one group of output channels; hc_mac.cuh), then all
// inverse-NTT tasks (one output polynomial limb each, in place).  Resident
// CTAs take tasks in that order from a global counter.  A MAC task first
// waits until every forward task of its layer and limb has finished; an
// inverse task waits until every MAC chunk of its layer, limb and channel
// group has finished.  Completion is counted per (layer, limb) and per
// (layer, group, limb) with release/acquire atomics.  Every dependency of a
// task was taken from the counter before it, by a CTA that is already
// running and never waits for a later task, so the waits always end; they
// are bounded anyway (a wait that runs out sets err = 4 and ends the CTA).
//
// Phases of different layers, and the tail of one phase with the head of the
// next, overlap on the device: no grid-wide barrier, no launch gaps.
#include "hc_kernels.cuh"
#include "hc_mac.cuh"

namespace hc {
namespace {

// CTA shape per degree: NTT tasks with one polynomial per CTA, 128 registers
// per thread (a 64-register shape with twice the threads spills ~1 KB per
// thread in the combined task code, so it is not offered).
template <int LOGN, int V> struct FusedShape;
template <> struct FusedShape<12, 1> { using Cfg = NttCfg<12, 4, 1, 2>; };  // T 256, C 16
template <> struct FusedShape<13, 1> { using Cfg = NttCfg<13, 5, 1, 2>; };  // T 256, C 32
template <> struct FusedShape<14, 1> { using Cfg = NttCfg<14, 5, 1, 1>; };  // T 512, C 32

constexpr uint32_t kSpinLimit = 1u << 24;  // polls of a dependency counter (~2 s) before giving up

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// every thread's global stores of the task, then one release increment
__device__ __forceinline__ void signal_done(uint32_t *ctr)
{
    __threadfence();
    fence_proxy_async_global();  // the stores are read next by TMA (async proxy) or by other CTAs
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(ctr, 1u);
}

// wait until *ctr >= target (thread 0 polls, the CTA follows); false on timeout
__device__ __forceinline__ bool wait_for(const uint32_t *ctr, uint32_t target, int *s_ok)
{
    if (threadIdx.x == 0) {
        uint32_t it = 0;
        bool ok = true;
        while (ld_acquire(ctr) < target) {
            if (++it > kSpinLimit) {
                ok = false;
                break;
            }
            __nanosleep(64);
        }
        fence_proxy_async_global();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <class Cfg, int NS>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_conv_fused(const __grid_constant__ FusedLayersT<NS> P, uint32_t *cnt, int *err)
{
    constexpr int T = Cfg::T, N = Cfg::N;
    extern __shared__ __align__(16) uint64_t dsm[];
    __shared__ __align__(8) uint64_t bars[1 + kMacStages];
    __shared__ uint32_t s_task;
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < 1 + kMacStages; ++i) mbar_init(&bars[i], 1);
        mbar_fence_init();
    }
    MacRing ring{0, 0};
    uint32_t *next = cnt;
    for (;;) {
        __syncthreads();  // the previous task is finished with shared memory
        if (tid == 0) s_task = atomicAdd(next, 1u);
        __syncthreads();
        const uint32_t t = s_task;
        if (t >= P.total) break;

        // locate the task: phase, layer, index within the layer's phase
        uint32_t li = 0;
        int phase;
        if (t < P.s[0].t_mac) {
            phase = 0;
            while (li + 1 < P.n && t >= P.s[li + 1].t_fwd) ++li;
        } else if (t < P.s[0].t_inv) {
            phase = 1;
            while (li + 1 < P.n && t >= P.s[li + 1].t_mac) ++li;
        } else {
            phase = 2;
            while (li + 1 < P.n && t >= P.s[li + 1].t_inv) ++li;
        }
        const FusedLayer &ly = P.s[li];
        const MacSeg &sg = ly.mac;
        const uint32_t L = sg.L;

        if (phase == 0) {  // forward NTT of one input polynomial limb into the scratch
            const uint32_t local = t - ly.t_fwd;
            const uint32_t limb = local / (2 * ly.I), poly = local % (2 * ly.I);
            const size_t off = ((size_t)poly * L + limb) * N;
            fwd_task<Cfg>(dsm, ly.in + off, const_cast<uint64_t *>(sg.X) + off, 0, sg.limbs[limb], tid);
            signal_done(cnt + ly.c_fwd + limb);
        } else if (phase == 1) {  // one MAC chunk
            const uint32_t local = t - ly.t_mac;
            const uint32_t chunk = local % sg.chunks, rest = local / sg.chunks;
            const uint32_t group = rest % sg.groups, limb = rest / sg.groups;
            if (!wait_for(cnt + ly.c_fwd + limb, 2 * ly.I, &s_ok)) {
                if (tid == 0) atomicExch(err, 4);
                break;
            }
            const uint32_t m0 = group * sg.MB, m1 = min(sg.M, m0 + sg.MB);
            if (!mac_task<kMacKC, T>(sg, chunk, limb, m0, m1, dsm, bars, ring, err)) break;
            signal_done(cnt + ly.c_mac + group * L + limb);
        } else {  // inverse NTT of one output polynomial limb, in place
            const uint32_t local = t - ly.t_inv;
            const uint32_t limb = local / (2 * ly.O), poly = local % (2 * ly.O);
            const uint32_t group = poly / (2 * sg.B * sg.MB);
            if (!wait_for(cnt + ly.c_mac + group * L + limb, sg.chunks, &s_ok)) {
                if (tid == 0) atomicExch(err, 4);
                break;
            }
            uint64_t *y = sg.Y + ((size_t)poly * L + limb) * N;
            inv_task<Cfg, true>(dsm, y, y, 0, sg.limbs[limb], tid);
        }
    }
}

template <int LOGN, int V, int NS>
hc_status run_fused(FusedLayersT<NS> &P, size_t smem, uint32_t ctr_words, uint32_t *ctr, int *err, cudaStream_t s)
{
    using Cfg = typename FusedShape<LOGN, V>::Cfg;
    auto kern = k_conv_fused<Cfg, NS>;
    static std::atomic<uint32_t> attr_done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(attr_done.load() & (1u << (dev & 31)))) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(k_conv_fused)");
        attr_done.fetch_or(1u << (dev & 31));
    }
    // resident CTAs per dynamic shared-memory size (cached per device; few distinct sizes)
    static std::atomic<uint64_t> cache[32][8];
    const uint32_t key = (uint32_t)(smem >> 10) + 1;
    int per_sm = 0, sms = 0;
    for (auto &c : cache[dev & 31]) {
        const uint64_t v = c.load();
        if ((uint32_t)(v >> 32) == key) {
            per_sm = (int)(v & 0xffff);
            sms = (int)((v >> 16) & 0xffff);
            break;
        }
    }
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::T, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_error(e, "k_conv_fused occupancy");
        if (per_sm < 1) return set_error(HC_ERR_UNSUPPORTED, "k_conv_fused does not fit on an SM");
        for (auto &c : cache[dev & 31]) {
            uint64_t expect = 0;
            if (c.compare_exchange_strong(expect, (uint64_t)key << 32 | (uint64_t)sms << 16 | (uint64_t)per_sm)) break;
        }
    }
    HC_CUDA_TRY(cudaMemsetAsync(ctr, 0, (size_t)ctr_words * sizeof(uint32_t), s));
    const uint32_t resident = (uint32_t)(per_sm * sms);
    const uint32_t grid = P.total < resident ? P.total : resident;
    static const char *const names[3] = {"k_conv_fused/N4096", "k_conv_fused/N8192", "k_conv_fused/N16384"};
    ProfileScope ps(names[LOGN - 12], s);
    kern<<<grid, Cfg::T, smem, s>>>(P, ctr, err);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HC_OK : cuda_error(e, "launch k_conv_fused");
}

template <int LOGN, int V, int NS>
hc_status fused_for_ns(const ConvJob *jobs, size_t n, uint32_t *ctr, cudaStream_t s)
{
    FusedLayersT<NS> P{};
    size_t smem = FusedShape<LOGN, V>::Cfg::SMEM_BYTES;
    uint32_t words = 1;  // [0]: the task counter
    const ConvJob *idx[NS];
    for (size_t i = 0; i < n; ++i) {
        if (jobs[i].ctx->logN != (uint32_t)LOGN || !jobs[i].blocked) continue;
        if (P.n == (uint32_t)NS) return set_error(HC_ERR_UNSUPPORTED, "too many layers for one fused launch");
        idx[P.n] = &jobs[i];
        FusedLayer &ly = P.s[P.n++];
        const ConvJob &j = jobs[i];
        ly.mac = make_mac_seg(j.ctx, j.ntt, job_weights(j), j.out, j.w->G, j.w->B, j.w->Mp, kMacKC);
        ly.in = j.in;
        ly.I = j.w->I;
        ly.O = j.w->O;
        ly.c_fwd = words;
        words += j.ctx->L;
        ly.c_mac = words;
        words += ly.mac.groups * j.ctx->L;
        const size_t ms = mac_seg_smem(ly.mac);
        if (ms > smem) smem = ms;
    }
    if (P.n == 0) return HC_OK;
    uint64_t t = 0;
    for (uint32_t i = 0; i < P.n; ++i) {
        P.s[i].t_fwd = (uint32_t)t;
        t += (uint64_t)P.s[i].mac.L * 2 * P.s[i].I;
    }
    for (uint32_t i = 0; i < P.n; ++i) {
        P.s[i].t_mac = (uint32_t)t;
        t += (uint64_t)P.s[i].mac.L * P.s[i].mac.groups * P.s[i].mac.chunks;
    }
    for (uint32_t i = 0; i < P.n; ++i) {
        P.s[i].t_inv = (uint32_t)t;
        t += (uint64_t)P.s[i].mac.L * 2 * P.s[i].O;
    }
    if (t > 0xffffffffu) return set_error(HC_ERR_INVALID_ARG, "fused launch too large");
    P.total = (uint32_t)t;
    return run_fused<LOGN, V, NS>(P, smem, words, ctr, timeout_flag(idx[0]->ctx), s);
}

template <int LOGN>
hc_status fused_for(const ConvJob *jobs, size_t n, uint32_t *ctr, cudaStream_t s)
{
    size_t count = 0;
    const ConvJob *first = nullptr;
    for (size_t i = 0; i < n; ++i)
        if (jobs[i].ctx->logN == (uint32_t)LOGN && jobs[i].blocked) {
            if (!first) first = &jobs[i];
            ++count;
        }
    if (!first) return HC_OK;
    // one layer: a one-entry table keeps the kernel's parameter block small
    return count == 1 ? fused_for_ns<LOGN, 1, 1>(jobs, n, ctr, s)
                      : fused_for_ns<LOGN, 1, kFusedMaxLayers>(jobs, n, ctr, s);
}

}  // namespace

size_t fused_counter_words(const ConvJob *jobs, size_t n, uint32_t logN)
{
    size_t words = 0;
    for (size_t i = 0; i < n; ++i) {
        if (jobs[i].ctx->logN != logN || !jobs[i].blocked) continue;
        const MacSeg sg = make_mac_seg(jobs[i].ctx, jobs[i].ntt, job_weights(jobs[i]), jobs[i].out, jobs[i].w->G,
                                       jobs[i].w->B, jobs[i].w->Mp, kMacKC);
        words += jobs[i].ctx->L * (1 + sg.groups);
    }
    return words ? words + 1 : 0;
}

hc_status launch_conv_fused(const ConvJob *jobs, size_t n, uint32_t logN, uint32_t *ctr, cudaStream_t s)
{
    switch (logN) {
    case 12: return fused_for<12>(jobs, n, ctr, s);
    case 13: return fused_for<13>(jobs, n, ctr, s);
    case 14: return fused_for<14>(jobs, n, ctr, s);
    default: return set_error(HC_ERR_UNSUPPORTED, "unsupported degree");
    }
}

}  // namespace hc
