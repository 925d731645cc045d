// hc_mixed.cu -- one persistent launch for a batch of standalone ct x pt
// products of uneven ring degree and limb count.
//
// Every product j computes out_j = INTT(NTT(ct_j) . pt_j) per component and
// limb (App. C.1).  The batch is cut into units -- one limb of one product,
// both components at N = 4096 and 8192, one component at N = 16384 -- so that
// every unit is one 512-thread CTA's worth of work with at most 128 KB of
// shared memory whatever its N.  One CTA per SM stays resident and pulls
// units from a global counter in the host's order (most expensive first),
// which balances uneven units across SMs without a tail of idle SMs per
// ring degree, and lets one launch cover every N.
#include "hc_kernels.cuh"

namespace hc {
namespace {

using MixCfg12 = NttCfg<12, 3, 2, 1>;  // C 8, both components, 64 KB
using MixCfg13 = NttCfg<13, 4, 2, 1>;  // C 16, both components, 128 KB
using MixCfg14 = NttCfg<14, 5, 1, 1>;  // C 32, one component, 128 KB
constexpr int kMixThreads = 512;
static_assert(MixCfg12::T == kMixThreads && MixCfg13::T == kMixThreads && MixCfg14::T == kMixThreads,
              "mixed-degree units share one CTA shape");
static_assert(mix_comps_per_unit(12) == MixCfg12::NP && mix_comps_per_unit(13) == MixCfg13::NP &&
                  mix_comps_per_unit(14) == MixCfg14::NP,
              "unit split must match the per-degree shapes");
constexpr size_t kMixSmem = MixCfg13::SMEM_BYTES > MixCfg14::SMEM_BYTES ? MixCfg13::SMEM_BYTES : MixCfg14::SMEM_BYTES;

__global__ void __launch_bounds__(kMixThreads, 1)
k_product_mixed(const MixItem *__restrict__ items, const uint32_t *__restrict__ units, uint32_t n_units,
                uint32_t *next)
{
    extern __shared__ uint64_t sm[];
    __shared__ uint32_t s_unit;
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(next, 1u);
        __syncthreads();
        const uint32_t u = s_unit;
        __syncthreads();  // every thread has read s_unit before the next write
        if (u >= n_units) return;
        const uint32_t code = __ldg(units + u);
        const MixItem &it = items[code >> 4];
        const uint32_t limb = (code >> 1) & 7, comp = code & 1;
        const LimbConst &lc = it.limbs[limb];
        if (it.logN == 12)
            product_task<MixCfg12>(sm, it.ct, it.pt, it.out, lc, it.L, limb, 0, false);
        else if (it.logN == 13)
            product_task<MixCfg13>(sm, it.ct, it.pt, it.out, lc, it.L, limb, 0, false);
        else
            product_task<MixCfg14>(sm, it.ct, it.pt, it.out, lc, it.L, limb, comp, false);
    }
}

}  // namespace

hc_status launch_product_mixed(const MixItem *items, const uint32_t *units, uint32_t n_units, uint32_t *next,
                               cudaStream_t s)
{
    if (n_units == 0) return HC_OK;
    static std::atomic<uint32_t> attr_done{0};
    static std::atomic<int> grid_cache[32];
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t bit = 1u << (dev & 31);
    if (!(attr_done.load() & bit)) {
        cudaError_t e = cudaFuncSetAttribute(k_product_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMixSmem);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(k_product_mixed)");
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_product_mixed, kMixThreads, kMixSmem);
        if (e != cudaSuccess) return cuda_error(e, "occupancy(k_product_mixed)");
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
        if (per_sm < 1) return set_error(HC_ERR_UNSUPPORTED, "k_product_mixed does not fit on an SM");
        grid_cache[dev & 31].store(per_sm * sms);
        attr_done.fetch_or(bit);
    }
    const uint32_t resident = (uint32_t)grid_cache[dev & 31].load();
    const uint32_t grid = n_units < resident ? n_units : resident;
    ProfileScope ps("k_product_mixed", s);
    k_product_mixed<<<grid, kMixThreads, kMixSmem, s>>>(items, units, n_units, next);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "launch k_product_mixed");
    return HC_OK;
}

}  // namespace hc
