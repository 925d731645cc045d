// hc_kernels.cu -- sm_103a kernels of the HE-convolution hot path and their launchers.
//
//   k_ntt_fwd   forward NTT of NP polynomials per CTA (in place or out of place)
//   k_ntt_inv   inverse NTT, NP polynomials per CTA
//   k_mac_intt  NTT-domain multiply-accumulate of a term list, then inverse NTT:
//               out[o] = INTT(sum_t ct_ntt[ct_t] . pt_ntt[pt_t])         (Sec. 6.2)
//   k_product   one standalone ct x pt product fused end to end:
//               out[j] (+)= INTT(NTT(ct[j]) . pt_ntt[j])                  (App. C.1)
//   k_lift_int8 signed 8-bit weight coefficients -> residues mod every q_i
//   k_range_check  checked mode: flag any residue >= q_i
//
// All kernels are plain integer code (no tensor cores: this is exact modular
// arithmetic, not a floating-point contraction).  One CTA owns NP whole
// polynomial limbs, so every transform reads and writes HBM exactly once.
#include <atomic>

#include "hc_ntt.cuh"

namespace hc {

// Launch shapes: 512 threads per CTA for every N; both ciphertext components
// share a CTA (and its twiddle loads) up to N = 8192.
template <int LOGN> struct FusedCfgSel;
template <> struct FusedCfgSel<12> { using type = NttCfg<12, 3, 2>; };
template <> struct FusedCfgSel<13> { using type = NttCfg<13, 4, 2>; };
template <> struct FusedCfgSel<14> { using type = NttCfg<14, 5, 1>; };
template <int LOGN> struct SingleCfgSel;
template <> struct SingleCfgSel<12> { using type = NttCfg<12, 3, 1>; };
template <> struct SingleCfgSel<13> { using type = NttCfg<13, 4, 1>; };
template <> struct SingleCfgSel<14> { using type = NttCfg<14, 5, 1>; };

// ---------------------------------------------------------------------------
// store the last inverse-round layout: slot r = v*KK + j holds element
// tid + T*(v + j*SUBS)  (coalesced across the warp)
template <class Cfg>
__device__ __forceinline__ int inv_out_elem(int tid, int r)
{
    using RS = RoundShape<Cfg, Cfg::NROUNDS - 1>;
    const int v = r >> RS::K, j = r & (RS::KK - 1);
    return tid + Cfg::T * (v + j * RS::SUBS);
}

// ---------------------------------------------------------------------------
template <class Cfg>
__global__ void __launch_bounds__(Cfg::T, 1)
k_ntt_fwd(const uint64_t *in, uint64_t *out, const LimbConst *__restrict__ limbs, uint32_t L,
          uint32_t n_groups)
{
    extern __shared__ uint64_t sm[];
    constexpr int NP = Cfg::NP, C = Cfg::C, T = Cfg::T, N = Cfg::N;
    const int tid = threadIdx.x;
    const uint32_t limb = blockIdx.x / n_groups, grp = blockIdx.x % n_groups;
    const LimbConst &lc = limbs[limb];
    const uint64_t q = lc.q;

    uint64_t x[NP][C];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const uint64_t *src = in + ((size_t)(grp * NP + p) * L + limb) * N;
#pragma unroll
        for (int r = 0; r < C; ++r) x[p][r] = __ldg(src + tid + r * T);
    }
    fwd_transform<Cfg>(x, sm, lc.tw_f, q, tid);

    // canonical residues, stored through shared memory as coalesced 16-byte pairs
    const uint64_t one_s = lc.one_s;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < C; ++r) {
#pragma unroll
        for (int p = 0; p < NP; ++p) sm[p * N + spos<Cfg>(tid * C + r)] = reduce64(x[p][r], q, one_s);
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(out + ((size_t)(grp * NP + p) * L + limb) * N);
#pragma unroll
        for (int r = 0; r < C / 2; ++r) {
            const int e = 2 * (tid + r * T);
            ulonglong2 v;
            v.x = sm[p * N + spos<Cfg>(e)];
            v.y = sm[p * N + spos<Cfg>(e + 1)];
            dst[tid + r * T] = v;
        }
    }
}

template <class Cfg>
__global__ void __launch_bounds__(Cfg::T, 1)
k_ntt_inv(const uint64_t *in, uint64_t *out, const LimbConst *__restrict__ limbs, uint32_t L,
          uint32_t n_groups)
{
    extern __shared__ uint64_t sm[];
    constexpr int NP = Cfg::NP, C = Cfg::C, N = Cfg::N;
    const int tid = threadIdx.x;
    const uint32_t limb = blockIdx.x / n_groups, grp = blockIdx.x % n_groups;
    const LimbConst &lc = limbs[limb];

    uint64_t x[NP][C];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const ulonglong2 *src =
            reinterpret_cast<const ulonglong2 *>(in + ((size_t)(grp * NP + p) * L + limb) * N + tid * C);
#pragma unroll
        for (int r = 0; r < C / 2; ++r) {
            const ulonglong2 v = __ldg(src + r);
            x[p][2 * r] = v.x;
            x[p][2 * r + 1] = v.y;
        }
    }
    inv_transform<Cfg>(x, sm, lc, lc.tw_i, tid);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        uint64_t *dst = out + ((size_t)(grp * NP + p) * L + limb) * N;
#pragma unroll
        for (int r = 0; r < C; ++r) dst[inv_out_elem<Cfg>(tid, r)] = x[p][r];
    }
}

// ---------------------------------------------------------------------------
// group = one output and NP of its components; limb-major item order so that
// consecutive CTAs (consecutive outputs) share weight polynomials in L2.
template <class Cfg>
__global__ void __launch_bounds__(Cfg::T, 1)
k_mac_intt(const uint64_t *__restrict__ ct_ntt, const uint64_t *__restrict__ pt_ntt,
           const uint32_t *__restrict__ term_ptr, const uint32_t *__restrict__ terms,
           uint64_t *__restrict__ out, const LimbConst *__restrict__ limbs, uint32_t L,
           uint32_t n_groups)
{
    extern __shared__ uint64_t sm[];
    constexpr int NP = Cfg::NP, C = Cfg::C, N = Cfg::N;
    constexpr int CPG = 2 / NP;  // component groups per output
    const int tid = threadIdx.x;
    const uint32_t limb = blockIdx.x / n_groups, grp = blockIdx.x % n_groups;
    const uint32_t o = grp / CPG;
    const uint32_t comp0 = (grp % CPG) * NP;
    const LimbConst &lc = limbs[limb];
    const uint64_t q = lc.q, r64 = lc.r64, r64_s = lc.r64_s, one_s = lc.one_s;
    const uint32_t t0 = __ldg(term_ptr + o), t1 = __ldg(term_ptr + o + 1);

    uint64_t x[NP][C];
#pragma unroll
    for (int cb = 0; cb < C; cb += 4) {
        uint64_t lo[NP][4], hi[NP][4];
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int i = 0; i < 4; ++i) lo[p][i] = hi[p][i] = 0;
        for (uint32_t t = t0; t < t1; ++t) {
            const uint32_t ci = __ldg(terms + 2 * t), pi = __ldg(terms + 2 * t + 1);
            const ulonglong2 *wp =
                reinterpret_cast<const ulonglong2 *>(pt_ntt + ((size_t)pi * L + limb) * N + tid * C + cb);
            const ulonglong2 w01 = __ldg(wp), w23 = __ldg(wp + 1);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const ulonglong2 *xp = reinterpret_cast<const ulonglong2 *>(
                    ct_ntt + (((size_t)ci * 2 + comp0 + p) * L + limb) * N + tid * C + cb);
                const ulonglong2 x01 = __ldg(xp), x23 = __ldg(xp + 1);
                mac128(lo[p][0], hi[p][0], x01.x, w01.x);
                mac128(lo[p][1], hi[p][1], x01.y, w01.y);
                mac128(lo[p][2], hi[p][2], x23.x, w23.x);
                mac128(lo[p][3], hi[p][3], x23.y, w23.y);
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int i = 0; i < 4; ++i) x[p][cb + i] = reduce128(lo[p][i], hi[p][i], q, r64, r64_s, one_s);
    }
    inv_transform<Cfg>(x, sm, lc, lc.tw_i, tid);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        uint64_t *dst = out + (((size_t)o * 2 + comp0 + p) * L + limb) * N;
#pragma unroll
        for (int r = 0; r < C; ++r) dst[inv_out_elem<Cfg>(tid, r)] = x[p][r];
    }
}

// ---------------------------------------------------------------------------
template <class Cfg>
__global__ void __launch_bounds__(Cfg::T, 1)
k_product(const uint64_t *__restrict__ ct, const uint64_t *__restrict__ pt_ntt,
          const uint32_t *__restrict__ out_index, uint64_t *out, const LimbConst *__restrict__ limbs,
          uint32_t L, uint32_t n_groups, int accumulate)
{
    extern __shared__ uint64_t sm[];
    constexpr int NP = Cfg::NP, C = Cfg::C, T = Cfg::T, N = Cfg::N;
    constexpr int CPG = 2 / NP;
    const int tid = threadIdx.x;
    const uint32_t limb = blockIdx.x / n_groups, grp = blockIdx.x % n_groups;
    const uint32_t j = grp / CPG;
    const uint32_t comp0 = (grp % CPG) * NP;
    const LimbConst &lc = limbs[limb];
    const uint64_t q = lc.q;

    uint64_t x[NP][C];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const uint64_t *src = ct + (((size_t)j * 2 + comp0 + p) * L + limb) * N;
#pragma unroll
        for (int r = 0; r < C; ++r) x[p][r] = __ldg(src + tid + r * T);
    }
    fwd_transform<Cfg>(x, sm, lc.tw_f, q, tid);  // lazy values < 29 q, contiguous layout

    const uint64_t r64 = lc.r64, r64_s = lc.r64_s, one_s = lc.one_s;
    const ulonglong2 *wp = reinterpret_cast<const ulonglong2 *>(pt_ntt + ((size_t)j * L + limb) * N + tid * C);
#pragma unroll
    for (int r = 0; r < C / 2; ++r) {
        const ulonglong2 w = __ldg(wp + r);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            uint64_t lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
            mac128(lo0, hi0, x[p][2 * r], w.x);
            mac128(lo1, hi1, x[p][2 * r + 1], w.y);
            x[p][2 * r] = reduce128(lo0, hi0, q, r64, r64_s, one_s);
            x[p][2 * r + 1] = reduce128(lo1, hi1, q, r64, r64_s, one_s);
        }
    }
    inv_transform<Cfg>(x, sm, lc, lc.tw_i, tid);

    const uint32_t oj = out_index ? __ldg(out_index + j) : j;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        uint64_t *dst = out + (((size_t)oj * 2 + comp0 + p) * L + limb) * N;
        if (accumulate) {
#pragma unroll
            for (int r = 0; r < C; ++r) {
                const int e = inv_out_elem<Cfg>(tid, r);
                dst[e] = csub(dst[e] + x[p][r], q);
            }
        } else {
#pragma unroll
            for (int r = 0; r < C; ++r) dst[inv_out_elem<Cfg>(tid, r)] = x[p][r];
        }
    }
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

// ===========================================================================
// launchers
// ===========================================================================
namespace {

// one cache bit per (kernel family, launch shape, device)
template <class Cfg, int KIND, class K>
hc_status prepare(K kernel, size_t smem)
{
    static std::atomic<uint32_t> done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t bit = 1u << (dev & 31);
    if (!(done.load(std::memory_order_relaxed) & bit)) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
        done.fetch_or(bit);
    }
    return HC_OK;
}

// kernel names reported by the tracing facility: [kind][log2 N - 12]
const char *const kKernelNames[4][3] = {
    {"k_ntt_fwd/N4096", "k_ntt_fwd/N8192", "k_ntt_fwd/N16384"},
    {"k_ntt_inv/N4096", "k_ntt_inv/N8192", "k_ntt_inv/N16384"},
    {"k_mac_intt/N4096", "k_mac_intt/N8192", "k_mac_intt/N16384"},
    {"k_product/N4096", "k_product/N8192", "k_product/N16384"},
};

template <class Cfg>
const char *kname(int kind)
{
    return kKernelNames[kind][Cfg::LOGN - 12];
}

hc_status after_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HC_OK : cuda_error(e, what);
}

template <class Cfg>
hc_status run_ntt_fwd(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_groups, cudaStream_t s)
{
    if (n_groups == 0) return HC_OK;
    auto kern = k_ntt_fwd<Cfg>;
    hc_status st = prepare<Cfg, 0>(kern, Cfg::SMEM_BYTES);
    if (st != HC_OK) return st;
    const size_t items = n_groups * ctx->L;
    if (items > 0x7fffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    ProfileScope ps(kname<Cfg>(0), s);
    kern<<<(unsigned)items, Cfg::T, Cfg::SMEM_BYTES, s>>>(in, out, ctx->d_limbs, ctx->L, (uint32_t)n_groups);
    return after_launch("k_ntt_fwd");
}

template <class Cfg>
hc_status run_ntt_inv(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_groups, cudaStream_t s)
{
    if (n_groups == 0) return HC_OK;
    auto kern = k_ntt_inv<Cfg>;
    hc_status st = prepare<Cfg, 1>(kern, Cfg::SMEM_BYTES);
    if (st != HC_OK) return st;
    const size_t items = n_groups * ctx->L;
    if (items > 0x7fffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    ProfileScope ps(kname<Cfg>(1), s);
    kern<<<(unsigned)items, Cfg::T, Cfg::SMEM_BYTES, s>>>(in, out, ctx->d_limbs, ctx->L, (uint32_t)n_groups);
    return after_launch("k_ntt_inv");
}

template <class Cfg>
hc_status run_mac_intt(const hc_ctx *ctx, const uint64_t *ct_ntt, const uint64_t *pt_ntt, MacTerms terms,
                       uint64_t *out, size_t n_out, cudaStream_t s)
{
    if (n_out == 0) return HC_OK;
    auto kern = k_mac_intt<Cfg>;
    hc_status st = prepare<Cfg, 2>(kern, Cfg::SMEM_BYTES);
    if (st != HC_OK) return st;
    const size_t n_groups = n_out * (2 / Cfg::NP);
    const size_t items = n_groups * ctx->L;
    if (items > 0x7fffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    ProfileScope ps(kname<Cfg>(2), s);
    kern<<<(unsigned)items, Cfg::T, Cfg::SMEM_BYTES, s>>>(ct_ntt, pt_ntt, terms.term_ptr, terms.terms, out,
                                                          ctx->d_limbs, ctx->L, (uint32_t)n_groups);
    return after_launch("k_mac_intt");
}

template <class Cfg>
hc_status run_product(const hc_ctx *ctx, const uint64_t *ct, const uint64_t *pt_ntt, const uint32_t *out_index,
                      uint64_t *out, size_t n, bool accumulate, cudaStream_t s)
{
    if (n == 0) return HC_OK;
    auto kern = k_product<Cfg>;
    hc_status st = prepare<Cfg, 3>(kern, Cfg::SMEM_BYTES);
    if (st != HC_OK) return st;
    const size_t n_groups = n * (2 / Cfg::NP);
    const size_t items = n_groups * ctx->L;
    if (items > 0x7fffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    ProfileScope ps(kname<Cfg>(3), s);
    kern<<<(unsigned)items, Cfg::T, Cfg::SMEM_BYTES, s>>>(ct, pt_ntt, out_index, out, ctx->d_limbs, ctx->L,
                                                          (uint32_t)n_groups, accumulate ? 1 : 0);
    return after_launch("k_product");
}

}  // namespace

#define HC_DISPATCH_LOGN(ctx, SEL, FN, ...)                                              \
    switch ((ctx)->logN) {                                                                \
    case 12: return FN<typename SEL<12>::type>(__VA_ARGS__);                              \
    case 13: return FN<typename SEL<13>::type>(__VA_ARGS__);                              \
    case 14: return FN<typename SEL<14>::type>(__VA_ARGS__);                              \
    default: return set_error(HC_ERR_UNSUPPORTED, "unsupported N = %u", (ctx)->N);       \
    }

hc_status launch_ntt_fwd(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_polys, cudaStream_t s)
{
    HC_DISPATCH_LOGN(ctx, SingleCfgSel, run_ntt_fwd, ctx, in, out, n_polys, s)
}

hc_status launch_ntt_inv(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_polys, cudaStream_t s)
{
    HC_DISPATCH_LOGN(ctx, SingleCfgSel, run_ntt_inv, ctx, in, out, n_polys, s)
}

namespace {
template <class Cfg>
hc_status run_ntt_fwd_ct(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_ct, cudaStream_t s)
{
    // NP = 2: one CTA per (ciphertext, limb); NP = 1: one per (component, limb)
    return run_ntt_fwd<Cfg>(ctx, in, out, n_ct * (2 / Cfg::NP), s);
}
}  // namespace

hc_status launch_ntt_fwd_ct(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_ct, cudaStream_t s)
{
    HC_DISPATCH_LOGN(ctx, FusedCfgSel, run_ntt_fwd_ct, ctx, in, out, n_ct, s)
}

hc_status launch_mac_intt(const hc_ctx *ctx, const uint64_t *ct_ntt, const uint64_t *pt_ntt, MacTerms terms,
                          uint64_t *out, size_t n_out, cudaStream_t s)
{
    HC_DISPATCH_LOGN(ctx, FusedCfgSel, run_mac_intt, ctx, ct_ntt, pt_ntt, terms, out, n_out, s)
}

hc_status launch_product(const hc_ctx *ctx, const uint64_t *ct, const uint64_t *pt_ntt, const uint32_t *out_index,
                         uint64_t *out, size_t n, bool accumulate, cudaStream_t s)
{
    HC_DISPATCH_LOGN(ctx, FusedCfgSel, run_product, ctx, ct, pt_ntt, out_index, out, n, accumulate, s)
}

hc_status launch_lift_int8(const hc_ctx *ctx, const int8_t *packed, uint64_t *out, size_t n_polys, cudaStream_t s)
{
    if (n_polys == 0) return HC_OK;
    const size_t total = n_polys * ctx->L * ctx->N;
    const unsigned blocks = (unsigned)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
    ProfileScope ps("k_lift_int8", s);
    k_lift_int8<<<blocks, 256, 0, s>>>(packed, out, ctx->d_limbs, ctx->L, ctx->N, n_polys);
    return after_launch("k_lift_int8");
}

hc_status launch_range_check(const hc_ctx *ctx, const uint64_t *p, size_t n_polys, int *flag, cudaStream_t s)
{
    if (n_polys == 0) return HC_OK;
    const size_t total = n_polys * ctx->L * ctx->N;
    const unsigned blocks = (unsigned)((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
    ProfileScope ps("k_range_check", s);
    k_range_check<<<blocks, 256, 0, s>>>(p, ctx->d_limbs, ctx->L, ctx->N, n_polys, flag);
    return after_launch("k_range_check");
}

}  // namespace hc
