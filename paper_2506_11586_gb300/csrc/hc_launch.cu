// hc_launch.cu -- dispatch of the public launchers to the per-N kernel
// instantiations and the launch variant recorded in the context, plus the
// small elementwise kernels (weight lifting, range checks).
#include "hc_internal.h"

namespace hc {

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


int default_variant(int kind, uint32_t logn)
{
    (void)kind;
    (void)logn;
    return 0;
}

namespace {

hc_status after(const char *what)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HC_OK : cuda_error(e, what);
}

hc_status dispatch(const hc_ctx *ctx, int kind, const LaunchArgs &a, cudaStream_t s)
{
    const int v = ctx->variant[kind];
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

hc_status launch_ntt_fwd_ct(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_ct, cudaStream_t s)
{
    LaunchArgs a{};
    a.in = in;
    a.out = out;
    a.n = n_ct;
    return dispatch(ctx, KK_FWDCT, a, s);
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
    const unsigned blocks = (unsigned)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
    ProfileScope ps("k_lift_int8", s);
    k_lift_int8<<<blocks, 256, 0, s>>>(packed, out, ctx->d_limbs, ctx->L, ctx->N, n_polys);
    return after("k_lift_int8");
}

hc_status launch_range_check(const hc_ctx *ctx, const uint64_t *p, size_t n_polys, int *flag, cudaStream_t s)
{
    if (n_polys == 0) return HC_OK;
    const size_t total = n_polys * ctx->L * ctx->N;
    const unsigned blocks = (unsigned)((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
    ProfileScope ps("k_range_check", s);
    k_range_check<<<blocks, 256, 0, s>>>(p, ctx->d_limbs, ctx->L, ctx->N, n_polys, flag);
    return after("k_range_check");
}

}  // namespace hc
