// hc_probe.cu -- throughput probe of the integer multiply pipe (hc_probe_int_rate).
//
// The layer's kernels are bound by 32-bit integer multiply-adds (IMAD), so their
// roofline needs the pipe's rate on the device at hand.  The probe runs long
// chains of one arithmetic form in every thread, eight independent chains per
// thread and 32 warps per SM, so that dependency latency is hidden and the pipe
// is the only limit, and times the launch with CUDA events.  Forms:
//   0  lazy Shoup multiplication (shoup_lazy): 5 wide + 4 narrow multiply-adds,
//      14 IMAD-equivalents, the butterfly's product;
//   1  narrow 32-bit multiply-add (mad.lo.u32): 1 IMAD-equivalent;
//   2  wide 32x32->64 multiply-add (mad.wide.u32): 2 IMAD-equivalents.
// The operands come from kernel arguments, so no chain can be folded, and every
// chain's final value is written out.
#include "hc_arith.cuh"
#include "hc_internal.h"

namespace hc {

namespace {

constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 4;

__global__ void __launch_bounds__(kProbeThreads) k_probe_int(uint32_t form, uint32_t iters, uint64_t a, uint64_t b,
                                                              uint64_t c, uint64_t *__restrict__ out)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = a ^ (tid * kProbeChains + k);
    if (form == 0) {
        // y <- y * w mod q lazily (result < 4q, a valid input again); b = w, c = w' (companion of w)
        const uint64_t nq = 0ull - (a | 1);
        for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k) x[k] = shoup_lazy(x[k], b, c, nq);
        }
    } else if (form == 1) {
        const uint32_t m = (uint32_t)b, d = (uint32_t)c;
        uint32_t y[kProbeChains];
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) y[k] = (uint32_t)x[k];
        for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k) asm("mad.lo.u32 %0, %0, %1, %2;" : "+r"(y[k]) : "r"(m), "r"(d));
        }
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = y[k];
    } else {
        const uint32_t m = (uint32_t)b;
        for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k) {
                // x <- lo32(x) * m + x (64-bit accumulate: the chain's dependency runs through x)
                uint64_t r;
                asm("{\n\t"
                    ".reg .u32 l, h;\n\t"
                    "mov.b64 {l, h}, %1;\n\t"
                    "mad.wide.u32 %0, l, %2, %1;\n\t"
                    "}"
                    : "=l"(r)
                    : "l"(x[k]), "r"(m));
                x[k] = r;
            }
        }
    }
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s ^= x[k];
    out[tid] = s;
}

}  // namespace

}  // namespace hc

extern "C" hc_status hc_probe_int_rate(const hc_ctx *ctx, uint32_t form, uint32_t iters, void *cuda_stream,
                                       double *ops_per_s, double *ms_out, double *imad_eq_per_op)
{
    using namespace hc;
    if (!ctx || ctx->magic != kMagicCtx) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (form > 2) return set_error(HC_ERR_INVALID_ARG, "form must be 0, 1 or 2");
    if (iters == 0 || iters > (1u << 24)) return set_error(HC_ERR_INVALID_ARG, "iters must be in [1, 2^24]");
    DeviceGuard g(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    const unsigned grid = ctx->sms * kProbeCtasPerSm;
    const size_t threads = (size_t)grid * kProbeThreads;
    uint64_t *d_out = (uint64_t *)dev_alloc(threads * sizeof(uint64_t), s);
    if (!d_out) return set_error(HC_ERR_OOM, "probe output allocation failed");
    const uint64_t q = ctx->q[0], w = (q >> 1) | 1;
    const uint64_t wp = (uint64_t)(((unsigned __int128)w << 64) / q);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    hc_status st = HC_OK;
    float ms = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = cuda_error(cudaGetLastError(), "cudaEventCreate");
    } else {
        // one untimed launch (clocks up, code loaded), then the timed one
        for (int rep = 0; rep < 2 && st == HC_OK; ++rep) {
            if (rep == 1) cudaEventRecord(e0, s);
            k_probe_int<<<grid, kProbeThreads, 0, s>>>(form, iters, q, w, wp, d_out);
            if (rep == 1) cudaEventRecord(e1, s);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_error(e, "launch k_probe_int");
        }
        if (st == HC_OK) {
            cudaError_t e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) st = cuda_error(e, "probe timing");
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(d_out, s);
    if (st != HC_OK) return st;
    const double ops = (double)threads * iters * kProbeChains;
    const double eq = form == 0 ? 14.0 : form == 1 ? 1.0 : 2.0;
    if (ops_per_s) *ops_per_s = ops / (ms / 1e3);
    if (ms_out) *ms_out = ms;
    if (imad_eq_per_op) *imad_eq_per_op = eq;
    return HC_OK;
}
