// hc_noalloc.cu -- hc_conv_ct_pt_noalloc: the convolution layer without any
// device allocation.
//
// hc_conv_ct_pt takes its scratch (the NTT'd input ciphertexts) from an
// allocator on every call.  Some callers must not allocate device memory:
// services whose whole device memory is reserved up front by another
// framework's caching allocator (a stray cudaMalloc would step outside that
// reservation), or latency-critical loops where cudaMalloc / cudaFree would
// synchronise the device.  For them this entry point keeps its scratch in one
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include <mutex>

#include "hc_internal.h"

namespace {

// 16 MiB of uint64 words: enough for the NTT'd inputs of a layer with
// I * 2 * L * N * 8 <= 16 MiB (e.g. I = 32 input ciphertexts at N = 8192, L = 3).
constexpr size_t kStaticScratchWords = (size_t)2 << 20;
static __device__ __align__(256) uint64_t g_conv_scratch[kStaticScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint64_t *g_scratch_addr[kMaxDevices] = {};

// Device address of g_conv_scratch on `dev`, looked up once per device with
// that device current.  In host code the symbol itself is only a host-side
// stand-in, so the kernels must be given this address instead.
hc_status scratch_address(int dev, uint64_t **out)
{
    if (dev < 0 || dev >= kMaxDevices) return hc::set_error(HC_ERR_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_conv_scratch);
        if (e != cudaSuccess) return hc::cuda_error(e, "cudaGetSymbolAddress(static scratch)");
        g_scratch_addr[dev] = static_cast<uint64_t *>(p);
    }
    *out = g_scratch_addr[dev];
    return HC_OK;
}

}  // namespace

extern "C" hc_status hc_conv_ct_pt_noalloc(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_ct_in,
                                           uint64_t *d_ct_out, void *cuda_stream)
{
    using namespace hc;
    if (!ctx || ctx->magic != kMagicCtx || !w || w->magic != kMagicWeights)
        return set_error(HC_ERR_INVALID_ARG, "invalid context or weights");
    if (w->ctx != ctx) return set_error(HC_ERR_INVALID_ARG, "weights were preprocessed for another context");
    if (!d_ct_in || !d_ct_out) return set_error(HC_ERR_INVALID_ARG, "null ciphertext buffer");
    if (w->mode == HC_WEIGHTS_NO_NTT) {  // needs no scratch at all
        DeviceGuard g(ctx->device);
        cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
        hc_status st = check_inputs(ctx, d_ct_in, (size_t)2 * w->I, s);
        return st == HC_OK ? launch_conv_direct(ctx, w, d_ct_in, d_ct_out, s) : st;
    }
    if (w->mode != HC_WEIGHTS_NTT_OFFLINE)
        return set_error(HC_ERR_UNSUPPORTED, "online NTT preprocessing needs allocated scratch");
    const size_t words = (size_t)w->I * 2 * ctx->L * ctx->N;
    if (words > kStaticScratchWords)
        return set_error(HC_ERR_BUDGET,
                         "layer needs %zu bytes of scratch; the static scratch of hc_conv_ct_pt_noalloc holds %zu",
                         words * sizeof(uint64_t), kStaticScratchWords * sizeof(uint64_t));
    DeviceGuard g(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    uint64_t *scratch = nullptr;
    hc_status st = scratch_address(ctx->device, &scratch);
    if (st != HC_OK) return st;
    st = check_inputs(ctx, d_ct_in, (size_t)2 * w->I, s);
    if (st != HC_OK) return st;
    // the forward NTT overwrites every scratch word the later phases read, so
    // nothing left over from an earlier call is ever used
    const size_t use = conv_scratch_words(ctx, w) < kStaticScratchWords ? conv_scratch_words(ctx, w)
                                                                        : kStaticScratchWords;
    return conv_layer(ctx, w, d_ct_in, d_ct_out, scratch, use, s);
}
