// hc_step.cu -- the server's step around a linear layer (Sec. 7): add the
// server's activation share to the client's ciphertexts, run the convolution
// with the NTT-preprocessed weights, subtract the server's random output mask,
// and extract only the output coefficients of c0 (Sec. 6.2: the results are
// sparse and only the output elements go back to the client).
//
// With Delta = floor(Q/t), adding Delta*x to c0 adds x to the plaintext and
// subtracting Delta*r subtracts r.  Both are elementwise and bound by HBM.
#include <cstring>

#include "hc_arith.cuh"
#include "hc_internal.h"

namespace hc {
namespace {

// Geometry of the step: the stride-1 layer computed (desc of the weights), its
// output packing, and the caller's input tensor with the phase split of a
// strided layer (s = 1, pb = 1, C1 = C0 for stride 1).
struct StepGeom {
    uint32_t Cw, Hw, Ww, Hpe, Wpe, B, Bw, oh, ow, Ho, Wo, offset, span, No, M;
    uint32_t C1, C0, H0, W0, pad0, s, pb;
};

StepGeom geom_of(const hc_weights *w)
{
    const hc_conv_desc &d = w->desc;
    StepGeom g;
    g.Cw = d.Cw;
    g.Hw = d.Hw;
    g.Ww = d.Ww;
    g.Hpe = d.H + 2 * d.pad;
    g.Wpe = d.W + 2 * d.pad;
    g.B = w->B;
    g.oh = d.Hw - d.kh + 1;
    g.ow = d.Ww - d.kw + 1;
    g.Ho = g.Hpe - d.kh + 1;
    g.Wo = g.Wpe - d.kw + 1;
    g.Bw = (g.Wo + g.ow - 1) / g.ow;
    g.offset = (d.Cw - 1) * d.Hw * d.Ww + (d.kh - 1) * d.Ww + (d.kw - 1);
    g.span = d.Cw * d.Hw * d.Ww;
    g.No = w->No;
    g.M = d.M;
    g.C1 = d.C;
    g.C0 = w->user.C;
    g.H0 = w->user.H;
    g.W0 = w->user.W;
    g.pad0 = w->user.pad;
    g.s = w->user.stride;
    g.pb = w->pb;
    return g;
}

// out = in with c0 += Delta * (server share packed like the input), c1 copied.
// Input coefficient (channel c1, padded position (r, q)) of the stride-1 layer
// holds x~[c1 % C0][s*r + a - pad0][s*q + b - pad0] of the caller's tensor,
// (a, b) = phase c1 / C0 split by pb (Sec. 8.1 networks; the polyphase split).
__global__ void k_share_add(const uint64_t *__restrict__ in, const uint64_t *__restrict__ share,
                            uint64_t *__restrict__ out, const LimbConst *__restrict__ limbs, uint32_t L, uint32_t N,
                            StepGeom g, uint32_t n_polys)
{
    const uint32_t area = g.Hw * g.Ww, span = g.Cw * area;
    for (uint32_t pi = blockIdx.y; pi < n_polys; pi += gridDim.y) {  // poly (item, component, limb)
        const uint32_t limb = pi % L, comp = (pi / L) & 1, item = pi / (2 * L);
        const uint64_t *src = in + (size_t)pi * N;
        uint64_t *dst = out + (size_t)pi * N;
        const uint32_t grp = item / g.B, b = item % g.B;
        const uint32_t r0 = (b / g.Bw) * g.oh, q0 = (b % g.Bw) * g.ow;  // block origin, padded coordinates
        const LimbConst &lc = limbs[limb];
        const uint64_t qm = lc.q;
        for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
            uint64_t v = src[k];
            if (comp == 0 && k < span) {
                const uint32_t c = k / area, rem = k - c * area, ii = rem / g.Ww, jj = rem - ii * g.Ww;
                const uint32_t ch1 = grp * g.Cw + c, r = r0 + ii, q = q0 + jj;
                if (ch1 < g.C1 && r < g.Hpe && q < g.Wpe) {
                    const uint32_t phase = ch1 / g.C0, ch = ch1 - phase * g.C0;
                    const int64_t R = (int64_t)g.s * r + phase / g.pb - g.pad0;
                    const int64_t Q = (int64_t)g.s * q + phase % g.pb - g.pad0;
                    if (R >= 0 && R < g.H0 && Q >= 0 && Q < g.W0) {
                        const uint64_t x = share[((size_t)ch * g.H0 + R) * g.W0 + Q];
                        const uint64_t dx = canon4(shoup_lazy(x, lc.delta, lc.delta_s, 0ull - qm), qm);
                        v = csub(v + dx, qm);
                    }
                }
            }
            dst[k] = v;
        }
    }
}

// launch k_share_add over the n_polys polynomials of [I][2][L][N]
cudaError_t share_add(const hc_ctx *ctx, const uint64_t *in, const uint64_t *share, uint64_t *out, const StepGeom &g,
                      uint32_t n_polys, cudaStream_t s)
{
    const dim3 grid((ctx->N + 1023) / 1024, n_polys < 65535 ? n_polys : 65535);
    k_share_add<<<grid, 256, 0, s>>>(in, share, out, ctx->d_limbs, ctx->L, ctx->N, g, n_polys);
    return cudaGetLastError();
}

// slots[o][l][s] = c0[n*span + offset + i*Ww + j] - Delta * r[m][row][col] for
// s = (n*oh + i)*ow + j, m = (o / B)*No + n (or 0 outside the output map / past M)
__global__ void k_extract_mask(const uint64_t *__restrict__ ct_out, const uint64_t *__restrict__ mask,
                               uint64_t *__restrict__ slots, const LimbConst *__restrict__ limbs, uint32_t L,
                               uint32_t N, StepGeom g, size_t total)
{
    const uint32_t per = g.oh * g.ow, S = g.No * per;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t sl = (uint32_t)(i % S);
        const size_t rest = i / S;
        const uint32_t limb = (uint32_t)(rest % L), o = (uint32_t)(rest / L);
        const uint32_t mp = o / g.B, b = o % g.B;
        const uint32_t n = sl / per, rem = sl % per;
        const uint32_t ii = rem / g.ow, jj = rem % g.ow;
        const uint32_t m = mp * g.No + n;
        const uint32_t row = (b / g.Bw) * g.oh + ii, col = (b % g.Bw) * g.ow + jj;
        uint64_t v = 0;
        if (m < g.M && row < g.Ho && col < g.Wo) {
            const uint32_t k = n * g.span + g.offset + ii * g.Ww + jj;
            v = ct_out[(((size_t)o * 2) * L + limb) * N + k];
            if (mask) {
                const LimbConst &lc = limbs[limb];
                const uint64_t q = lc.q;
                const uint64_t r = mask[((size_t)m * g.Ho + row) * g.Wo + col];
                const uint64_t dr = canon4(shoup_lazy(r, lc.delta, lc.delta_s, 0ull - q), q);
                v = v >= dr ? v - dr : v + q - dr;
            }
        }
        slots[i] = v;
    }
}

// grid of a grid-stride elementwise kernel: 16 CTAs of 256 threads per SM at most
unsigned grid_for(const hc_ctx *ctx, size_t total)
{
    const size_t b = (total + 255) / 256, cap = (size_t)ctx->sms * 16;
    return (unsigned)(b < cap ? (b ? b : 1) : cap);
}

struct Scratch {
    void *p = nullptr;
    cudaStream_t s;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() { dev_free(p, s); }
};

}  // namespace
}  // namespace hc

extern "C" hc_status hc_conv_server_step(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_ct_in,
                                         const uint64_t *d_share, const uint64_t *d_mask, uint64_t *d_ct_out,
                                         uint64_t *d_c0_slots, void *cuda_stream)
{
    using namespace hc;
    if (!ctx || ctx->magic != kMagicCtx || !w || w->magic != kMagicWeights)
        return set_error(HC_ERR_INVALID_ARG, "invalid context or weights");
    if (w->ctx != ctx) return set_error(HC_ERR_INVALID_ARG, "weights were preprocessed for another context");
    if (!d_ct_in || !d_ct_out || !d_c0_slots) return set_error(HC_ERR_INVALID_ARG, "null buffer");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    hc_status st = check_inputs(ctx, d_ct_in, (size_t)2 * w->I, s);
    if (st != HC_OK) return st;
    const StepGeom g = geom_of(w);
    const size_t in_words = (size_t)w->I * 2 * ctx->L * ctx->N;
    Scratch scratch(s);
    const uint64_t *src = d_ct_in;
    if (d_share) {
        scratch.p = dev_alloc(in_words * sizeof(uint64_t), s);
        if (!scratch.p) return set_error(HC_ERR_OOM, "scratch allocation failed");
        uint64_t *shared_in = (uint64_t *)scratch.p;
        ProfileScope ps("k_share_add", s);
        const cudaError_t e = share_add(ctx, d_ct_in, d_share, shared_in, g, 2 * w->I * ctx->L, s);
        if (e != cudaSuccess) return cuda_error(e, "launch k_share_add");
        src = shared_in;
    }
    st = conv_any(ctx, w, src, d_ct_out, s);  // any preprocessing mode
    if (st != HC_OK) return st;
    const size_t slot_words = (size_t)w->O * ctx->L * g.No * g.oh * g.ow;
    ProfileScope ps("k_extract_mask", s);
    k_extract_mask<<<grid_for(ctx, slot_words), 256, 0, s>>>(d_ct_out, d_mask, d_c0_slots, ctx->d_limbs, ctx->L, ctx->N, g,
                                                        slot_words);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HC_OK : cuda_error(e, "launch k_extract_mask");
}

namespace hc {
hc_status build_slot_table(hc_weights *w)
{
    const hc_conv_desc &d = w->desc;
    const uint32_t oh = d.Hw - d.kh + 1, ow = d.Ww - d.kw + 1, span = d.Cw * d.Hw * d.Ww;
    const uint32_t offset = (d.Cw - 1) * d.Hw * d.Ww + (d.kh - 1) * d.Ww + (d.kw - 1);
    const size_t S = (size_t)w->No * oh * ow;
    if (S == 0 || (size_t)w->No * span > w->ctx->N) return set_error(HC_ERR_INVALID_ARG, "invalid layer geometry");
    std::vector<SlotEntry> t(S);
    for (uint32_t n = 0; n < w->No; ++n)
        for (uint32_t i = 0; i < oh; ++i)
            for (uint32_t j = 0; j < ow; ++j) {
                SlotEntry &e = t[((size_t)n * oh + i) * ow + j];
                e.k = (uint16_t)(n * span + offset + i * d.Ww + j);  // < N <= 16384
                e.n = (uint16_t)n;
                e.i = (uint16_t)i;
                e.j = (uint16_t)j;
            }
    w->d_slot_table = (SlotEntry *)dev_alloc_persistent(S * sizeof(SlotEntry));
    if (!w->d_slot_table) return set_error(HC_ERR_OOM, "device allocation of the slot table failed");
    const cudaError_t e = cudaMemcpy(w->d_slot_table, t.data(), S * sizeof(SlotEntry), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? HC_OK : cuda_error(e, "uploading the slot table");
}
}  // namespace hc

// The server step returning only what the client needs (Sec. 6.2, Sec. 7): the
// full c1 of every output ciphertext and the masked output slots of its c0.
// The inverse transform writes them directly (k_ntt_inv_extract); c0 is never
// stored in full.
extern "C" hc_status hc_conv_server_step_sparse(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_ct_in,
                                                const uint64_t *d_share, const uint64_t *d_mask, uint64_t *d_c1_out,
                                                uint64_t *d_c0_slots, void *cuda_stream)
{
    using namespace hc;
    if (!ctx || ctx->magic != kMagicCtx || !w || w->magic != kMagicWeights)
        return set_error(HC_ERR_INVALID_ARG, "invalid context or weights");
    if (w->ctx != ctx) return set_error(HC_ERR_INVALID_ARG, "weights were preprocessed for another context");
    if (!d_ct_in || !d_c1_out || !d_c0_slots) return set_error(HC_ERR_INVALID_ARG, "null buffer");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    const StepGeom g = geom_of(w);
    const size_t LN = (size_t)ctx->L * ctx->N;
    const size_t in_words = (size_t)w->I * 2 * LN, y_words = (size_t)w->O * 2 * LN;
    if (w->mode == HC_WEIGHTS_NO_NTT || !conv_job_blocked(ctx, w)) {
        // no inverse transform to fuse into: the full step into scratch, then c1 out of it
        Scratch full(s);
        full.p = dev_alloc(y_words * sizeof(uint64_t), s);
        if (!full.p) return set_error(HC_ERR_OOM, "scratch allocation failed");
        uint64_t *y = (uint64_t *)full.p;
        hc_status st = hc_conv_server_step(ctx, w, d_ct_in, d_share, d_mask, y, d_c0_slots, cuda_stream);
        if (st != HC_OK) return st;
        HC_CUDA_TRY(cudaMemcpy2DAsync(d_c1_out, LN * sizeof(uint64_t), y + LN, 2 * LN * sizeof(uint64_t),
                                      LN * sizeof(uint64_t), w->O, cudaMemcpyDeviceToDevice, s));
        return HC_OK;
    }
    hc_status st = check_inputs(ctx, d_ct_in, (size_t)2 * w->I, s);
    if (st != HC_OK) return st;
    Scratch xs(s), ys(s), ws(s);
    xs.p = dev_alloc(in_words * sizeof(uint64_t), s);
    ys.p = dev_alloc(y_words * sizeof(uint64_t), s);
    if (!xs.p || !ys.p) return set_error(HC_ERR_OOM, "scratch allocation failed");
    uint64_t *x = (uint64_t *)xs.p, *y = (uint64_t *)ys.p;
    const uint64_t *src = d_ct_in;
    if (d_share) {
        ProfileScope ps("k_share_add", s);
        const cudaError_t e = share_add(ctx, d_ct_in, d_share, x, g, 2 * w->I * ctx->L, s);
        if (e != cudaSuccess) return cuda_error(e, "launch k_share_add");
        src = x;
    }
    const uint64_t *wpt = w->d_pt;
    if (w->mode == HC_WEIGHTS_NTT_ONLINE) {
        ws.p = dev_alloc((size_t)w->P * LN * sizeof(uint64_t), s);
        if (!ws.p) return set_error(HC_ERR_OOM, "scratch allocation failed");
        st = launch_ntt_fwd(ctx, w->d_pt, (uint64_t *)ws.p, w->P, s);
        if (st != HC_OK) return st;
        wpt = (const uint64_t *)ws.p;
    }
    ExtractArgs ex{y, d_c1_out, d_c0_slots, d_mask, w->d_slot_table, w->O, g.No * g.oh * g.ow, g.B, g.Bw,
                   g.oh, g.ow, g.Ho, g.Wo, g.No, g.M};
    if (ctx->variant[KK_CONV] == 2) {
        // launch form 2: one forward -> MAC -> epilogue chain per limb on parallel streams
        ConvJob job{ctx, w, src, y, x, true, wpt, &ex};
        return launch_limb_chains(&job, 1, ctx->logN, s);
    }
    st = launch_ntt_fwd_ct(ctx, src, x, w->I, s);  // in place after the share add
    if (st == HC_OK) st = launch_mac_conv(ctx, x, wpt, y, w->G, w->B, w->Mp, s);
    if (st != HC_OK) return st;
    return launch_inv_extract(ctx, ex, s);
}
