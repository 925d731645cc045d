// hc_zp.cu -- BFV SIMD encoding over Z_P and the matrix-vector weights of
// HELiKs-style linear layers (SecONNds-P, Sec. 6.1: the linear algebra runs on
// plaintext vectors in Z_P^N; Sec. 2.3: the weights are NTT-preprocessed).
//
// Slots.  P = 1 mod 2N, zeta the smallest primitive 2N-th root mod P (the
// context's psi).  Slot (r, c), r in {0, 1}, c < N/2, of a polynomial p holds
// p(zeta^e), e = 5^c mod 2N for r = 0 and -5^c mod 2N for r = 1.  The forward
// NTT of the library puts p(psi^(2 rev(k) + 1)) at index k, so slot (r, c) is
// NTT index rev((e - 1) / 2): encoding scatters the slots to those indices and
// runs the inverse NTT mod P; decoding runs the forward NTT and gathers.
//
// Matrix-vector weights (the diagonal method).  A vector v of length n (a power
// of two dividing N/2) is held periodically, slot (r, t) = v[t mod n].  With
// w_i[r][t] = W[(t - i) mod n][t mod n] for i < n, the iteration of
// hc_mac_rotate, sum_i rot^i(vtilde * w_i), holds (W v)[j mod n] at slot (r, j):
// the product, in the input's format.  W is zero-padded to n x n.
#include <algorithm>

#include "hc_internal.h"

namespace hc {
namespace {

// slot (r, c) -> NTT index rev((e - 1) / 2), e = +-5^c mod 2N
__device__ __forceinline__ uint32_t slot_ntt_index(uint32_t r, uint32_t c, uint32_t N, uint32_t logN)
{
    const uint32_t m = 2 * N - 1;  // 2N is a power of two
    uint32_t e = 1, b = 5, k = c;
    while (k) {
        if (k & 1) e = (e * b) & m;
        b = (b * b) & m;
        k >>= 1;
    }
    if (r) e = (2 * N - e) & m;
    return __brev((e - 1) >> 1) >> (32 - logN);
}

// A[p][slot_ntt_index(r, c)] = slots[p][r][c]
__global__ void k_zp_scatter(const uint64_t *__restrict__ slots, uint64_t *__restrict__ A, uint32_t N,
                             uint32_t logN, size_t total)
{
    const uint32_t half = N / 2;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t p = t / N;
        const uint32_t j = (uint32_t)(t % N), r = j / half, c = j % half;
        A[p * N + slot_ntt_index(r, c, N, logN)] = slots[t];
    }
}

// slots[p][r][c] = A[p][slot_ntt_index(r, c)]
__global__ void k_zp_gather(const uint64_t *__restrict__ A, uint64_t *__restrict__ slots, uint32_t N,
                            uint32_t logN, size_t total)
{
    const uint32_t half = N / 2;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t p = t / N;
        const uint32_t j = (uint32_t)(t % N), r = j / half, c = j % half;
        slots[t] = A[p * N + slot_ntt_index(r, c, N, logN)];
    }
}

// out[p][i][k] = centered lift of poly[p][k] (in [0, P)) into q_i
__global__ void k_zp_lift(const uint64_t *__restrict__ poly, uint64_t *__restrict__ out,
                          const LimbConst *__restrict__ limbs, uint64_t P, uint32_t L, uint32_t N, size_t total)
{
    const uint64_t half = (P - 1) / 2;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const uint32_t k = (uint32_t)(t % N);
        const size_t r = t / N;
        const uint32_t i = (uint32_t)(r % L);
        const size_t p = r / L;
        const uint64_t v = poly[p * N + k];
        out[t] = v > half ? limbs[i].q - (P - v) : v;  // P < q_i
    }
}

// slots[i][r][t] = W[(t - i) mod n][t mod n] (zero outside n_out x n_in), for i < n
__global__ void k_zp_diagonals(const uint64_t *__restrict__ W, uint64_t *__restrict__ slots, uint32_t n_out,
                               uint32_t n_in, uint32_t n, uint32_t N, size_t total)
{
    const uint32_t half = N / 2, mask = n - 1;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)(x / N);
        const uint32_t t = (uint32_t)(x % N) % half;
        const uint32_t row = (t - i) & mask, col = t & mask;
        slots[x] = row < n_out && col < n_in ? W[(size_t)row * n_in + col] : 0;
    }
}

// Weight slot vectors of a Z_P convolution, plaintexts [p0, p0 + n) of the layer's
// [Y][kk][C] list: plaintext p = (y*kk + i)*C + c holds the constant
// K[2y + r][c][i] in slot row r (0 past M); K is [M][C][kk] residues mod P.
__global__ void k_zp_conv_slots(const uint64_t *__restrict__ K, uint64_t *__restrict__ slots, uint32_t M,
                                uint32_t C, uint32_t kk, size_t p0, uint32_t N, size_t total)
{
    const uint32_t half = N / 2;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        const size_t p = p0 + x / N;
        const uint32_t r = (uint32_t)(x % N) / half;
        const uint32_t c = (uint32_t)(p % C), i = (uint32_t)(p / C % kk), y = (uint32_t)(p / C / kk);
        const uint32_t m = 2 * y + r;
        slots[x] = m < M ? K[((size_t)m * C + c) * kk + i] : 0;
    }
}

// grid of a grid-stride elementwise kernel: 16 CTAs of 256 threads per SM at most
unsigned grid_for(const hc_ctx *ctx, size_t total)
{
    const size_t b = (total + 255) / 256, cap = (size_t)ctx->sms * 16;
    return (unsigned)(b < cap ? (b ? b : 1) : cap);
}

bool ctx_valid(const hc_ctx *c) { return c && c->magic == kMagicCtx; }

}  // namespace

hc_status zp_conv_geometry(const hc_conv_desc *d, uint32_t N, ZpConvGeom *g)
{
    if (!d->C || !d->H || !d->W || !d->M || !d->kh || !d->kw)
        return set_error(HC_ERR_INVALID_ARG, "empty convolution");
    if (d->stride > 1) return set_error(HC_ERR_UNSUPPORTED, "Z_P convolutions are stride 1");
    const uint64_t Hp = (uint64_t)d->H + 2ull * d->pad, Wp = (uint64_t)d->W + 2ull * d->pad;
    if (d->kh > Hp || d->kw > Wp) return set_error(HC_ERR_INVALID_ARG, "kernel larger than the padded image");
    if (Hp * Wp > N / 2)
        return set_error(HC_ERR_INVALID_ARG, "padded image of %llu slots does not fit one slot row (%u)",
                         (unsigned long long)(Hp * Wp), N / 2);
    g->Hp = (uint32_t)Hp;
    g->Wp = (uint32_t)Wp;
    g->Ho = (uint32_t)Hp - d->kh + 1;
    g->Wo = (uint32_t)Wp - d->kw + 1;
    g->Y = (d->M + 1) / 2;
    g->step_row = (uint32_t)Wp - d->kw + 1;
    return HC_OK;
}

namespace {

// ctx_p must be a one-limb context (the plaintext prime)
hc_status check_plain_ctx(const hc_ctx *ctx_p)
{
    if (!ctx_valid(ctx_p)) return set_error(HC_ERR_INVALID_ARG, "invalid plaintext context");
    if (ctx_p->L != 1) return set_error(HC_ERR_INVALID_ARG, "the plaintext context must have one modulus P");
    return HC_OK;
}

struct Scratch {
    void *p = nullptr;
    cudaStream_t s;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() { dev_free(p, s); }
};

hc_status encode_into(const hc_ctx *ctx_p, const uint64_t *slots, size_t n, uint64_t *poly, cudaStream_t s)
{
    const size_t total = n * ctx_p->N;
    ProfileScope ps("k_zp_scatter", s);
    k_zp_scatter<<<grid_for(ctx_p, total), 256, 0, s>>>(slots, poly, ctx_p->N, ctx_p->logN, total);
    HC_CUDA_TRY(cudaGetLastError());
    return launch_ntt_inv(ctx_p, poly, poly, n, s);
}

hc_status lift_ntt_into(const hc_ctx *ctx, uint64_t P, const uint64_t *poly, size_t n, uint64_t *out, cudaStream_t s)
{
    const size_t total = n * ctx->L * ctx->N;
    {
        ProfileScope ps("k_zp_lift", s);
        k_zp_lift<<<grid_for(ctx, total), 256, 0, s>>>(poly, out, ctx->d_limbs, P, ctx->L, ctx->N, total);
        HC_CUDA_TRY(cudaGetLastError());
    }
    return launch_ntt_fwd(ctx, out, out, n, s);
}

}  // namespace
}  // namespace hc

using namespace hc;

extern "C" {

hc_status hc_zp_encode(const hc_ctx *ctx_p, const uint64_t *d_slots, size_t n, uint64_t *d_poly, void *cuda_stream)
{
    hc_status st = check_plain_ctx(ctx_p);
    if (st != HC_OK || n == 0) return st;
    if (!d_slots || !d_poly) return set_error(HC_ERR_INVALID_ARG, "null buffer");
    if (d_slots == d_poly) return set_error(HC_ERR_INVALID_ARG, "in place encoding is not supported");
    if (n * ctx_p->N > 0x7fffffffffull) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    DeviceGuard dg(ctx_p->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    st = check_inputs(ctx_p, d_slots, n, s);
    if (st != HC_OK) return st;
    return encode_into(ctx_p, d_slots, n, d_poly, s);
}

hc_status hc_zp_decode(const hc_ctx *ctx_p, const uint64_t *d_poly, size_t n, uint64_t *d_slots, void *cuda_stream)
{
    hc_status st = check_plain_ctx(ctx_p);
    if (st != HC_OK || n == 0) return st;
    if (!d_slots || !d_poly) return set_error(HC_ERR_INVALID_ARG, "null buffer");
    if (d_slots == d_poly) return set_error(HC_ERR_INVALID_ARG, "in place decoding is not supported");
    if (n * ctx_p->N > 0x7fffffffffull) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    DeviceGuard dg(ctx_p->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    st = check_inputs(ctx_p, d_poly, n, s);
    if (st != HC_OK) return st;
    Scratch tmp(s);
    tmp.p = dev_alloc(n * ctx_p->N * sizeof(uint64_t), s);
    if (!tmp.p) return set_error(HC_ERR_OOM, "scratch allocation failed");
    uint64_t *A = (uint64_t *)tmp.p;
    st = launch_ntt_fwd(ctx_p, d_poly, A, n, s);
    if (st != HC_OK) return st;
    const size_t total = n * ctx_p->N;
    ProfileScope ps("k_zp_gather", s);
    k_zp_gather<<<grid_for(ctx_p, total), 256, 0, s>>>(A, d_slots, ctx_p->N, ctx_p->logN, total);
    HC_CUDA_TRY(cudaGetLastError());
    return HC_OK;
}

hc_status hc_zp_lift_ntt(const hc_ctx *ctx, uint64_t P, const uint64_t *d_poly, size_t n, uint64_t *d_out,
                         void *cuda_stream)
{
    if (!ctx_valid(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (n == 0) return HC_OK;
    if (!d_poly || !d_out) return set_error(HC_ERR_INVALID_ARG, "null buffer");
    if (P < 3 || !(P & 1)) return set_error(HC_ERR_INVALID_ARG, "plaintext modulus must be odd and >= 3");
    for (uint32_t i = 0; i < ctx->L; ++i)
        if (P >= ctx->q[i]) return set_error(HC_ERR_INVALID_ARG, "plaintext modulus must be below every q_i");
    DeviceGuard dg(ctx->device);
    return lift_ntt_into(ctx, P, d_poly, n, d_out, reinterpret_cast<cudaStream_t>(cuda_stream));
}

hc_status hc_zp_matvec_preprocess(const hc_ctx *ctx, const hc_ctx *ctx_p, const uint64_t *h_W, uint32_t n_out,
                                  uint32_t n_in, uint64_t *d_out, size_t out_words, uint32_t *n_terms,
                                  void *cuda_stream)
{
    if (!ctx_valid(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    hc_status st = check_plain_ctx(ctx_p);
    if (st != HC_OK) return st;
    if (ctx_p->N != ctx->N) return set_error(HC_ERR_INVALID_ARG, "contexts of different ring degree");
    if (!h_W || !d_out || !n_terms || n_out == 0 || n_in == 0)
        return set_error(HC_ERR_INVALID_ARG, "null buffer or empty matrix");
    const uint64_t P = ctx_p->q[0];
    for (uint32_t i = 0; i < ctx->L; ++i)
        if (P >= ctx->q[i]) return set_error(HC_ERR_INVALID_ARG, "P must be below every q_i");
    const uint32_t N = ctx->N;
    uint32_t n = 1;
    while (n < n_out || n < n_in) n *= 2;
    if (n > N / 2) return set_error(HC_ERR_INVALID_ARG, "matrix of %u x %u does not fit N/2 = %u slots", n_out, n_in,
                                    N / 2);
    *n_terms = n;
    if (out_words < (size_t)n * ctx->L * N)
        return set_error(HC_ERR_INVALID_ARG, "d_out holds %zu words, %zu needed", out_words, (size_t)n * ctx->L * N);
    const size_t wn = (size_t)n_out * n_in;
    for (size_t i = 0; i < wn; ++i)
        if (h_W[i] >= P) return set_error(HC_ERR_RANGE, "matrix entry %zu is not below P", i);
    DeviceGuard dg(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    // scratch: W, the diagonal slot vectors [n][N], their encodings [n][N]
    const size_t w_words = (wn + 1) & ~(size_t)1;
    Scratch tmp(s);
    tmp.p = dev_alloc((w_words + 2 * (size_t)n * N) * sizeof(uint64_t), s);
    if (!tmp.p) return set_error(HC_ERR_OOM, "scratch allocation failed");
    uint64_t *dW = (uint64_t *)tmp.p, *slots = dW + w_words, *poly = slots + (size_t)n * N;
    HC_CUDA_TRY(cudaMemcpyAsync(dW, h_W, wn * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    {
        const size_t total = (size_t)n * N;
        ProfileScope ps("k_zp_diagonals", s);
        k_zp_diagonals<<<grid_for(ctx_p, total), 256, 0, s>>>(dW, slots, n_out, n_in, n, N, total);
        HC_CUDA_TRY(cudaGetLastError());
    }
    st = encode_into(ctx_p, slots, n, poly, s);
    if (st == HC_OK) st = lift_ntt_into(ctx, P, poly, n, d_out, s);
    if (st != HC_OK) return st;
    HC_CUDA_TRY(cudaStreamSynchronize(s));  // the host matrix must outlive the upload
    return HC_OK;
}

hc_status hc_zp_conv_preprocess(const hc_ctx *ctx, const hc_ctx *ctx_p, const hc_conv_desc *desc,
                                const uint64_t *h_K, uint64_t *d_out, size_t out_words, void *cuda_stream)
{
    if (!ctx_valid(ctx)) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    hc_status st = check_plain_ctx(ctx_p);
    if (st != HC_OK) return st;
    if (ctx_p->N != ctx->N) return set_error(HC_ERR_INVALID_ARG, "contexts of different ring degree");
    if (!desc || !h_K || !d_out) return set_error(HC_ERR_INVALID_ARG, "null descriptor or buffer");
    const uint64_t P = ctx_p->q[0];
    for (uint32_t i = 0; i < ctx->L; ++i)
        if (P >= ctx->q[i]) return set_error(HC_ERR_INVALID_ARG, "P must be below every q_i");
    ZpConvGeom g;
    st = zp_conv_geometry(desc, ctx->N, &g);
    if (st != HC_OK) return st;
    const uint32_t N = ctx->N, kk = desc->kh * desc->kw;
    const size_t n = (size_t)g.Y * kk * desc->C, kw_ = (size_t)desc->M * desc->C * kk;
    if (out_words < n * ctx->L * N)
        return set_error(HC_ERR_INVALID_ARG, "d_out holds %zu words, %zu needed", out_words, n * ctx->L * N);
    for (size_t i = 0; i < kw_; ++i)
        if (h_K[i] >= P) return set_error(HC_ERR_RANGE, "kernel entry %zu is not below P", i);
    DeviceGuard dg(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    // scratch: K, then slot vectors and their encodings for up to kChunk plaintexts at a time
    constexpr size_t kChunk = 1024;
    const size_t chunk = n < kChunk ? n : kChunk;
    const size_t k_words = (kw_ + 31) & ~(size_t)31;
    Scratch tmp(s);
    tmp.p = dev_alloc((k_words + 2 * chunk * N) * sizeof(uint64_t), s);
    if (!tmp.p) return set_error(HC_ERR_OOM, "scratch allocation failed");
    uint64_t *dK = (uint64_t *)tmp.p, *slots = dK + k_words, *poly = slots + chunk * N;
    HC_CUDA_TRY(cudaMemcpyAsync(dK, h_K, kw_ * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    for (size_t p0 = 0; p0 < n; p0 += chunk) {
        const size_t m = n - p0 < chunk ? n - p0 : chunk, total = m * N;
        {
            ProfileScope ps("k_zp_conv_slots", s);
            k_zp_conv_slots<<<grid_for(ctx_p, total), 256, 0, s>>>(dK, slots, desc->M, desc->C, kk, p0, N, total);
            HC_CUDA_TRY(cudaGetLastError());
        }
        st = encode_into(ctx_p, slots, m, poly, s);
        if (st == HC_OK) st = lift_ntt_into(ctx, P, poly, m, d_out + p0 * ctx->L * N, s);
        if (st != HC_OK) return st;
    }
    HC_CUDA_TRY(cudaStreamSynchronize(s));  // the host kernel must outlive the upload
    return HC_OK;
}

}  // extern "C"
