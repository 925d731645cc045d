// hc_rotate.cu -- slot rotations of RLWE ciphertexts and the
// multiply-accumulate-rotate iteration of HELiKs-style linear layers over Z_P
// (SecONNds-P, Sec. 6.1: each iteration multiplies the input ciphertext by an
// NTT-preprocessed weight plaintext, accumulates, and rotates the accumulator
// by one slot; Sec. 2.1: rotations need a key-switching step with public
// evaluation keys).
//
// A rotation is the Galois automorphism sigma_g (X -> X^g) followed by key
// switching with one special prime p_sp and one digit per ciphertext limb:
//   d = sigma_g(c1);  D_j = d mod q_j lifted to every modulus of Q*p_sp;
//   (u0, u1) = sum_j NTT(D_j) . k_j over Q*p_sp, back to coefficients;
//   v = (u - [u]_{p_sp}) / p_sp over Q, [.] the centered residue;
//   out = (sigma_g(c0) + v0, v1).
// The key k_j = (b_j, a_j), b_j = -a_j s + e_j + p_sp * Qh_j [Qh_j^-1]_{q_j} sigma_g(s)
// (Qh_j = Q / q_j), comes from the secret-key holder; the GPU keeps it in the
// NTT domain over Q*p_sp.
#include <algorithm>
#include <new>
#include <vector>

#include "hc_arith.cuh"
#include "hc_internal.h"

// per ciphertext limb i: p_sp mod q_i, p_sp^-1 mod q_i with its Shoup companion
struct ModDown {
    uint64_t p_mod_q, pinv, pinv_s;
};

struct hc_galois_key {
    uint32_t magic;
    const hc_ctx *ctx;     // ciphertext context: q_0 .. q_{L-1}
    hc_ctx *qp;            // owned: q_0 .. q_{L-1}, p_sp
    int device;
    uint32_t g, ginv;      // Galois element and its inverse mod 2N
    uint64_t special;
    uint64_t *d_key;       // [L][2][L+1][N], NTT domain over Q*p_sp
    ModDown *d_md;         // [L]
};

namespace hc {
namespace {

__device__ __forceinline__ uint64_t negmod(uint64_t v, uint64_t q) { return v ? q - v : 0; }

__device__ __forceinline__ uint64_t reduce_any(uint64_t v, const LimbConst &lc)
{
    return canon3(reduce_lazy(v, (uint32_t)lc.one_s, 0ull - lc.q), lc.q);
}

// The three kernels below run on 2-D grids: blockIdx.y walks the rows (one
// polynomial limb of the output per row, the row's indices decoded once per
// block), x the N coefficients (N a power of two, so no division per element).
constexpr uint32_t kKsBlock = 256;

// digits of sigma_g(c1): dig[ct][j][i][k] = sigma_g(c1)[j][k] mod m_i over the L+1
// moduli m_i of Q*p_sp (gather: output coefficient k takes source k*ginv mod 2N);
// rows (ct, j)
__global__ void k_ks_digits(const uint64_t *__restrict__ ct, uint64_t *__restrict__ dig,
                            const LimbConst *__restrict__ lq, const LimbConst *__restrict__ lqp, uint32_t L,
                            uint32_t N, uint32_t ginv, uint32_t rows)
{
    const uint32_t k = blockIdx.x * kKsBlock + threadIdx.x;
    const uint32_t mask2 = 2 * N - 1;
    const uint32_t src = (uint32_t)(((uint64_t)k * ginv) & mask2);
    for (uint32_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const uint32_t c = r / L, j = r - c * L;
        const uint64_t qj = lq[j].q;
        const uint64_t *c1 = ct + ((size_t)(c * 2 + 1) * L + j) * N;
        const uint64_t v = src < N ? c1[src] : negmod(c1[src - N], qj);
        uint64_t *d = dig + (size_t)r * (L + 1) * N + k;
        for (uint32_t i = 0; i <= L; ++i) d[(size_t)i * N] = i == j ? v : reduce_any(v, lqp[i]);
    }
}

// u[ct][comp][i][k] = sum_j dig[ct][j][i][k] * key[j][comp][i][k] mod m_i (NTT domain);
// rows (ct, i)
__global__ void k_ks_mac(const uint64_t *__restrict__ dig, const uint64_t *__restrict__ key,
                         uint64_t *__restrict__ u, const LimbConst *__restrict__ lqp, uint32_t L, uint32_t N,
                         uint32_t rows)
{
    const uint32_t k = blockIdx.x * kKsBlock + threadIdx.x;
    const uint32_t L1 = L + 1;
    for (uint32_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const uint32_t c = r / L1, i = r - c * L1;
        const LimbConst &lc = lqp[i];
        const uint64_t q = lc.q, nq = 0ull - q;
        MacAcc a0, a1;
        mac_zero(a0);
        mac_zero(a1);
        for (uint32_t j = 0; j < L; ++j) {
            const uint64_t x = dig[((size_t)(c * L + j) * L1 + i) * N + k];
            mac_add(a0, x, key[((size_t)(j * 2) * L1 + i) * N + k]);
            mac_add(a1, x, key[((size_t)(j * 2 + 1) * L1 + i) * N + k]);
        }
        const uint32_t ones = (uint32_t)lc.one_s;
        u[((size_t)(c * 2) * L1 + i) * N + k] = mac_reduce(a0, q, nq, lc.r64, lc.r64_s, ones);
        u[((size_t)(c * 2 + 1) * L1 + i) * N + k] = mac_reduce(a1, q, nq, lc.r64, lc.r64_s, ones);
    }
}

// out[ct][comp][i][k] = (comp == 0 ? sigma_g(c0)[i][k] : 0) + (u_i - [u_sp]) / p_sp
//                       (+ add[ct][comp][i][k] when add is given) mod q_i;  rows (ct, comp, i)
// (add may be out itself: each element is read before it is written, by the same thread)
__global__ void k_ks_mod_down(const uint64_t *__restrict__ ct, const uint64_t *__restrict__ u, uint64_t *out,
                              const uint64_t *add, const LimbConst *__restrict__ lq,
                              const ModDown *__restrict__ md, uint64_t special, uint32_t L, uint32_t N,
                              uint32_t ginv, uint32_t rows)
{
    const uint32_t k = blockIdx.x * kKsBlock + threadIdx.x;
    const uint32_t mask2 = 2 * N - 1, L1 = L + 1;
    const uint64_t half = (special - 1) / 2;
    const uint32_t src = (uint32_t)(((uint64_t)k * ginv) & mask2);
    for (uint32_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const uint32_t cc = r / L, i = r - cc * L;  // cc = ct * 2 + comp
        const uint32_t comp = cc & 1;
        const LimbConst &lc = lq[i];
        const uint64_t q = lc.q;
        const uint64_t ui = u[((size_t)cc * L1 + i) * N + k];
        const uint64_t usp = u[((size_t)cc * L1 + L) * N + k];
        const uint64_t rsp = reduce_any(usp, lc);  // usp mod q_i
        // the centered residue: usp - p_sp when usp > (p_sp - 1) / 2
        const uint64_t pm = md[i].p_mod_q;
        const uint64_t cen = usp > half ? (rsp >= pm ? rsp - pm : rsp + q - pm) : rsp;
        const uint64_t diff = ui >= cen ? ui - cen : ui + q - cen;
        uint64_t v = canon4(shoup_lazy(diff, md[i].pinv, md[i].pinv_s, 0ull - q), q);
        if (comp == 0) {
            const uint64_t *c0 = ct + ((size_t)cc * L + i) * N;
            const uint64_t a = src < N ? c0[src] : negmod(c0[src - N], q);
            v = csub(v + a, q);
        }
        const size_t o = (size_t)r * N + k;
        if (add) v = csub(v + add[o], q);
        out[o] = v;
    }
}

// grid of one of the kernels above: N / kKsBlock blocks across, rows (at most 65535) down
dim3 ks_grid(uint32_t N, size_t rows)
{
    return dim3(N / kKsBlock, (unsigned)(rows < 65535 ? (rows ? rows : 1) : 65535));
}

// term list of mn outputs with one term each: output o = ciphertext o mod m times
// plaintext o / m
__global__ void k_outer_terms(uint32_t *term_ptr, uint32_t *terms, uint32_t m, uint32_t mn)
{
    for (uint32_t o = blockIdx.x * blockDim.x + threadIdx.x; o <= mn; o += gridDim.x * blockDim.x) {
        term_ptr[o] = o;
        if (o < mn) {
            terms[2 * o] = o % m;
            terms[2 * o + 1] = o / m;
        }
    }
}

// term list of a Z_P convolution's products: output o = i*Y + y (kernel offset i,
// output ciphertext y) sums the C terms (input c, weight plaintext (y*kk + i)*C + c)
__global__ void k_conv_terms(uint32_t *term_ptr, uint32_t *terms, uint32_t Y, uint32_t kk, uint32_t C,
                             uint32_t n_out)
{
    for (uint32_t o = blockIdx.x * blockDim.x + threadIdx.x; o <= n_out; o += gridDim.x * blockDim.x) {
        term_ptr[o] = o * C;
        if (o < n_out) {
            const uint32_t i = o / Y, y = o % Y;
            for (uint32_t c = 0; c < C; ++c) {
                terms[2 * (o * C + c)] = c;
                terms[2 * (o * C + c) + 1] = (y * kk + i) * C + c;
            }
        }
    }
}

struct Buf {
    void *p = nullptr;
    cudaStream_t s;
    explicit Buf(cudaStream_t st) : s(st) {}
    ~Buf() { dev_free(p, s); }
};

bool key_ok(const hc_galois_key *k) { return k && k->magic == kMagicGaloisKey; }

// out = rotate(in) (+ add, elementwise, when given; add may equal out, not in)
hc_status rotate_into(const hc_ctx *ctx, const hc_galois_key *key, const uint64_t *in, uint64_t *out, size_t n,
                      cudaStream_t s, const uint64_t *add = nullptr)
{
    const uint32_t L = ctx->L, N = ctx->N;
    const size_t dig_words = n * L * (L + 1) * (size_t)N, u_words = n * 2 * (L + 1) * (size_t)N;
    Buf dig(s), u(s);
    dig.p = dev_alloc(dig_words * 8, s);
    u.p = dev_alloc(u_words * 8, s);
    if (!dig.p || !u.p) return set_error(HC_ERR_OOM, "scratch allocation failed");
    uint64_t *dd = (uint64_t *)dig.p, *uu = (uint64_t *)u.p;
    if ((size_t)n * 2 * (L + 1) > 0xffffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    {
        ProfileScope ps("k_ks_digits", s);
        const uint32_t rows = (uint32_t)(n * L);
        k_ks_digits<<<ks_grid(N, rows), kKsBlock, 0, s>>>(in, dd, ctx->d_limbs, key->qp->d_limbs, L, N, key->ginv,
                                                         rows);
        HC_CUDA_TRY(cudaGetLastError());
    }
    hc_status st = launch_ntt_fwd(key->qp, dd, dd, n * L, s);  // digits: n*L polys over Q*p_sp
    if (st != HC_OK) return st;
    {
        ProfileScope ps("k_ks_mac", s);
        const uint32_t rows = (uint32_t)(n * (L + 1));
        k_ks_mac<<<ks_grid(N, rows), kKsBlock, 0, s>>>(dd, key->d_key, uu, key->qp->d_limbs, L, N, rows);
        HC_CUDA_TRY(cudaGetLastError());
    }
    st = launch_ntt_inv(key->qp, uu, uu, 2 * n, s);
    if (st != HC_OK) return st;
    ProfileScope ps("k_ks_mod_down", s);
    const uint32_t rows = (uint32_t)(n * 2 * L);
    k_ks_mod_down<<<ks_grid(N, rows), kKsBlock, 0, s>>>(in, uu, out, add, ctx->d_limbs, key->d_md, key->special, L,
                                                        N, key->ginv, rows);
    HC_CUDA_TRY(cudaGetLastError());
    return HC_OK;
}

}  // namespace

void galois_key_destroy(hc_galois_key *k)
{
    DeviceGuard g(k->device);
    dev_free_persistent(k->d_key);
    dev_free_persistent(k->d_md);
    hc_free(k->qp);
    k->magic = kMagicDead;
    delete k;
}

}  // namespace hc

using namespace hc;

extern "C" {

hc_status hc_galois_key_create(const hc_ctx *ctx, uint64_t special_prime, uint32_t galois_elt, const uint64_t *h_key,
                               hc_galois_key **out, void *cuda_stream)
{
    if (!out) return set_error(HC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx || ctx->magic != kMagicCtx) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (!h_key) return set_error(HC_ERR_INVALID_ARG, "h_key is NULL");
    const uint32_t L = ctx->L, N = ctx->N;
    if (L + 1 > kMaxLimbs) return set_error(HC_ERR_INVALID_ARG, "no room for the special prime (L = %u)", L);
    if (!(galois_elt & 1) || galois_elt >= 2 * N)
        return set_error(HC_ERR_INVALID_ARG, "Galois element must be odd and below 2N (got %u)", galois_elt);
    for (uint32_t i = 0; i < L; ++i)
        if (ctx->q[i] == special_prime) return set_error(HC_ERR_BAD_MODULUS, "special prime equals q[%u]", i);
    DeviceGuard dg(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    uint64_t moduli[kMaxLimbs];
    for (uint32_t i = 0; i < L; ++i) moduli[i] = ctx->q[i];
    moduli[L] = special_prime;
    hc_ctx *qp = nullptr;
    hc_status st = hc_ctx_create_ex(N, moduli, L + 1, ctx->t, 0, &qp);  // validates the special prime
    if (st != HC_OK) return st;
    hc_galois_key *k = new (std::nothrow) hc_galois_key();
    if (!k) {
        hc_free(qp);
        return set_error(HC_ERR_OOM, "host allocation failed");
    }
    k->magic = kMagicGaloisKey;
    k->ctx = ctx;
    k->qp = qp;
    k->device = ctx->device;
    k->g = galois_elt;
    uint32_t ginv = 1;
    while ((uint64_t)ginv * galois_elt % (2 * N) != 1) ginv += 2;  // odd residues form a group mod 2N
    k->ginv = ginv;
    k->special = special_prime;
    std::vector<ModDown> md(L);
    for (uint32_t i = 0; i < L; ++i) {
        const uint64_t q = ctx->q[i];
        md[i].p_mod_q = special_prime % q;
        md[i].pinv = powmod_u64(md[i].p_mod_q, q - 2, q);
        md[i].pinv_s = shoup_companion(md[i].pinv, q);
    }
    const size_t key_words = (size_t)L * 2 * (L + 1) * N;
    k->d_key = (uint64_t *)dev_alloc_persistent(key_words * 8);
    k->d_md = (ModDown *)dev_alloc_persistent(L * sizeof(ModDown));
    if (!k->d_key || !k->d_md) {
        galois_key_destroy(k);
        return set_error(HC_ERR_OOM, "device allocation of the Galois key failed");
    }
    cudaError_t e = cudaMemcpy(k->d_key, h_key, key_words * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(k->d_md, md.data(), L * sizeof(ModDown), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        galois_key_destroy(k);
        return cuda_error(e, "uploading the Galois key");
    }
    st = check_inputs(qp, k->d_key, (size_t)2 * L, s);
    if (st == HC_OK) st = launch_ntt_fwd(qp, k->d_key, k->d_key, (size_t)2 * L, s);
    if (st == HC_OK) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "Galois key preprocessing");
    }
    if (st != HC_OK) {
        galois_key_destroy(k);
        return st;
    }
    *out = k;
    return HC_OK;
}

hc_status hc_ct_rotate(const hc_ctx *ctx, const hc_galois_key *key, const uint64_t *d_ct_in, uint64_t *d_ct_out,
                       size_t n_ct, void *cuda_stream)
{
    if (!ctx || ctx->magic != kMagicCtx || !key_ok(key)) return set_error(HC_ERR_INVALID_ARG, "invalid context or key");
    if (key->ctx != ctx) return set_error(HC_ERR_INVALID_ARG, "key was made for another context");
    if (n_ct == 0) return HC_OK;
    if (!d_ct_in || !d_ct_out) return set_error(HC_ERR_INVALID_ARG, "null ciphertext buffer");
    if (d_ct_in == d_ct_out) return set_error(HC_ERR_INVALID_ARG, "in place rotation is not supported");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    hc_status st = check_inputs(ctx, d_ct_in, 2 * n_ct, s);
    if (st != HC_OK) return st;
    return rotate_into(ctx, key, d_ct_in, d_ct_out, n_ct, s);
}

hc_status hc_mac_rotate_many(const hc_ctx *ctx, const hc_galois_key *key, const uint64_t *d_ct, uint32_t m,
                             const uint64_t *d_w_ntt, uint32_t n, uint64_t *d_out, void *cuda_stream)
{
    if (!ctx || ctx->magic != kMagicCtx || !key_ok(key)) return set_error(HC_ERR_INVALID_ARG, "invalid context or key");
    if (key->ctx != ctx) return set_error(HC_ERR_INVALID_ARG, "key was made for another context");
    if (!d_ct || !d_w_ntt || !d_out || n == 0 || m == 0) return set_error(HC_ERR_INVALID_ARG, "null buffer or empty batch");
    if ((uint64_t)n * m > 0x3fffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    hc_status st = check_inputs(ctx, d_ct, (size_t)2 * m, s);
    if (st == HC_OK) st = check_inputs(ctx, d_w_ntt, n, s);
    if (st != HC_OK) return st;
    // The products x_j * w_i do not depend on the accumulators: all m*n run first, in
    // one launch (forward NTT of the x_j once, then one MAC + inverse NTT per product);
    // the chain then only rotates and adds, all m accumulators per step, the add fused
    // into the key switch's last kernel:
    //   P_i = x * w_i (m ciphertexts);  acc = P_{n-1};  acc = rot(acc) + P_i, i = n-2 .. 0.
    const uint32_t L = ctx->L, N = ctx->N;
    const size_t ct_words = (size_t)2 * L * N, mn = (size_t)m * n;
    const size_t term_words = (3 * mn + 1 + 1) / 2;  // mn + 1 offsets and 2mn indices, as uint32
    Buf tmp(s);
    tmp.p = dev_alloc(((mn + m) * ct_words + term_words) * 8, s);
    if (!tmp.p) return set_error(HC_ERR_OOM, "scratch allocation failed");
    uint64_t *ctn = (uint64_t *)tmp.p, *prods = ctn + (size_t)m * ct_words;  // prods [n][m][2][L][N]
    uint32_t *term_ptr = reinterpret_cast<uint32_t *>(prods + mn * ct_words), *terms = term_ptr + mn + 1;
    st = launch_ntt_fwd(ctx, d_ct, ctn, (size_t)2 * m, s);
    if (st != HC_OK) return st;
    k_outer_terms<<<(unsigned)((mn + 256) / 256), 256, 0, s>>>(term_ptr, terms, m, (uint32_t)mn);
    HC_CUDA_TRY(cudaGetLastError());
    uint64_t *first = n == 1 ? d_out : prods;  // P_0 of a one-term iteration is the result
    st = launch_mac_intt(ctx, ctn, d_w_ntt, MacTerms{term_ptr, terms}, first, mn, s);
    if (st != HC_OK || n == 1) return st;
    const size_t step = (size_t)m * ct_words;
    const uint64_t *acc = prods + (size_t)(n - 1) * step;
    for (uint32_t i = n - 1; i-- > 0;) {
        uint64_t *pi = prods + (size_t)i * step;
        uint64_t *dst = i == 0 ? d_out : pi;
        st = rotate_into(ctx, key, acc, dst, m, s, pi);
        if (st != HC_OK) return st;
        acc = dst;
    }
    return HC_OK;
}

hc_status hc_mac_rotate(const hc_ctx *ctx, const hc_galois_key *key, const uint64_t *d_ct, const uint64_t *d_w_ntt,
                        uint32_t n, uint64_t *d_out, void *cuda_stream)
{
    return hc_mac_rotate_many(ctx, key, d_ct, 1, d_w_ntt, n, d_out, cuda_stream);
}

hc_status hc_zp_plain_preprocess(const hc_ctx *ctx, uint64_t P, const uint64_t *h_plain, size_t n, uint64_t *d_out,
                                 void *cuda_stream)
{
    if (!ctx || ctx->magic != kMagicCtx) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (n == 0) return HC_OK;
    if (!h_plain || !d_out) return set_error(HC_ERR_INVALID_ARG, "null buffer");
    if (P < 3 || P >= (1ull << 50)) return set_error(HC_ERR_INVALID_ARG, "plaintext modulus out of range");
    const uint32_t L = ctx->L, N = ctx->N;
    // centered lift of every coefficient into each q_i, on the host; NTT on the device
    std::vector<uint64_t> lifted(n * L * N);
    for (size_t p = 0; p < n; ++p)
        for (uint32_t k = 0; k < N; ++k) {
            const uint64_t v = h_plain[p * N + k];
            if (v >= P) return set_error(HC_ERR_RANGE, "plaintext coefficient %llu >= P", (unsigned long long)v);
            const bool neg = v > (P - 1) / 2;
            for (uint32_t i = 0; i < L; ++i) {
                const uint64_t q = ctx->q[i];
                lifted[(p * L + i) * N + k] = neg ? q - (P - v) % q : v % q;
            }
        }
    DeviceGuard dg(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    HC_CUDA_TRY(cudaMemcpyAsync(d_out, lifted.data(), lifted.size() * 8, cudaMemcpyHostToDevice, s));
    hc_status st = launch_ntt_fwd(ctx, d_out, d_out, n, s);
    if (st != HC_OK) return st;
    HC_CUDA_TRY(cudaStreamSynchronize(s));  // the host copy must outlive the upload
    return HC_OK;
}

hc_status hc_zp_conv(const hc_ctx *ctx, const hc_conv_desc *desc, const hc_galois_key *key_1,
                     const hc_galois_key *key_row, const uint64_t *d_w_ntt, const uint64_t *d_ct_in,
                     uint64_t *d_ct_out, void *cuda_stream)
{
    if (!ctx || ctx->magic != kMagicCtx) return set_error(HC_ERR_INVALID_ARG, "invalid context");
    if (!desc || !d_w_ntt || !d_ct_in || !d_ct_out) return set_error(HC_ERR_INVALID_ARG, "null descriptor or buffer");
    ZpConvGeom g;
    hc_status st = zp_conv_geometry(desc, ctx->N, &g);
    if (st != HC_OK) return st;
    const uint32_t L = ctx->L, N = ctx->N, C = desc->C, kk = desc->kh * desc->kw, Y = g.Y;
    // the two rotations of the iteration: by 1 slot within a kernel row, by Wp - kw + 1 to the next
    const uint32_t g1 = 5, grow = (uint32_t)powmod_u64(5, g.step_row, 2ull * N);
    if (desc->kw > 1 && (!key_ok(key_1) || key_1->ctx != ctx || key_1->g != g1))
        return set_error(HC_ERR_INVALID_ARG, "key_1 must be a Galois key of element 5 for this context");
    if (desc->kh > 1 && (!key_ok(key_row) || key_row->ctx != ctx || key_row->g != grow))
        return set_error(HC_ERR_INVALID_ARG, "key_row must be a Galois key of element 5^%u mod 2N = %u", g.step_row,
                         grow);
    const uint64_t n_out64 = (uint64_t)kk * Y;
    if (n_out64 * C > 0x3fffffffu) return set_error(HC_ERR_INVALID_ARG, "layer too large");
    const uint32_t n_out = (uint32_t)n_out64;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    st = check_inputs(ctx, d_ct_in, (size_t)2 * C, s);
    if (st != HC_OK) return st;
    // P_{y,i} = sum_c x_c * w_{y,i,c}: forward NTT of the C inputs once, then one MAC +
    // inverse NTT launch over the kk*Y outputs (ordered [i][y], so that the chain's step
    // i rotates all Y accumulators at once); the chain then rotates and adds, the add
    // fused into the key switch's last kernel:
    //   acc = P_{kk-1};  acc = rot^(step_i)(acc) + P_i, i = kk-2 .. 0.
    const size_t ct_words = (size_t)2 * L * N;
    const size_t prod_words = kk > 1 ? (size_t)n_out * ct_words : 0;
    const size_t term_words = ((size_t)n_out + 1 + 2 * (size_t)n_out * C + 1) / 2;
    Buf tmp(s);
    tmp.p = dev_alloc(((size_t)C * ct_words + prod_words + term_words) * 8, s);
    if (!tmp.p) return set_error(HC_ERR_OOM, "scratch allocation failed");
    uint64_t *ctn = (uint64_t *)tmp.p, *prods = ctn + (size_t)C * ct_words;
    uint32_t *term_ptr = reinterpret_cast<uint32_t *>(prods + prod_words), *terms = term_ptr + n_out + 1;
    st = launch_ntt_fwd(ctx, d_ct_in, ctn, (size_t)2 * C, s);
    if (st != HC_OK) return st;
    k_conv_terms<<<(n_out + 256) / 256, 256, 0, s>>>(term_ptr, terms, Y, kk, C, n_out);
    HC_CUDA_TRY(cudaGetLastError());
    st = launch_mac_intt(ctx, ctn, d_w_ntt, MacTerms{term_ptr, terms}, kk == 1 ? d_ct_out : prods, n_out, s);
    if (st != HC_OK || kk == 1) return st;
    const size_t step = (size_t)Y * ct_words;
    const uint64_t *acc = prods + (size_t)(kk - 1) * step;
    for (uint32_t i = kk - 1; i-- > 0;) {
        // offsets i and i + 1 lie in one kernel row unless i + 1 starts a new one
        const hc_galois_key *key = (i + 1) % desc->kw == 0 ? key_row : key_1;
        uint64_t *pi = prods + (size_t)i * step;
        uint64_t *dst = i == 0 ? d_ct_out : pi;
        st = rotate_into(ctx, key, acc, dst, Y, s, pi);
        if (st != HC_OK) return st;
        acc = dst;
    }
    return HC_OK;
}

}  // extern "C"
