/*
 * hc_oracle.c — plain, slow, obviously-correct CPU oracle for the HE
 * convolution hot path of SecONNds (arXiv 2506.11586).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library links, includes or
 * calls this file; only tests/, the smoke check and the CPU-baseline leg of
 * the benchmark load it.  It shares no code, header or table with the CUDA
 * path.
 *
 * Every routine is the textbook definition, written with unsigned __int128
 * and the % operator, with no blocking, reordering or fast reduction:
 *
 *   - ring R_q = Z_q[X]/(X^N + 1)                        (Sec. 2.1)
 *   - negacyclic product c = a*b in R_q                  (App. C; the printed
 *     sum omits the X^N = -1 wrap term, the ring forces it, so it is added)
 *   - NTT: evaluation at the odd powers of a primitive 2N-th root psi,
 *     output slot k holding a(psi^(2*rev(k)+1))         (App. C.1)
 *   - INTT: the exact inverse of that map (natural order, N^-1 folded in)
 *   - deterministic Miller-Rabin, NTT-friendly prime search, minimal psi
 *     (the paper fixes none of N, Q, psi; these are the readings used)
 *
 * OpenMP only splits independent output coefficients across threads; the
 * arithmetic of each coefficient is the plain sum.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>

typedef unsigned __int128 u128;

/* ---- scalar modular arithmetic (definition: (a*b) mod q) ---------------- */

uint64_t or_mulmod(uint64_t a, uint64_t b, uint64_t q)
{
    return (uint64_t)(((u128)a * (u128)b) % (u128)q);
}

uint64_t or_addmod(uint64_t a, uint64_t b, uint64_t q)
{
    return (uint64_t)(((u128)a + (u128)b) % (u128)q);
}

uint64_t or_submod(uint64_t a, uint64_t b, uint64_t q)
{
    /* (a - b) mod q for a, b in [0, q) */
    return (uint64_t)(((u128)a + (u128)q - (u128)(b % q)) % (u128)q);
}

uint64_t or_powmod(uint64_t base, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    uint64_t b = base % q;
    while (e) {
        if (e & 1) r = or_mulmod(r, b, q);
        b = or_mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}

/* ---- primality: deterministic Miller-Rabin, bases 2..37 ------------------
 * The first twelve primes as bases decide primality for every n < 3.3e24,
 * which covers all 64-bit integers. */
int or_is_prime(uint64_t n)
{
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; ++i) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (int i = 0; i < 12; ++i) {
        uint64_t x = or_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; ++r) {
            x = or_mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* The `count` largest primes q < 2^bits with q = 1 (mod 2^log2_step), in
 * descending order.  Returns how many were written (fewer only if the range
 * runs out).  This is the canonical prime choice of the build: the paper
 * names neither N nor Q. */
size_t or_ntt_primes(uint32_t bits, uint32_t log2_step, size_t count, uint64_t *out)
{
    if (bits < 2 || bits > 62 || log2_step >= bits) return 0;
    uint64_t step = (uint64_t)1 << log2_step;
    uint64_t limit = (uint64_t)1 << bits;       /* q < limit */
    uint64_t q = ((limit - 1) / step) * step + 1;
    if (q >= limit) q -= step;
    size_t n = 0;
    while (n < count && q > step) {
        if (or_is_prime(q)) out[n++] = q;
        q -= step;
    }
    return n;
}

/* ---- minimal primitive 2N-th root of unity --------------------------------
 * For 2N a power of two, x is a primitive 2N-th root iff x^N = -1 (mod q).
 * Find one such root w, then the whole set is { w^k : k odd, k < 2N }; the
 * canonical psi is its minimum.  Returns 0 when q != 1 (mod 2N) or no root
 * is found. */
uint64_t or_min_psi(uint64_t q, uint32_t N)
{
    uint64_t twoN = 2ull * N;
    if (N == 0 || (q - 1) % twoN != 0) return 0;
    uint64_t w = 0;
    for (uint64_t c = 2; c < q && c < 1000000; ++c) {
        uint64_t x = or_powmod(c, (q - 1) / twoN, q);
        if (or_powmod(x, N, q) == q - 1) { w = x; break; }
    }
    if (w == 0) return 0;
    uint64_t w2 = or_mulmod(w, w, q);
    uint64_t cur = w, best = w;           /* cur = w^k, k odd */
    for (uint64_t k = 1; k < twoN; k += 2) {
        if (cur < best) best = cur;
        cur = or_mulmod(cur, w2, q);
    }
    return best;
}

uint32_t or_bitrev(uint32_t k, uint32_t logn)
{
    uint32_t r = 0;
    for (uint32_t i = 0; i < logn; ++i) r |= ((k >> i) & 1u) << (logn - 1 - i);
    return r;
}

static uint32_t ilog2_u32(uint32_t n)
{
    uint32_t l = 0;
    while ((1u << l) < n) ++l;
    return l;
}

/* ---- NTT by its definition: O(N^2) ----------------------------------------
 * out[k] = sum_j a[j] * psi^((2*rev(k)+1)*j)  (mod q).
 * Only the output indices listed in ks (nk of them) are computed; ks == NULL
 * means all N, in order. */
void or_ntt_direct_at(const uint64_t *a, uint32_t N, uint64_t q, uint64_t psi,
                      const uint32_t *ks, size_t nk, uint64_t *out)
{
    uint32_t logn = ilog2_u32(N);
    size_t cnt = ks ? nk : N;
    #pragma omp parallel for schedule(dynamic, 8)
    for (size_t ii = 0; ii < cnt; ++ii) {
        uint32_t k = ks ? ks[ii] : (uint32_t)ii;
        uint64_t x = or_powmod(psi, 2ull * or_bitrev(k, logn) + 1, q);
        uint64_t xp = 1, acc = 0;
        for (uint32_t j = 0; j < N; ++j) {
            acc = or_addmod(acc, or_mulmod(a[j] % q, xp, q), q);
            xp = or_mulmod(xp, x, q);
        }
        out[ii] = acc;
    }
}

void or_ntt_direct(const uint64_t *a, uint32_t N, uint64_t q, uint64_t psi, uint64_t *out)
{
    or_ntt_direct_at(a, N, q, psi, NULL, 0, out);
}

/* Inverse of the map above: a[j] = N^-1 * sum_k A[k] * psi^(-(2*rev(k)+1)*j).
 * Computes the coefficient indices listed in js (all N when js == NULL). */
void or_intt_direct_at(const uint64_t *A, uint32_t N, uint64_t q, uint64_t psi,
                       const uint32_t *js, size_t nj, uint64_t *out)
{
    uint32_t logn = ilog2_u32(N);
    uint64_t psi_inv = or_powmod(psi, q - 2, q);
    uint64_t n_inv = or_powmod(N % q, q - 2, q);
    size_t cnt = js ? nj : N;
    #pragma omp parallel for schedule(dynamic, 8)
    for (size_t ii = 0; ii < cnt; ++ii) {
        uint32_t j = js ? js[ii] : (uint32_t)ii;
        uint64_t acc = 0;
        for (uint32_t k = 0; k < N; ++k) {
            uint64_t e = ((2ull * or_bitrev(k, logn) + 1) * (uint64_t)j) % (2ull * N);
            acc = or_addmod(acc, or_mulmod(A[k] % q, or_powmod(psi_inv, e, q), q), q);
        }
        out[ii] = or_mulmod(acc, n_inv, q);
    }
}

void or_intt_direct(const uint64_t *A, uint32_t N, uint64_t q, uint64_t psi, uint64_t *out)
{
    or_intt_direct_at(A, N, q, psi, NULL, 0, out);
}

/* ---- negacyclic product by the schoolbook sum -----------------------------
 * c[k] = sum_{i+j=k} a[i] b[j]  -  sum_{i+j=k+N} a[i] b[j]   (mod q)
 * Coefficient k only (so a sample of outputs costs O(N) each). */
static uint64_t negacyclic_coeff(const uint64_t *a, const uint64_t *b, uint32_t N,
                                 uint64_t q, uint32_t k)
{
    u128 pos = 0, neg = 0;
    /* i + j = k with 0 <= i <= k */
    for (uint32_t i = 0; i <= k; ++i) {
        pos += (u128)or_mulmod(a[i] % q, b[k - i] % q, q);
        if (pos >= ((u128)1 << 120)) pos %= q;
    }
    /* i + j = k + N with k < i < N, j = k + N - i in (k, N) */
    for (uint32_t i = k + 1; i < N; ++i) {
        neg += (u128)or_mulmod(a[i] % q, b[k + N - i] % q, q);
        if (neg >= ((u128)1 << 120)) neg %= q;
    }
    uint64_t p = (uint64_t)(pos % q), n = (uint64_t)(neg % q);
    return or_submod(p, n, q);
}

void or_negacyclic_at(const uint64_t *a, const uint64_t *b, uint32_t N, uint64_t q,
                      const uint32_t *ks, size_t nk, uint64_t *out)
{
    size_t cnt = ks ? nk : N;
    #pragma omp parallel for schedule(dynamic, 16)
    for (size_t ii = 0; ii < cnt; ++ii) {
        uint32_t k = ks ? ks[ii] : (uint32_t)ii;
        out[ii] = negacyclic_coeff(a, b, N, q, k);
    }
}

void or_negacyclic(const uint64_t *a, const uint64_t *b, uint32_t N, uint64_t q, uint64_t *out)
{
    or_negacyclic_at(a, b, N, q, NULL, 0, out);
}

/* Batched dense product: n independent pairs, pair p uses modulus
 * qs[p % L] (layout [n/L][L][N] when the batch is [item][limb]). */
void or_negacyclic_batch(const uint64_t *a, const uint64_t *b, size_t n, uint32_t N,
                         const uint64_t *qs, uint32_t L, uint64_t *out)
{
    #pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (size_t p = 0; p < n; ++p)
        for (uint32_t k = 0; k < N; ++k)
            out[p * N + k] = negacyclic_coeff(a + p * N, b + p * N, N, qs[p % L], k);
}

/* Same sum when b has small signed integer coefficients given as a sparse
 * list (idx[t], val[t]), t < nnz: only the nonzero terms of the schoolbook
 * sum are visited.  b is lifted to R_q as val mod q.  Used for conv weight
 * plaintexts (int8) and ternary secret keys.  Coefficients listed in ks
 * (all N when ks == NULL). */
void or_negacyclic_sparse_at(const uint64_t *a, const uint32_t *idx, const int64_t *val,
                             size_t nnz, uint32_t N, uint64_t q,
                             const uint32_t *ks, size_t nk, uint64_t *out)
{
    size_t cnt = ks ? nk : N;
    #pragma omp parallel for schedule(static)
    for (size_t ii = 0; ii < cnt; ++ii) {
        uint32_t k = ks ? ks[ii] : (uint32_t)ii;
        uint64_t acc = 0;
        for (size_t t = 0; t < nnz; ++t) {
            uint32_t j = idx[t];                 /* b has term val * X^j */
            int64_t v = val[t];
            uint64_t vq = v >= 0 ? ((uint64_t)v) % q : q - ((uint64_t)(-v)) % q;
            if (vq == q) vq = 0;
            uint64_t term;
            int negate;
            if (j <= k) { term = or_mulmod(a[k - j] % q, vq, q); negate = 0; }
            else        { term = or_mulmod(a[k + N - j] % q, vq, q); negate = 1; }
            acc = negate ? or_submod(acc, term, q) : or_addmod(acc, term, q);
        }
        out[ii] = acc;
    }
}

/* The same schoolbook sum when b is ternary (coefficients in {-1, 0, 1}),
 * given as the index lists of its +1 and -1 coefficients: every term is
 * +-a[.], so the sum needs additions only.  a must hold canonical residues
 * (< q).  Coefficients listed in ks (all N when ks == NULL). */
void or_negacyclic_ternary_at(const uint64_t *a, const uint32_t *pos, size_t npos,
                              const uint32_t *neg, size_t nneg, uint32_t N, uint64_t q,
                              const uint32_t *ks, size_t nk, uint64_t *out)
{
    size_t cnt = ks ? nk : N;
    #pragma omp parallel for schedule(static)
    for (size_t ii = 0; ii < cnt; ++ii) {
        uint32_t k = ks ? ks[ii] : (uint32_t)ii;
        u128 plus = 0, minus = 0;
        for (size_t t = 0; t < npos; ++t) {
            uint32_t j = pos[t];
            if (j <= k) plus += a[k - j]; else minus += a[k + N - j];
        }
        for (size_t t = 0; t < nneg; ++t) {
            uint32_t j = neg[t];
            if (j <= k) minus += a[k - j]; else plus += a[k + N - j];
        }
        out[ii] = or_submod((uint64_t)(plus % q), (uint64_t)(minus % q), q);
    }
}
