// hc_host.cu -- host-side support of libhconv: errors, allocation, device guard,
// number theory for context set-up, and the convolution partition / packing.
#include <cstdarg>
#include <cstring>

#include "hc_internal.h"

namespace hc {

// ---------------------------------------------------------------- errors ----
static thread_local char g_last_error[512] = "";

hc_status set_error(hc_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

hc_status cuda_error(cudaError_t e, const char *what)
{
    hc_status s = (e == cudaErrorMemoryAllocation) ? HC_ERR_OOM : HC_ERR_CUDA;
    return set_error(s, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

const char *last_error() { return g_last_error; }

// ------------------------------------------------------------ allocation ----
static hc_alloc_fn g_alloc = nullptr;
static hc_free_fn g_free = nullptr;
static void *g_user = nullptr;

void set_allocator(hc_alloc_fn a, hc_free_fn f, void *user)
{
    if (a == nullptr || f == nullptr) {
        g_alloc = nullptr;
        g_free = nullptr;
        g_user = nullptr;
    } else {
        g_alloc = a;
        g_free = f;
        g_user = user;
    }
}

void *dev_alloc(size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 256;
    if (g_alloc) return g_alloc(bytes, (void *)s, g_user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *p, cudaStream_t s)
{
    if (!p) return;
    if (g_free) {
        g_free(p, (void *)s, g_user);
        return;
    }
    cudaFreeAsync(p, s);
}

void *dev_alloc_persistent(size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (g_alloc) return g_alloc(bytes, nullptr, g_user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free_persistent(void *p)
{
    if (!p) return;
    if (g_free) {
        g_free(p, nullptr, g_user);
        return;
    }
    cudaFree(p);
}

DeviceGuard::DeviceGuard(int dev)
{
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
        if (cudaSetDevice(dev) == cudaSuccess) changed = true;
    }
}

DeviceGuard::~DeviceGuard()
{
    if (changed) cudaSetDevice(prev);
}

// --------------------------------------------------------- number theory ----
typedef unsigned __int128 u128;

uint64_t mulmod_u64(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }

uint64_t powmod_u64(uint64_t a, uint64_t e, uint64_t q)
{
    uint64_t acc = 1 % q, base = a % q;
    for (; e; e >>= 1) {
        if (e & 1) acc = mulmod_u64(acc, base, q);
        base = mulmod_u64(base, base, q);
    }
    return acc;
}

// Miller-Rabin with the witnesses {2, 3, ..., 37}: exact for all n < 2^64.
bool is_prime_u64(uint64_t n)
{
    if (n < 2) return false;
    const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t p : small) {
        if (n % p == 0) return n == p;
    }
    int r = __builtin_ctzll(n - 1);
    uint64_t d = (n - 1) >> r;
    for (uint64_t a : small) {
        uint64_t x = powmod_u64(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int i = 1; i < r && witness; ++i) {
            x = mulmod_u64(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

// Smallest x with x^N = -1 (mod q), i.e. the smallest primitive 2N-th root of
// unity: one root w is c^((q-1)/2N) for the first c that works, and the full
// set of primitive roots is {w^k : k odd}.
uint64_t min_primitive_2n_root(uint64_t q, uint32_t N)
{
    const uint64_t m = 2ull * N;
    if ((q - 1) % m) return 0;
    uint64_t w = 0;
    for (uint64_t c = 2; c < q && c < (1u << 20); ++c) {
        const uint64_t cand = powmod_u64(c, (q - 1) / m, q);
        if (powmod_u64(cand, N, q) == q - 1) {
            w = cand;
            break;
        }
    }
    if (!w) return 0;
    const uint64_t w2 = mulmod_u64(w, w, q);
    uint64_t best = w, cur = w;
    for (uint32_t i = 1; i < N; ++i) {
        cur = mulmod_u64(cur, w2, q);
        if (cur < best) best = cur;
    }
    return best;
}

uint64_t shoup_companion(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

void delta_residues(const uint64_t *moduli, uint32_t L, uint64_t t, uint64_t *out)
{
    // Q = prod q_i as little-endian 64-bit words (L <= 8 limbs of < 50 bits: < 7 words)
    uint64_t Q[9] = {1, 0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t i = 0; i < L; ++i) {
        u128 carry = 0;
        for (int w = 0; w < 9; ++w) {
            const u128 v = (u128)Q[w] * moduli[i] + carry;
            Q[w] = (uint64_t)v;
            carry = v >> 64;
        }
    }
    // D = floor(Q / t) by short division from the top word
    uint64_t D[9];
    u128 rem = 0;
    for (int w = 8; w >= 0; --w) {
        const u128 cur = (rem << 64) | Q[w];
        D[w] = (uint64_t)(cur / t);
        rem = cur % t;
    }
    // D mod q_i by Horner over the words
    for (uint32_t i = 0; i < L; ++i) {
        u128 r = 0;
        for (int w = 8; w >= 0; --w) r = ((r << 64) | D[w]) % moduli[i];
        out[i] = (uint64_t)r;
    }
}

uint32_t bit_reverse(uint32_t k, uint32_t logn)
{
    uint32_t r = 0;
    for (uint32_t i = 0; i < logn; ++i, k >>= 1) r = (r << 1) | (k & 1u);
    return r;
}

}  // namespace hc
