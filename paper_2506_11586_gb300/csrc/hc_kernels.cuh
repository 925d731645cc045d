// hc_kernels.cuh -- sm_103a kernels of the HE-convolution hot path, their
// launch shapes and launchers.  Instantiated once per ring degree in
// hc_kernels_n12.cu / _n13.cu / _n14.cu (compiled in parallel).
//
//   k_ntt_fwd   forward NTT of NP polynomials per CTA (in place or out of place)
//   k_ntt_inv   inverse NTT, NP polynomials per CTA
//   k_mac_intt  NTT-domain multiply-accumulate of a term list, then inverse NTT:
//               out[o] = INTT(sum_t ct_ntt[ct_t] . pt_ntt[pt_t])         (Sec. 6.2)
//   k_product   one standalone ct x pt product fused end to end:
//               out[j] (+)= INTT(NTT(ct[j]) . pt_ntt[j])                  (App. C.1)
//
// All kernels are plain integer code (no tensor cores: this is exact modular
// arithmetic, not a floating-point contraction).  One CTA owns NP whole
// polynomial limbs, so every transform reads and writes HBM exactly once.
#pragma once

#include <atomic>

#include "hc_async.cuh"
#include "hc_ntt.cuh"

namespace hc {

// ---------------------------------------------------------------------------
// Launch-shape variants per ring degree: (log2 C, NP, CTAs per SM).  C residues
// of each of NP polynomials per thread, T = N / C threads per CTA, registers
// sized for MINB resident CTAs.  Single-polynomial kernels (KK_FWD, KK_INV)
// use NP = 1 with the same C and MINB.
template <int LOGN, int V> struct Variant;
template <> struct Variant<12, 0> { static constexpr int LOGC = 3, NP = 2, MINB = 1; };   // T 512, 128 regs
template <> struct Variant<12, 1> { static constexpr int LOGC = 4, NP = 2, MINB = 2; };   // T 256, 128 regs
template <> struct Variant<12, 2> { static constexpr int LOGC = 3, NP = 1, MINB = 2; };   // T 512, 64 regs
template <> struct Variant<13, 0> { static constexpr int LOGC = 4, NP = 2, MINB = 1; };   // T 512, 128 regs
template <> struct Variant<13, 1> { static constexpr int LOGC = 5, NP = 1, MINB = 2; };   // T 256, 128 regs
template <> struct Variant<13, 2> { static constexpr int LOGC = 3, NP = 1, MINB = 1; };   // T 1024, 64 regs
template <> struct Variant<14, 0> { static constexpr int LOGC = 5, NP = 1, MINB = 1; };   // T 512, 128 regs
template <> struct Variant<14, 1> { static constexpr int LOGC = 4, NP = 1, MINB = 1; };   // T 1024, 64 regs
template <> struct Variant<14, 2> { static constexpr int LOGC = 5, NP = 1, MINB = 1; };   // (same as 0)

// shapes of the persistent inverse NTTs (inverse kinds, variant 2): TMA-fed
// double buffer at N = 4096, prefetching into the exchange buffer above
template <int LOGN> struct InvTma;
template <> struct InvTma<12> { using Cfg = NttCfg<12, 4, 1, 2>; };  // T 256, 2 x 32 KB
template <int LOGN> struct InvPf;
template <> struct InvPf<13> { using Cfg = NttCfg<13, 5, 1, 2>; };   // T 256, 64 KB, two CTAs per SM
template <> struct InvPf<14> { using Cfg = NttCfg<14, 5, 1, 1>; };   // T 512, 128 KB
template <int LOGN, int V>
constexpr bool use_inv_tma = V == 2 && LOGN == 12;
template <int LOGN, int V>
constexpr bool use_inv_pf = V == 2 && LOGN >= 13;
// the forward kinds' variant 2 at N >= 8192: one limb per cluster of two CTAs,
// each running a half transform of this shape
template <int LOGN> struct FwdPair;
template <> struct FwdPair<13> { using Cfg = NttCfg<12, 4, 1, 3>; };  // T 256, 32 KB, three clusters' CTAs per SM
template <> struct FwdPair<14> { using Cfg = NttCfg<13, 5, 1, 2>; };  // T 256, 64 KB
template <int LOGN, int V>
constexpr bool use_fwd_pair = V == 2 && LOGN >= 13;


template <int LOGN, int V, bool SINGLE>
using VCfg = NttCfg<LOGN, Variant<LOGN, V>::LOGC, SINGLE ? 1 : Variant<LOGN, V>::NP, Variant<LOGN, V>::MINB>;

// segment of a multi-segment launch that owns this CTA (segments in CTA order)
template <int NS>
__device__ __forceinline__ const NttSeg &find_seg(const NttSegsT<NS> &segs)
{
    uint32_t i = 0;
    while (i + 1 < segs.n && blockIdx.x >= segs.s[i + 1].cta_begin) ++i;
    return segs.s[i];
}

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

// after the block has filled shared memory: x[p][r] = element tid*C + r
// (the inverse transform's round-0 layout)
template <class Cfg>
__device__ __forceinline__ void load_round0(uint64_t (&x)[Cfg::NP][Cfg::C], const uint64_t *sm, int tid)
{
    __syncthreads();
#pragma unroll
    for (int r = 0; r < Cfg::C; ++r)
#pragma unroll
        for (int p = 0; p < Cfg::NP; ++p) x[p][r] = sm[p * Cfg::N + spos<Cfg>(tid * Cfg::C + r)];
}

// ---------------------------------------------------------------------------
// Forward NTT of NP polynomials (src + p*pstride, p < NP) into dst (same
// strides), canonical output, stored through shared memory as coalesced
// 16-byte pairs.  One CTA task.
template <class Cfg>
__device__ __forceinline__ void fwd_task(uint64_t *sm, const uint64_t *src, uint64_t *dst, size_t pstride,
                                         const LimbConst &lc, int tid)
{
    constexpr int NP = Cfg::NP, C = Cfg::C, T = Cfg::T, N = Cfg::N;
    const uint64_t q = lc.q;
    uint64_t x[NP][C];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
        for (int r = 0; r < C; ++r) x[p][r] = __ldg(src + p * pstride + tid + r * T);
    }
    fwd_transform<Cfg>(x, sm, lc.tw_f, lc.tw_r, q, tid);

    const uint32_t ones = (uint32_t)lc.one_s;
    const uint64_t nq = 0ull - q;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < C; ++r) {
#pragma unroll
        for (int p = 0; p < NP; ++p) sm[p * N + spos<Cfg>(tid * C + r)] = canon3(reduce_lazy(x[p][r], ones, nq), q);
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        ulonglong2 *d = reinterpret_cast<ulonglong2 *>(dst + p * pstride);
#pragma unroll
        for (int r = 0; r < C / 2; ++r) {
            const int e = 2 * (tid + r * T);
            ulonglong2 v;
            v.x = sm[p * N + spos<Cfg>(e)];
            v.y = sm[p * N + spos<Cfg>(e + 1)];
            d[tid + r * T] = v;
        }
    }
}

// Inverse NTT of NP polynomials (src + p*pstride) into dst (may equal src).
// COHERENT loads bypass the non-coherent read-only path, for inputs written
// earlier by other CTAs of the same launch.  One CTA task.
template <class Cfg, bool COHERENT = false>
__device__ __forceinline__ void inv_core(uint64_t (&x)[Cfg::NP][Cfg::C], uint64_t *sm, const uint64_t *src,
                                         size_t pstride, const LimbConst &lc, int tid)
{
    constexpr int NP = Cfg::NP, C = Cfg::C, N = Cfg::N;
    // coalesced 16-byte loads into shared memory, then the round-0 layout
    // (element tid*C + r) out of it
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(src + p * pstride);
#pragma unroll
        for (int r = 0; r < C / 2; ++r) {
            const int e = 2 * (tid + r * Cfg::T);
            const ulonglong2 v = COHERENT ? __ldcg(s2 + tid + r * Cfg::T) : __ldg(s2 + tid + r * Cfg::T);
            sm[p * N + spos<Cfg>(e)] = v.x;
            sm[p * N + spos<Cfg>(e + 1)] = v.y;
        }
    }
    load_round0<Cfg>(x, sm, tid);
    inv_transform<Cfg>(x, sm, lc, lc.tw_i, tid);
}

template <class Cfg, bool COHERENT = false>
__device__ __forceinline__ void inv_task(uint64_t *sm, const uint64_t *src, uint64_t *dst, size_t pstride,
                                         const LimbConst &lc, int tid)
{
    constexpr int NP = Cfg::NP, C = Cfg::C;
    uint64_t x[NP][C];
    inv_core<Cfg, COHERENT>(x, sm, src, pstride, lc, tid);
    // the transform's results are read by no later kernel of the layer: streaming
    // stores (evict first), so that L2 keeps what the next kernels read
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        unsigned long long *d = reinterpret_cast<unsigned long long *>(dst + p * pstride);
#pragma unroll
        for (int r = 0; r < C; ++r) __stcs(d + inv_out_elem<Cfg>(tid, r), (unsigned long long)x[p][r]);
    }
}

template <class Cfg, int NS>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_ntt_fwd(const __grid_constant__ NttSegsT<NS> segs)
{
    extern __shared__ uint64_t sm[];
    const NttSeg &sg = find_seg(segs);
    const uint32_t local = blockIdx.x - sg.cta_begin;
    const uint32_t limb = sg.limb0 + local / sg.n_groups, grp = local % sg.n_groups;
    const size_t off = ((size_t)grp * Cfg::NP * sg.L + limb) * Cfg::N;
    fwd_task<Cfg>(sm, sg.in + off, sg.out + off, (size_t)sg.L * Cfg::N, sg.limbs[limb], threadIdx.x);
}

template <class Cfg, int NS>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_ntt_inv(const __grid_constant__ NttSegsT<NS> segs)
{
    extern __shared__ uint64_t sm[];
    const NttSeg &sg = find_seg(segs);
    const uint32_t local = blockIdx.x - sg.cta_begin;
    const uint32_t limb = sg.limb0 + local / sg.n_groups, grp = local % sg.n_groups;
    const size_t off = ((size_t)grp * Cfg::NP * sg.L + limb) * Cfg::N;
    inv_task<Cfg>(sm, sg.in + off, sg.out + off, (size_t)sg.L * Cfg::N, sg.limbs[limb], threadIdx.x);
}

// Inverse NTT of a layer's outputs with the server step's epilogue (Sec. 7, Sec.
// 6.2: only the output coefficients of c0 go back, masked): one CTA per output
// polynomial (limb-major).  c1 is stored in full; c0 goes through shared memory
// and only its S output slots are written, each minus Delta * mask.
template <class Cfg>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_ntt_inv_extract(const __grid_constant__ ExtractArgs ex, const LimbConst *__restrict__ limbs, uint32_t L)
{
    static_assert(Cfg::NP == 1, "one polynomial per CTA");
    extern __shared__ uint64_t sm[];
    const int tid = threadIdx.x;
    const uint32_t per_limb = ex.O * 2;
    const uint32_t limb = ex.limb0 + blockIdx.x / per_limb, pi = blockIdx.x % per_limb;
    const uint32_t o = pi >> 1, comp = pi & 1;
    const LimbConst &lc = limbs[limb];
    uint64_t x[1][Cfg::C];
    inv_core<Cfg>(x, sm, ex.y + ((size_t)pi * L + limb) * Cfg::N, 0, lc, tid);
    if (comp) {
        uint64_t *d = ex.c1 + ((size_t)o * L + limb) * Cfg::N;
#pragma unroll
        for (int r = 0; r < Cfg::C; ++r) d[inv_out_elem<Cfg>(tid, r)] = x[0][r];
        return;
    }
    __syncthreads();  // the transform's last reads of shared memory are done
#pragma unroll
    for (int r = 0; r < Cfg::C; ++r) sm[spos<Cfg>(inv_out_elem<Cfg>(tid, r))] = x[0][r];
    __syncthreads();
    const uint32_t mp = o / ex.B, b = o % ex.B;
    const uint32_t row0 = (b / ex.Bw) * ex.oh, col0 = (b % ex.Bw) * ex.ow;
    const uint64_t q = lc.q;
    uint64_t *out = ex.slots + ((size_t)o * L + limb) * ex.S;
    for (uint32_t s = tid; s < ex.S; s += Cfg::T) {
        const SlotEntry e = ex.table[s];
        const uint32_t m = mp * ex.No + e.n, row = row0 + e.i, col = col0 + e.j;
        uint64_t v = 0;
        if (m < ex.M && row < ex.Ho && col < ex.Wo) {
            v = sm[spos<Cfg>(e.k)];
            if (ex.mask) {
                const uint64_t r = ex.mask[((size_t)m * ex.Ho + row) * ex.Wo + col];
                const uint64_t dr = canon4(shoup_lazy(r, lc.delta, lc.delta_s, 0ull - q), q);
                v = v >= dr ? v - dr : v + q - dr;
            }
        }
        out[s] = v;
    }
}

// ---------------------------------------------------------------------------
// group = one output and NP of its components; limb-major item order so that
// consecutive CTAs (consecutive outputs) share weight polynomials in L2.
template <class Cfg>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
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
    const uint64_t q = lc.q, nq = 0ull - q, r64 = lc.r64, r64_s = lc.r64_s;
    const uint32_t ones = (uint32_t)lc.one_s;
    const uint32_t t0 = __ldg(term_ptr + o), t1 = __ldg(term_ptr + o + 1);

    // MAC in the coalesced pair layout: thread tid owns residue pairs
    // e = 2*(tid + r*T), so each warp-wide 16-byte load covers 512 contiguous
    // bytes.  Sums go to shared memory in canonical form.
    const size_t limb_off = (size_t)limb * N;
#pragma unroll 1
    for (int r = 0; r < C / 2; ++r) {
        const int e = 2 * (tid + r * Cfg::T);
        MacAcc acc[NP][2];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            mac_zero(acc[p][0]);
            mac_zero(acc[p][1]);
        }
#pragma unroll 4
        for (uint32_t t = t0; t < t1; ++t) {
            const uint32_t ci = __ldg(terms + 2 * t), pi = __ldg(terms + 2 * t + 1);
            const ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2 *>(pt_ntt + (size_t)pi * L * N + limb_off + e));
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const ulonglong2 xv = __ldg(reinterpret_cast<const ulonglong2 *>(
                    ct_ntt + ((size_t)ci * 2 + comp0 + p) * L * N + limb_off + e));
                mac_add(acc[p][0], xv.x, w.x);
                mac_add(acc[p][1], xv.y, w.y);
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            sm[p * N + spos<Cfg>(e)] = mac_reduce(acc[p][0], q, nq, r64, r64_s, ones);
            sm[p * N + spos<Cfg>(e + 1)] = mac_reduce(acc[p][1], q, nq, r64, r64_s, ones);
        }
    }
    uint64_t x[NP][C];
    load_round0<Cfg>(x, sm, tid);
    inv_transform<Cfg>(x, sm, lc, lc.tw_i, tid);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        uint64_t *dst = out + (((size_t)o * 2 + comp0 + p) * L + limb) * N;
#pragma unroll
        for (int r = 0; r < C; ++r) dst[inv_out_elem<Cfg>(tid, r)] = x[p][r];
    }
}

// ---------------------------------------------------------------------------
// Persistent, TMA-fed inverse NTT of whole polynomial limbs.  A grid of
// resident CTAs walks the units (one polynomial limb each, limb-major within
// a segment) round robin; while a CTA transforms unit u from one
// shared-memory buffer, the TMA engine already copies its next unit into the
// other (one 1-D bulk copy of N words), so the global-load latency of the
// next unit hides behind the current one's butterflies.  The copied buffer is
// linear; thread tid needs words tid*C .. tid*C + C-1 (the inverse round-0
// layout), which it reads as C/2 16-byte vectors in a per-thread rotated
// order -- conflict-free for every quarter-warp -- and un-rotates in
// registers.  The same buffer then serves the shared-memory exchanges.
// Waits are bounded: a wait that runs out sets err = 2, drains the CTA's
// copies in flight (bounded) and ends the CTA.
template <int V>
__device__ __forceinline__ void unrotate(ulonglong2 (&t)[V], uint32_t rho)
{
    constexpr int LOGV = V == 4 ? 2 : V == 8 ? 3 : V == 16 ? 4 : -1;
    static_assert(LOGV > 0, "4, 8 or 16 vectors per thread");
    static_for<0, LOGV>([&](auto kc) {
        constexpr int S = 1 << decltype(kc)::value;
        const bool c = (rho >> decltype(kc)::value) & 1;
        ulonglong2 u[V];
#pragma unroll
        for (int j = 0; j < V; ++j) u[j] = c ? t[(j - S + V) % V] : t[j];
#pragma unroll
        for (int j = 0; j < V; ++j) t[j] = u[j];
    });
}

template <class Cfg, int NS>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_ntt_inv_tma(const __grid_constant__ NttSegsT<NS> segs, uint32_t total, int *err)
{
    static_assert(Cfg::NP == 1, "one polynomial per unit");
    extern __shared__ __align__(16) uint64_t sm[];  // [2][N]
    __shared__ __align__(8) uint64_t bars[2];
    constexpr int C = Cfg::C, N = Cfg::N, V = C / 2;
    constexpr uint32_t BYTES = N * sizeof(uint64_t);
    const int tid = threadIdx.x;
    const uint32_t G = gridDim.x;

    // unit u -> its segment, limb and polynomial (segment units: limb-major)
    auto locate = [&](uint32_t u, uint32_t &si, uint32_t &limb, uint32_t &poly) {
        si = 0;
        while (si + 1 < segs.n && u >= segs.s[si + 1].cta_begin) ++si;
        const uint32_t local = u - segs.s[si].cta_begin;
        limb = segs.s[si].limb0 + local / segs.s[si].n_groups;
        poly = local % segs.s[si].n_groups;
    };
    auto issue = [&](uint32_t u, int b) {
        uint32_t si, limb, poly;
        locate(u, si, limb, poly);
        const NttSeg &sg = segs.s[si];
        mbar_arrive_expect_tx(&bars[b], BYTES);
        bulk_g2s(sm + (size_t)b * N, sg.in + ((size_t)poly * sg.L + limb) * N, BYTES, &bars[b]);
    };
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0 && blockIdx.x < total) issue(blockIdx.x, 0);

    bool ok = true;
    uint32_t k = 0, u = blockIdx.x;
    for (; u < total; u += G, ++k) {
        const int b = k & 1;
        __syncthreads();  // every thread is done with the other buffer (unit k - 1)
        if (tid == 0 && u + G < total) {
            fence_proxy_async();
            issue(u + G, b ^ 1);
        }
        ok = mbar_wait(&bars[b], (k >> 1) & 1);
        ok = __syncthreads_and(ok);
        if (!ok) break;

        uint32_t si, limb, poly;
        locate(u, si, limb, poly);
        const NttSeg &sg = segs.s[si];
        const LimbConst &lc = sg.limbs[limb];
        uint64_t *buf = sm + (size_t)b * N;
        const uint32_t rho = V >= 8 ? (uint32_t)tid : (uint32_t)tid >> 1;
        const ulonglong2 *vec = reinterpret_cast<const ulonglong2 *>(buf) + (size_t)tid * V;
        ulonglong2 t[V];
#pragma unroll
        for (int r = 0; r < V; ++r) t[r] = vec[(r + rho) & (V - 1)];
        unrotate<V>(t, rho);
        uint64_t x[1][C];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            x[0][2 * j] = t[j].x;
            x[0][2 * j + 1] = t[j].y;
        }
        inv_transform<Cfg>(x, buf, lc, lc.tw_i, tid);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(sg.out + ((size_t)poly * sg.L + limb) * N);
#pragma unroll
        for (int r = 0; r < C; ++r) __stcs(dst + inv_out_elem<Cfg>(tid, r), (unsigned long long)x[0][r]);  // as inv_task
    }
    if (!ok && tid == 0) {
        atomicExch(err, 2);
        // drain: the copy this unit waited for, and the next one if it was issued
        mbar_wait(&bars[k & 1], (k >> 1) & 1);
        if (u + G < total) mbar_wait(&bars[(k + 1) & 1], ((k + 1) >> 1) & 1);
    }
}

// Persistent inverse NTT that prefetches: resident CTAs walk the units
// (polynomial limbs) round robin; a CTA's one shared-memory buffer serves the
// transform's exchanges, and once the last exchange has been read (the
// transform's hook, before its last register round) every thread issues the
// next unit's cp.async copies into it (8-byte words, coalesced in global
// memory, swizzled in shared memory), so that the next load overlaps the last
// round and the stores.
template <class Cfg, int NS>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_ntt_inv_pf(const __grid_constant__ NttSegsT<NS> segs, uint32_t total)
{
    static_assert(Cfg::NP == 1, "one polynomial per unit");
    extern __shared__ __align__(16) uint64_t sm[];  // [N], swizzled
    constexpr int C = Cfg::C, N = Cfg::N, T = Cfg::T;
    const int tid = threadIdx.x;
    const uint32_t G = gridDim.x;

    auto locate = [&](uint32_t u, uint32_t &si, uint32_t &limb, uint32_t &poly) {
        si = 0;
        while (si + 1 < segs.n && u >= segs.s[si + 1].cta_begin) ++si;
        const uint32_t local = u - segs.s[si].cta_begin;
        limb = segs.s[si].limb0 + local / segs.s[si].n_groups;
        poly = local % segs.s[si].n_groups;
    };
    // warp w copies its own block [32wC, 32(w+1)C) of the unit (32 consecutive words
    // per instruction): the round-0 layout (element tid*C + r) and the first
    // exchange stay inside the warp's block, so a warp barrier makes the copies visible
    auto prefetch = [&](uint32_t u) {
        uint32_t si, limb, poly;
        locate(u, si, limb, poly);
        const uint64_t *src = segs.s[si].in + ((size_t)poly * segs.s[si].L + limb) * N;
        const int base = (tid & ~31) * C + (tid & 31);
#pragma unroll
        for (int r = 0; r < C; ++r) {
            const int e = base + 32 * r;
            cp_async8(sm + spos<Cfg>(e), src + e);
        }
        cp_async_commit();
    };
    static_assert(T % 32 == 0, "whole warps");
    uint32_t u = blockIdx.x;
    if (u < total) prefetch(u);
    for (; u < total; u += G) {
        cp_async_wait_all();
        xsync<true>();  // the warp's copies of its block of this unit have landed
        uint32_t si, limb, poly;
        locate(u, si, limb, poly);
        const NttSeg &sg = segs.s[si];
        const LimbConst &lc = sg.limbs[limb];
        uint64_t x[1][C];
#pragma unroll
        for (int r = 0; r < C; ++r) x[0][r] = sm[spos<Cfg>(tid * C + r)];
        const uint32_t next = u + G;
        inv_transform<Cfg>(x, sm, lc, lc.tw_i, tid, [&] {
            __syncthreads();  // the last exchange has been read by every thread
            if (next < total) prefetch(next);
        });
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(sg.out + ((size_t)poly * sg.L + limb) * N);
#pragma unroll
        for (int r = 0; r < C; ++r) __stcs(dst + inv_out_elem<Cfg>(tid, r), (unsigned long long)x[0][r]);  // as inv_task
    }
}

// Forward NTT of one polynomial limb by a cluster of two CTAs (one limb's
// latency split over two SMs).  Stage 0 pairs x[j] with x[j + N/2]; CTA c
// (cluster rank) computes the pairs j in [c N/4, (c+1) N/4) and writes x[j] + w
// x[j + N/2] into CTA 0's shared memory and x[j] - w x[j + N/2] into CTA 1's,
// both at position j (distributed shared memory); after a cluster barrier the
// halves are independent and CTA c runs stages 1 .. log2 N - 1 on half c as a
// transform of N/2 residues (HCfg) with the full table's twiddles
// (fwd_transform's HALF mode), then stores half c canonical, as 16-byte pairs.
// The arithmetic is the one-CTA transform's, stage by stage.
template <class HCfg, int NS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(HCfg::T, HCfg::MINB)
k_ntt_fwd_pair(const __grid_constant__ NttSegsT<NS> segs)
{
    static_assert(HCfg::NP == 1, "one polynomial per cluster");
    extern __shared__ __align__(16) uint64_t sm[];  // [N/2]: the half, then the exchanges
    constexpr int C = HCfg::C, T = HCfg::T, NH = HCfg::N;
    const int tid = threadIdx.x;
    const uint32_t rank = cluster_rank();
    const uint32_t unit = blockIdx.x >> 1;
    uint32_t si = 0;
    while (si + 1 < segs.n && unit >= segs.s[si + 1].cta_begin) ++si;
    const NttSeg &sg = segs.s[si];
    const uint32_t local = unit - sg.cta_begin;
    const uint32_t limb = sg.limb0 + local / sg.n_groups, poly = local % sg.n_groups;
    const size_t off = ((size_t)poly * sg.L + limb) * (2 * (size_t)NH);
    const uint64_t *src = sg.in + off;
    const LimbConst &lc = sg.limbs[limb];
    const uint64_t q = lc.q, nq = 0ull - q, q4 = 4 * q;
    const ulonglong2 w = __ldg(lc.tw_f + 1);
    const uint32_t to0 = cluster_map(sm, 0), to1 = cluster_map(sm, 1);
    cluster_sync();  // both CTAs are running before either writes into the other
#pragma unroll
    for (int r = 0; r < C / 2; ++r) {
        const uint32_t j = rank * (NH / 2) + tid + r * T;  // < NH
        const uint64_t X = __ldg(src + j), Y = __ldg(src + j + NH);
        const uint64_t t = shoup_lazy(Y, w.x, w.y, nq);   // < 4q
        st_cluster_u64(to0 + j * 8, X + t);
        st_cluster_u64(to1 + j * 8, X - t + q4);
    }
    cluster_sync();  // the halves are complete; no remote access after this point
    uint64_t x[1][C];
#pragma unroll
    for (int r = 0; r < C; ++r) x[0][r] = sm[tid + r * T];
    fwd_transform<HCfg, 0, true>(x, sm, lc.tw_f, nullptr, q, tid, 2 + (int)rank);
    const uint32_t ones = (uint32_t)lc.one_s;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < C; ++r) sm[spos<HCfg>(tid * C + r)] = canon3(reduce_lazy(x[0][r], ones, nq), q);
    __syncthreads();
    ulonglong2 *d = reinterpret_cast<ulonglong2 *>(sg.out + off + (size_t)rank * NH);
#pragma unroll
    for (int r = 0; r < C / 2; ++r) {
        const int e = 2 * (tid + r * T);
        ulonglong2 v;
        v.x = sm[spos<HCfg>(e)];
        v.y = sm[spos<HCfg>(e + 1)];
        d[tid + r * T] = v;
    }
}

// Inverse NTT of one polynomial limb by a cluster of two CTAs: CTA c runs
// stages 0 .. log2 N - 2 on half c (positions [c N/2, (c+1) N/2)) as a
// transform of N/2 residues with the full table's twiddles (inv_transform's
// HALF mode) and leaves the half in its shared memory in natural order; after a
// cluster barrier it computes the last stage (pairs j, j + N/2, N^-1 merged)
// for j in [c N/4, (c+1) N/4), reading both halves through distributed shared
// memory, and stores both outputs; a last cluster barrier keeps each CTA's
// shared memory alive until its peer has read it.
template <class HCfg, int NS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(HCfg::T, HCfg::MINB)
k_ntt_inv_pair(const __grid_constant__ NttSegsT<NS> segs)
{
    static_assert(HCfg::NP == 1, "one polynomial per cluster");
    extern __shared__ __align__(16) uint64_t sm[];  // [N/2]
    constexpr int C = HCfg::C, T = HCfg::T, NH = HCfg::N;
    const int tid = threadIdx.x;
    const uint32_t rank = cluster_rank();
    const uint32_t unit = blockIdx.x >> 1;
    uint32_t si = 0;
    while (si + 1 < segs.n && unit >= segs.s[si + 1].cta_begin) ++si;
    const NttSeg &sg = segs.s[si];
    const uint32_t local = unit - sg.cta_begin;
    const uint32_t limb = sg.limb0 + local / sg.n_groups, poly = local % sg.n_groups;
    const size_t off = ((size_t)poly * sg.L + limb) * (2 * (size_t)NH);
    const LimbConst &lc = sg.limbs[limb];
    const uint64_t q = lc.q, nq = 0ull - q;
    // half c: coalesced 16-byte loads into shared memory, then the round-0 layout
    const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(sg.in + off + (size_t)rank * NH);
#pragma unroll
    for (int r = 0; r < C / 2; ++r) {
        const int e = 2 * (tid + r * T);
        const ulonglong2 v = __ldg(s2 + tid + r * T);
        sm[spos<HCfg>(e)] = v.x;
        sm[spos<HCfg>(e + 1)] = v.y;
    }
    uint64_t x[1][C];
    load_round0<HCfg>(x, sm, tid);
    inv_transform<HCfg, 0, NoHook, true>(x, sm, lc, lc.tw_i, tid, NoHook{}, 2 + (int)rank);
    __syncthreads();  // the transform's last exchange has been read
#pragma unroll
    for (int r = 0; r < C; ++r) sm[inv_out_elem<HCfg>(tid, r)] = x[0][r];
    const uint32_t from0 = cluster_map(sm, 0), from1 = cluster_map(sm, 1);
    cluster_sync();  // both halves are in shared memory
    const uint64_t qs = q << (HCfg::LOGN);  // bound of the last stage's inputs (stage log2 N - 1)
    uint64_t *out = sg.out + off;
#pragma unroll
    for (int r = 0; r < C / 2; ++r) {
        const uint32_t j = rank * (NH / 2) + tid + r * T;  // < NH
        const uint64_t X = ld_cluster_u64(from0 + j * 8), Y = ld_cluster_u64(from1 + j * 8);
        out[j] = canon4(shoup_lazy(X + Y, lc.ninv, lc.ninv_s, nq), q);
        out[j + NH] = canon4(shoup_lazy(X - Y + qs, lc.ninvw, lc.ninvw_s, nq), q);
    }
    cluster_sync();  // the peer has read this CTA's half
}

// ---------------------------------------------------------------------------
// One task of a standalone product: NP components (comp0, comp0 + 1, ...) of
// one limb.  ct is the product's ciphertext [2][L][N], pt its NTT-domain
// plaintext [L][N], out its output ciphertext [2][L][N]:
//   out[c][limb] (+)= INTT(NTT(ct[c][limb]) . pt[limb])                  (App. C.1)
template <class Cfg>
__device__ __forceinline__ void product_task(uint64_t *sm, const uint64_t *__restrict__ ct,
                                             const uint64_t *__restrict__ pt, uint64_t *out, const LimbConst &lc,
                                             uint32_t L, uint32_t limb, uint32_t comp0, bool accumulate)
{
    constexpr int NP = Cfg::NP, C = Cfg::C, T = Cfg::T, N = Cfg::N;
    const int tid = threadIdx.x;
    const uint64_t q = lc.q;

    uint64_t x[NP][C];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const uint64_t *src = ct + ((size_t)(comp0 + p) * L + limb) * N;
#pragma unroll
        for (int r = 0; r < C; ++r) x[p][r] = __ldg(src + tid + r * T);
    }
    fwd_transform<Cfg>(x, sm, lc.tw_f, lc.tw_r, q, tid);  // lazy values < 57 q, contiguous layout

    const uint64_t nq = 0ull - q, r64 = lc.r64, r64_s = lc.r64_s;
    const uint32_t ones = (uint32_t)lc.one_s;
    const ulonglong2 *wp = reinterpret_cast<const ulonglong2 *>(pt + (size_t)limb * N + tid * C);
#pragma unroll
    for (int r = 0; r < C / 2; ++r) {
        const ulonglong2 w = __ldg(wp + r);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            MacAcc a0, a1;
            mac_zero(a0);
            mac_zero(a1);
            mac_add(a0, x[p][2 * r], w.x);       // x < 2^56 (lazy forward output)
            mac_add(a1, x[p][2 * r + 1], w.y);
            x[p][2 * r] = mac_reduce(a0, q, nq, r64, r64_s, ones);
            x[p][2 * r + 1] = mac_reduce(a1, q, nq, r64, r64_s, ones);
        }
    }
    inv_transform<Cfg>(x, sm, lc, lc.tw_i, tid);

#pragma unroll
    for (int p = 0; p < NP; ++p) {
        uint64_t *dst = out + ((size_t)(comp0 + p) * L + limb) * N;
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

template <class Cfg>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_product(const uint64_t *__restrict__ ct, const uint64_t *__restrict__ pt_ntt,
          const uint32_t *__restrict__ out_index, uint64_t *out, const LimbConst *__restrict__ limbs,
          uint32_t L, uint32_t n_groups, int accumulate)
{
    extern __shared__ uint64_t sm[];
    constexpr int CPG = 2 / Cfg::NP;
    constexpr size_t N = Cfg::N;
    const uint32_t limb = blockIdx.x / n_groups, grp = blockIdx.x % n_groups;
    const uint32_t j = grp / CPG;
    const uint32_t comp0 = (grp % CPG) * Cfg::NP;
    const uint32_t oj = out_index ? __ldg(out_index + j) : j;
    product_task<Cfg>(sm, ct + (size_t)j * 2 * L * N, pt_ntt + (size_t)j * L * N, out + (size_t)oj * 2 * L * N,
                      limbs[limb], L, limb, comp0, accumulate != 0);
}


// ===========================================================================
// launchers
// ===========================================================================
namespace detail {

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
inline const char *kname_of(int kind, int logn)
{
    static const char *const names[4][3] = {
        {"k_ntt_fwd/N4096", "k_ntt_fwd/N8192", "k_ntt_fwd/N16384"},
        {"k_ntt_inv/N4096", "k_ntt_inv/N8192", "k_ntt_inv/N16384"},
        {"k_mac_intt/N4096", "k_mac_intt/N8192", "k_mac_intt/N16384"},
        {"k_product/N4096", "k_product/N8192", "k_product/N16384"},
    };
    return names[kind][logn - 12];
}

template <class Cfg>
const char *kname(int kind)
{
    return kname_of(kind, Cfg::LOGN);
}

inline hc_status after_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HC_OK : cuda_error(e, what);
}

template <class Cfg, int KIND, int NS>
hc_status run_ntt_segs(const NttSegsT<NS> &segs, cudaStream_t s, bool inverse)
{
    uint32_t items = 0;
    for (uint32_t i = 0; i < segs.n; ++i) items = segs.s[i].cta_begin + segs.s[i].n_groups * seg_limbs(segs.s[i]);
    if (items == 0) return HC_OK;
    if (inverse) {
        auto kern = k_ntt_inv<Cfg, NS>;
        hc_status st = prepare<Cfg, KIND * 1000 + NS>(kern, Cfg::SMEM_BYTES);
        if (st != HC_OK) return st;
        ProfileScope ps(kname<Cfg>(KK_INV), s);
        kern<<<items, Cfg::T, Cfg::SMEM_BYTES, s>>>(segs);
        return after_launch("k_ntt_inv");
    }
    auto kern = k_ntt_fwd<Cfg, NS>;
    hc_status st = prepare<Cfg, KIND * 1000 + NS>(kern, Cfg::SMEM_BYTES);
    if (st != HC_OK) return st;
    ProfileScope ps(kname<Cfg>(KK_FWD), s);
    kern<<<items, Cfg::T, Cfg::SMEM_BYTES, s>>>(segs);
    return after_launch("k_ntt_fwd");
}

// persistent TMA-fed inverse NTT: segs' cta_begin are unit offsets (n_groups
// polynomials x L limbs per segment); one launch of resident CTAs
template <class Cfg, int NS>
hc_status run_ntt_inv_tma(const NttSegsT<NS> &segs, int *err, cudaStream_t s)
{
    uint32_t total = 0;
    for (uint32_t i = 0; i < segs.n; ++i) total = segs.s[i].cta_begin + segs.s[i].n_groups * seg_limbs(segs.s[i]);
    if (total == 0) return HC_OK;
    constexpr size_t smem = 2 * Cfg::SMEM_BYTES;
    auto kern = k_ntt_inv_tma<Cfg, NS>;
    static std::atomic<int> resident[32];
    int dev = 0;
    cudaGetDevice(&dev);
    int r = resident[dev & 31].load();
    if (r == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0, sms = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::T, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_error(e, "k_ntt_inv_tma set-up");
        if (per_sm < 1) return set_error(HC_ERR_UNSUPPORTED, "k_ntt_inv_tma does not fit on an SM");
        r = per_sm * sms;
        resident[dev & 31].store(r);
    }
    const uint32_t grid = total < (uint32_t)r ? total : (uint32_t)r;
    ProfileScope ps(kname<Cfg>(KK_INV), s);
    kern<<<grid, Cfg::T, smem, s>>>(segs, total, err);
    return after_launch("k_ntt_inv_tma");
}

template <class HCfg, int NS>
hc_status run_ntt_inv_pair(const NttSegsT<NS> &segs, cudaStream_t s);

// persistent prefetching inverse NTT: segs' cta_begin are unit offsets
// (n_groups polynomials x L limbs per segment); one launch of resident CTAs.
// With fewer limbs than resident CTAs no CTA would prefetch, and the limbs run
// as two-CTA clusters (k_ntt_inv_pair, halves of shape PCfg) instead: measured
// on GB300, 7-14 % lower latency for a few limbs, 11 % higher time for 1536.
template <class Cfg, class PCfg, int NS>
hc_status run_ntt_inv_pf(const NttSegsT<NS> &segs, cudaStream_t s)
{
    uint32_t total = 0;
    for (uint32_t i = 0; i < segs.n; ++i) total = segs.s[i].cta_begin + segs.s[i].n_groups * seg_limbs(segs.s[i]);
    if (total == 0) return HC_OK;
    constexpr size_t smem = Cfg::SMEM_BYTES;
    auto kern = k_ntt_inv_pf<Cfg, NS>;
    static std::atomic<int> resident[32];
    int dev = 0;
    cudaGetDevice(&dev);
    int r = resident[dev & 31].load();
    if (r == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0, sms = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::T, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_error(e, "k_ntt_inv_pf set-up");
        if (per_sm < 1) return set_error(HC_ERR_UNSUPPORTED, "k_ntt_inv_pf does not fit on an SM");
        r = per_sm * sms;
        resident[dev & 31].store(r);
    }
    if (total < (uint32_t)r) return run_ntt_inv_pair<PCfg>(segs, s);
    const uint32_t grid = total < (uint32_t)r ? total : (uint32_t)r;
    ProfileScope ps(kname<Cfg>(KK_INV), s);
    kern<<<grid, Cfg::T, smem, s>>>(segs, total);
    return after_launch("k_ntt_inv_pf");
}

// forward NTTs by clusters of two CTAs: segs' cta_begin are unit offsets (n_groups
// polynomials x L limbs per segment); two CTAs per unit
template <class HCfg, int NS>
hc_status run_ntt_fwd_pair(const NttSegsT<NS> &segs, cudaStream_t s)
{
    uint32_t total = 0;
    for (uint32_t i = 0; i < segs.n; ++i) total = segs.s[i].cta_begin + segs.s[i].n_groups * seg_limbs(segs.s[i]);
    if (total == 0) return HC_OK;
    if (total > 0x3fffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    auto kern = k_ntt_fwd_pair<HCfg, NS>;
    hc_status st = prepare<HCfg, 7000 + NS>(kern, HCfg::SMEM_BYTES);
    if (st != HC_OK) return st;
    ProfileScope ps(kname_of(KK_FWD, HCfg::LOGN + 1), s);
    kern<<<2 * total, HCfg::T, HCfg::SMEM_BYTES, s>>>(segs);
    return after_launch("k_ntt_fwd_pair");
}

template <class HCfg, int NS>
hc_status run_ntt_inv_pair(const NttSegsT<NS> &segs, cudaStream_t s)
{
    uint32_t total = 0;
    for (uint32_t i = 0; i < segs.n; ++i) total = segs.s[i].cta_begin + segs.s[i].n_groups * seg_limbs(segs.s[i]);
    if (total == 0) return HC_OK;
    if (total > 0x3fffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    auto kern = k_ntt_inv_pair<HCfg, NS>;
    hc_status st = prepare<HCfg, 8000 + NS>(kern, HCfg::SMEM_BYTES);
    if (st != HC_OK) return st;
    ProfileScope ps(kname_of(KK_INV, HCfg::LOGN + 1), s);
    kern<<<2 * total, HCfg::T, HCfg::SMEM_BYTES, s>>>(segs);
    return after_launch("k_ntt_inv_pair");
}

// one-segment launch: n_groups CTAs per limb
inline NttSegs1 one_seg(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_groups)
{
    NttSegs1 segs{};
    segs.n = 1;
    segs.s[0] = NttSeg{in, out, ctx->d_limbs, ctx->L, (uint32_t)n_groups, 0};
    return segs;
}

template <class Cfg>
hc_status run_ntt_fwd(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_groups, cudaStream_t s)
{
    if (n_groups == 0) return HC_OK;
    if (n_groups * ctx->L > 0x7fffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    return run_ntt_segs<Cfg, KK_FWD>(one_seg(ctx, in, out, n_groups), s, false);
}

template <class Cfg>
hc_status run_ntt_inv(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_groups, cudaStream_t s)
{
    if (n_groups == 0) return HC_OK;
    if (n_groups * ctx->L > 0x7fffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    return run_ntt_segs<Cfg, KK_INV>(one_seg(ctx, in, out, n_groups), s, true);
}

template <class Cfg>
hc_status run_mac_intt(const hc_ctx *ctx, const uint64_t *ct_ntt, const uint64_t *pt_ntt, MacTerms terms,
                       uint64_t *out, size_t n_out, cudaStream_t s)
{
    if (n_out == 0) return HC_OK;
    auto kern = k_mac_intt<Cfg>;
    hc_status st = prepare<Cfg, KK_MAC>(kern, Cfg::SMEM_BYTES);
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
hc_status run_inv_extract(const hc_ctx *ctx, const ExtractArgs &ex, cudaStream_t s)
{
    if (ex.O == 0) return HC_OK;
    auto kern = k_ntt_inv_extract<Cfg>;
    hc_status st = prepare<Cfg, KK_INV_EXTRACT>(kern, Cfg::SMEM_BYTES);
    if (st != HC_OK) return st;
    const uint32_t Lc = ex.Lc ? ex.Lc : ctx->L;
    if (ex.limb0 + Lc > ctx->L) return set_error(HC_ERR_INVALID_ARG, "limb range out of bounds");
    const size_t items = (size_t)ex.O * 2 * Lc;
    if (items > 0x7fffffffu) return set_error(HC_ERR_INVALID_ARG, "layer too large");
    ProfileScope ps("k_ntt_inv_extract", s);
    kern<<<(unsigned)items, Cfg::T, Cfg::SMEM_BYTES, s>>>(ex, ctx->d_limbs, ctx->L);
    return after_launch("k_ntt_inv_extract");
}

template <class Cfg>
hc_status run_product(const hc_ctx *ctx, const uint64_t *ct, const uint64_t *pt_ntt, const uint32_t *out_index,
                      uint64_t *out, size_t n, bool accumulate, cudaStream_t s)
{
    if (n == 0) return HC_OK;
    auto kern = k_product<Cfg>;
    hc_status st = prepare<Cfg, KK_PROD>(kern, Cfg::SMEM_BYTES);
    if (st != HC_OK) return st;
    const size_t n_groups = n * (2 / Cfg::NP);
    const size_t items = n_groups * ctx->L;
    if (items > 0x7fffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
    ProfileScope ps(kname<Cfg>(3), s);
    kern<<<(unsigned)items, Cfg::T, Cfg::SMEM_BYTES, s>>>(ct, pt_ntt, out_index, out, ctx->d_limbs, ctx->L,
                                                          (uint32_t)n_groups, accumulate ? 1 : 0);
    return after_launch("k_product");
}

}  // namespace detail

template <int LOGN, int V>
hc_status launch_variant(const hc_ctx *ctx, int kind, const LaunchArgs &a, cudaStream_t s)
{
    using Fused = VCfg<LOGN, V, false>;
    using Single = VCfg<LOGN, V, true>;
    if constexpr (use_inv_tma<LOGN, V> || use_inv_pf<LOGN, V>) {
        auto run = [&](const auto &segs) {
            if constexpr (use_inv_tma<LOGN, V>)
                return detail::run_ntt_inv_tma<typename InvTma<LOGN>::Cfg>(segs, timeout_flag(ctx), s);
            else
                return detail::run_ntt_inv_pf<typename InvPf<LOGN>::Cfg, typename FwdPair<LOGN>::Cfg>(segs, s);
        };
        if (kind == KK_INV || kind == KK_INVCT) {
            const size_t polys = kind == KK_INV ? a.n : 2 * a.n;
            if (polys == 0) return HC_OK;
            if (polys * ctx->L > 0x7fffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
            return run(detail::one_seg(ctx, a.in, a.out, polys));
        }
        if (kind == KK_INVCT_SEGS) {
            NttSegs segs = *a.segs;
            uint32_t begin = 0;
            for (uint32_t i = 0; i < segs.n; ++i) {
                segs.s[i].n_groups *= 2;  // polynomials
                segs.s[i].cta_begin = begin;
                begin += segs.s[i].n_groups * seg_limbs(segs.s[i]);
            }
            return run(segs);
        }
    }
    if constexpr (use_fwd_pair<LOGN, V>) {
        using HC = typename FwdPair<LOGN>::Cfg;
        if (kind == KK_FWD || kind == KK_FWDCT) {
            const size_t polys = kind == KK_FWD ? a.n : 2 * a.n;
            if (polys == 0) return HC_OK;
            if (polys * ctx->L > 0x7fffffffu) return set_error(HC_ERR_INVALID_ARG, "batch too large");
            return detail::run_ntt_fwd_pair<HC>(detail::one_seg(ctx, a.in, a.out, polys), s);
        }
        if (kind == KK_FWDCT_SEGS) {
            NttSegs segs = *a.segs;
            uint32_t begin = 0;
            for (uint32_t i = 0; i < segs.n; ++i) {
                segs.s[i].n_groups *= 2;  // polynomials
                segs.s[i].cta_begin = begin;
                begin += segs.s[i].n_groups * seg_limbs(segs.s[i]);
            }
            return detail::run_ntt_fwd_pair<HC>(segs, s);
        }
    }
    switch (kind) {
    case KK_FWD: return detail::run_ntt_fwd<Single>(ctx, a.in, a.out, a.n, s);
    case KK_INV: return detail::run_ntt_inv<Single>(ctx, a.in, a.out, a.n, s);
    case KK_FWDCT: return detail::run_ntt_fwd<Fused>(ctx, a.in, a.out, a.n * (2 / Fused::NP), s);
    case KK_INVCT: return detail::run_ntt_inv<Fused>(ctx, a.in, a.out, a.n * (2 / Fused::NP), s);
    case KK_FWDCT_SEGS:
    case KK_INVCT_SEGS: {
        // segment n_groups are given in ciphertexts; scale to CTAs of this shape
        NttSegs segs = *a.segs;
        uint32_t begin = 0;
        for (uint32_t i = 0; i < segs.n; ++i) {
            segs.s[i].n_groups *= 2 / Fused::NP;
            segs.s[i].cta_begin = begin;
            begin += segs.s[i].n_groups * seg_limbs(segs.s[i]);
        }
        return kind == KK_FWDCT_SEGS ? detail::run_ntt_segs<Fused, KK_FWDCT>(segs, s, false)
                                     : detail::run_ntt_segs<Fused, KK_INVCT>(segs, s, true);
    }
    case KK_MAC: return detail::run_mac_intt<Fused>(ctx, a.in, a.pt, a.terms, a.out, a.n, s);
    case KK_PROD: return detail::run_product<Fused>(ctx, a.in, a.pt, a.out_index, a.out, a.n, a.accumulate, s);
    case KK_INV_EXTRACT:
        // variant 2 of the inverse kinds is persistent at N >= 8192; the epilogue
        // kernel (one output limb per CTA, shared memory busy until its last store)
        // takes the best one-CTA shape there, variant 1's
        if constexpr (V == 2 && LOGN >= 13)
            return detail::run_inv_extract<VCfg<LOGN, 1, true>>(ctx, *a.ex, s);
        else
            return detail::run_inv_extract<Single>(ctx, *a.ex, s);
    default: return set_error(HC_ERR_INVALID_ARG, "unknown kernel kind %d", kind);
    }
}

template <int LOGN>
hc_status launch_n(const hc_ctx *ctx, int kind, int variant, const LaunchArgs &a, cudaStream_t s)
{
    switch (variant) {
    case 0: return launch_variant<LOGN, 0>(ctx, kind, a, s);
    case 1: return launch_variant<LOGN, 1>(ctx, kind, a, s);
    case 2: return launch_variant<LOGN, 2>(ctx, kind, a, s);
    default: return set_error(HC_ERR_INVALID_ARG, "unknown launch variant %d", variant);
    }
}

}  // namespace hc
