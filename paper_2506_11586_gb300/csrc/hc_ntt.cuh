// hc_ntt.cuh -- register-resident negacyclic NTT engine for one CTA.
//
// A CTA transforms NP polynomials of N = 2^LOGN residues (NP = 2: both
// components of one ciphertext limb, sharing every twiddle load) with
// T = N / C threads; each thread holds C = 2^LOGC residues of every
// polynomial in registers.  The log2 N butterfly stages run in rounds of
// LOGC stages entirely inside registers; between rounds the CTA exchanges
// data through shared memory (one write, one read per element).
//
// Forward (App. C.1, natural order in, slot order out): Cooley-Tukey stages
// with the psi powers merged into the twiddles (Longa & Naehrig 2016); stage
// s has 2^s groups of 2t = N / 2^s elements, group i uses psi^rev(2^s + i).
// Inverse: Gentleman-Sande stages, stage s (half distance 2^s) has
// N / 2^(s+1) groups, group i uses psi^-rev(N/2^(s+1) + i); N^-1 is merged
// into the last stage.
//
// Lazy bounds (q < 2^50, N <= 2^14; shoup_lazy returns values < 4q):
//   forward: inputs < q; each stage adds 4q -> outputs < (4 log2 N + 1) q < 2^56
//   inverse: inputs < q; stage 0 corrects its products to < 2q, so stage-s
//            inputs are < 2^s q and X - Y + 2^s q < 2^(s+1) q <= 2^64; the last
//            stage's Shoup steps (N^-1 merged) and two corrections give
//            canonical output.
// Twiddle loads: in the inverse's first round and the forward's last round
// every thread needs its own twiddles (N/2 distinct ones in the inverse's
// first stage); read from the natural tables a warp's 32 loads would hit 32
// lines, so those rounds read context tables rearranged so that a warp's
// loads are consecutive (LimbConst::tw_r); the other rounds share each
// twiddle among neighbouring threads and read the natural tables.
// Shared-memory layout: element e of polynomial p lives at word
// p * N + (e ^ ((e >> LOGC) & 15)); the XOR swizzle makes every 8-byte
// access pattern below conflict-free (the 16 threads of each half-warp touch
// 16 distinct bank pairs) without padding.
#pragma once

#include <type_traits>

#include "hc_arith.cuh"
#include "hc_internal.h"

namespace hc {

template <int LOGN_, int LOGC_, int NP_, int MINB_ = 1>
struct NttCfg {
    static constexpr int LOGN = LOGN_;
    static constexpr int LOGC = LOGC_;
    static constexpr int NP = NP_;
    static constexpr int MINB = MINB_;  // CTAs per SM the register budget is sized for
    static constexpr int N = 1 << LOGN;
    static constexpr int C = 1 << LOGC;
    static constexpr int T = N / C;
    static constexpr int NROUNDS = (LOGN + LOGC - 1) / LOGC;
    static constexpr int SW = N;  // shared words per polynomial
    static constexpr size_t SMEM_BYTES = (size_t)NP * SW * sizeof(uint64_t);
    static_assert(LOGC >= 2 && LOGC <= LOGN, "bad radix");
};

template <class Cfg>
__device__ __forceinline__ int spos(int e)
{
    return e ^ ((e >> Cfg::LOGC) & 15);
}

template <class Cfg, int R>
struct RoundShape {
    static constexpr int S0 = R * Cfg::LOGC;
    static constexpr int K = (Cfg::LOGN - S0) < Cfg::LOGC ? (Cfg::LOGN - S0) : Cfg::LOGC;
    static constexpr int KK = 1 << K;
    static constexpr int SUBS = Cfg::C >> K;  // sub-transforms per thread
};

// ---- element owned by (thread, register slot r) in each round ----------------
// forward round: sub-transform u = tid*SUBS + v covers, at stride S = N >> (S0+K),
// the KK elements (u / S) * (N >> S0) + (u % S) + j*S.
template <class Cfg, int R>
__device__ __forceinline__ int fwd_elem(int tid, int r)
{
    using RS = RoundShape<Cfg, R>;
    constexpr int S = Cfg::N >> (RS::S0 + RS::K);
    const int v = r >> RS::K, j = r & (RS::KK - 1);
    const int u = tid * RS::SUBS + v;
    return (u / S) * (Cfg::N >> RS::S0) + (u % S) + j * S;
}

// inverse round: sub-transform u = tid + v*T covers, at stride S = 2^S0, the KK
// elements (u / S) * (S << K) + (u % S) + j*S.
template <class Cfg, int R>
__device__ __forceinline__ int inv_elem(int tid, int r)
{
    using RS = RoundShape<Cfg, R>;
    constexpr int S = 1 << RS::S0;
    const int v = r >> RS::K, j = r & (RS::KK - 1);
    const int u = tid + v * Cfg::T;
    return (u / S) * (S << RS::K) + (u % S) + j * S;
}

// ---- compile-time loop -------------------------------------------------------------
template <int I, int END, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (I < END) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, END>(f);
    }
}

// ---- one forward round: K Cooley-Tukey stages in registers ---------------------
// HALF: the transform is one half of a transform of twice the size, after that
// transform's first stage (see k_ntt_fwd_pair): local stage s, group i uses the
// full table's entry tmul*2^s + i, tmul = 2 + the half's index; every round
// reads the natural table.
template <class Cfg, int R, int SIG, bool HALF = false>
__device__ __forceinline__ void fwd_stage(uint64_t (&x)[Cfg::NP][Cfg::C], const ulonglong2 *__restrict__ tw,
                                          const ulonglong2 *__restrict__ twr, uint64_t q, int v, int g0, int tid,
                                          int tmul = 1)
{
    using RS = RoundShape<Cfg, R>;
    static_assert(Cfg::LOGC >= 3 && Cfg::LOGC <= 5, "last-round tables exist for LOGC = 3, 4, 5");
    constexpr int half = RS::KK >> (SIG + 1);
    constexpr bool last = R == Cfg::NROUNDS - 1 && !HALF;  // every thread has its own twiddles (g0 = tid*SUBS + v)
    const uint64_t nq = 0ull - q, q4 = 4 * q;
#pragma unroll
    for (int lam = 0; lam < (1 << SIG); ++lam) {
        // last round: the rearranged table, stage S0 + SIG at [2^(S0+SIG) - 2^S0],
        // entry ((v << SIG) + lam)*T + tid, so that a warp reads consecutive entries
        const ulonglong2 w =
            last ? __ldg(twr + (size_t)(3 + Cfg::LOGC - 3) * Cfg::N + ((1 << (RS::S0 + SIG)) - (1 << RS::S0)) +
                         ((v << SIG) + lam) * Cfg::T + tid)
                 : __ldg(tw + ((HALF ? tmul : 1) << (RS::S0 + SIG)) + (g0 << SIG) + lam);
#pragma unroll
        for (int jj = 0; jj < half; ++jj) {
            const int j = v * RS::KK + lam * 2 * half + jj;
#pragma unroll
            for (int p = 0; p < Cfg::NP; ++p) {
                const uint64_t X = x[p][j];
                const uint64_t t = shoup_lazy(x[p][j + half], w.x, w.y, nq);  // < 4q
                x[p][j] = X + t;
                x[p][j + half] = X - t + q4;
            }
        }
    }
}

template <class Cfg, int R, bool HALF = false>
__device__ __forceinline__ void fwd_round(uint64_t (&x)[Cfg::NP][Cfg::C], const ulonglong2 *__restrict__ tw,
                                          const ulonglong2 *__restrict__ twr, uint64_t q, int tid, int tmul = 1)
{
    using RS = RoundShape<Cfg, R>;
    constexpr int S = Cfg::N >> (RS::S0 + RS::K);
    static_for<0, RS::SUBS>([&](auto vc) {
        constexpr int v = decltype(vc)::value;
        const int g0 = (tid * RS::SUBS + v) / S;
        static_for<0, RS::K>([&](auto sc) {
            fwd_stage<Cfg, R, decltype(sc)::value, HALF>(x, tw, twr, q, v, g0, tid, tmul);
        });
    });
}

// ---- one inverse round: K Gentleman-Sande stages in registers ------------------
// HALF: the transform is one half of a transform of twice the size, before that
// transform's last stage (see k_ntt_inv_pair): stage s, group i uses the full
// table's entry tmul*(N >> (s+1)) + i (N this transform's size, tmul = 2 + the
// half's index); every round reads the natural table and no stage is the last.
template <class Cfg, int R, int SIG, bool HALF = false>
__device__ __forceinline__ void inv_stage(uint64_t (&x)[Cfg::NP][Cfg::C], const LimbConst &lc,
                                          const ulonglong2 *__restrict__ tw, int v, int blk, int tmul = 1)
{
    using RS = RoundShape<Cfg, R>;
    static_assert(Cfg::LOGC >= 3 && Cfg::LOGC <= 5, "first-round tables exist for LOGC = 3, 4, 5");
    constexpr int s = RS::S0 + SIG;  // global stage
    constexpr int dist = 1 << SIG;
    constexpr int ngrp = RS::KK >> (SIG + 1);
    const uint64_t q = lc.q, nq = 0ull - q;
    const uint64_t qs = q << s;       // bound of the stage's inputs
    if constexpr (s == Cfg::LOGN - 1 && !HALF) {
        // last stage: N^-1 merged into both outputs, canonical result
#pragma unroll
        for (int grp = 0; grp < ngrp; ++grp) {
#pragma unroll
            for (int jj = 0; jj < dist; ++jj) {
                const int j = v * RS::KK + grp * 2 * dist + jj;
#pragma unroll
                for (int p = 0; p < Cfg::NP; ++p) {
                    const uint64_t X = x[p][j], Y = x[p][j + dist];
                    x[p][j] = canon4(shoup_lazy(X + Y, lc.ninv, lc.ninv_s, nq), q);
                    x[p][j + dist] = canon4(shoup_lazy(X - Y + qs, lc.ninvw, lc.ninvw_s, nq), q);
                }
            }
        }
    } else {
#pragma unroll
        for (int grp = 0; grp < ngrp; ++grp) {
            // first round: blk is the thread index, and the rearranged table gives the
            // warp consecutive entries; later rounds share each twiddle across threads
            const ulonglong2 w =
                R == 0 && !HALF
                    ? __ldg(lc.tw_r + (size_t)(Cfg::LOGC - 3) * Cfg::N + (Cfg::N - (Cfg::N >> s)) + grp * Cfg::T + blk)
                    : __ldg(tw + (HALF ? tmul : 1) * (Cfg::N >> (s + 1)) + blk * ngrp + grp);
#pragma unroll
            for (int jj = 0; jj < dist; ++jj) {
                const int j = v * RS::KK + grp * 2 * dist + jj;
#pragma unroll
                for (int p = 0; p < Cfg::NP; ++p) {
                    const uint64_t X = x[p][j], Y = x[p][j + dist];
                    x[p][j] = X + Y;
                    const uint64_t t = shoup_lazy(X - Y + qs, w.x, w.y, nq);  // < 4q
                    x[p][j + dist] = (s == 0) ? csub(t, 2 * q) : t;
                }
            }
        }
    }
}

template <class Cfg, int R, bool HALF = false>
__device__ __forceinline__ void inv_round(uint64_t (&x)[Cfg::NP][Cfg::C], const LimbConst &lc,
                                          const ulonglong2 *__restrict__ tw, int tid, int tmul = 1)
{
    using RS = RoundShape<Cfg, R>;
    constexpr int S = 1 << RS::S0;
    static_for<0, RS::SUBS>([&](auto vc) {
        constexpr int v = decltype(vc)::value;
        const int blk = (tid + v * Cfg::T) / S;
        static_for<0, RS::K>([&](auto sc) {
            inv_stage<Cfg, R, decltype(sc)::value, HALF>(x, lc, tw, v, blk, tmul);
        });
    });
}

// ---- warp-local rounds ---------------------------------------------------------------
// A round is warp-local when every thread's elements in it lie in its own warp's
// block of 32*C consecutive elements (warp w: [32wC, 32(w+1)C)).  An exchange
// between two warp-local rounds moves data only within each warp's block, so a
// warp barrier replaces the CTA barrier on both of its sides: the writes go to
// the warp's own block, whose last readers (the previous round's layout) were
// the warp's own threads.  Inverse round R (u = tid when it has one
// sub-transform per thread, stride S = C^R): local iff it has one sub-transform
// per thread and C^R <= 32 -- rounds 0 and 1 for every shape here.  Forward
// round R (stride N >> (RC + K) over blocks of N >> RC): local iff
// log2 N - R log2 C <= 5 + log2 C -- the last two rounds (three for some
// shapes).  Checked for every shape on a CPU model of fwd_elem / inv_elem.
#ifndef HC_WARP_LOCAL_XCHG
#define HC_WARP_LOCAL_XCHG 1
#endif
template <class Cfg, int R>
constexpr bool inv_round_local()
{
    return RoundShape<Cfg, R>::K == Cfg::LOGC && R * Cfg::LOGC <= 5;
}
template <class Cfg, int R>
constexpr bool fwd_round_local()
{
    return Cfg::LOGN - R * Cfg::LOGC <= 5 + Cfg::LOGC;
}
template <bool WARP>
__device__ __forceinline__ void xsync()
{
    if constexpr (WARP && HC_WARP_LOCAL_XCHG)
        __syncwarp();
    else
        __syncthreads();
}

// ---- exchanges through shared memory ---------------------------------------------
template <class Cfg, int RFROM>
__device__ __forceinline__ void fwd_exchange(uint64_t (&x)[Cfg::NP][Cfg::C], uint64_t *sm, int tid)
{
    constexpr bool local = fwd_round_local<Cfg, RFROM>() && fwd_round_local<Cfg, RFROM + 1>();
    xsync<local>();
#pragma unroll
    for (int r = 0; r < Cfg::C; ++r) {
        const int e = spos<Cfg>(fwd_elem<Cfg, RFROM>(tid, r));
#pragma unroll
        for (int p = 0; p < Cfg::NP; ++p) sm[p * Cfg::SW + e] = x[p][r];
    }
    xsync<local>();
#pragma unroll
    for (int r = 0; r < Cfg::C; ++r) {
        const int e = spos<Cfg>(fwd_elem<Cfg, RFROM + 1>(tid, r));
#pragma unroll
        for (int p = 0; p < Cfg::NP; ++p) x[p][r] = sm[p * Cfg::SW + e];
    }
}

template <class Cfg, int RFROM>
__device__ __forceinline__ void inv_exchange(uint64_t (&x)[Cfg::NP][Cfg::C], uint64_t *sm, int tid)
{
    constexpr bool local = inv_round_local<Cfg, RFROM>() && inv_round_local<Cfg, RFROM + 1>();
    xsync<local>();
#pragma unroll
    for (int r = 0; r < Cfg::C; ++r) {
        const int e = spos<Cfg>(inv_elem<Cfg, RFROM>(tid, r));
#pragma unroll
        for (int p = 0; p < Cfg::NP; ++p) sm[p * Cfg::SW + e] = x[p][r];
    }
    xsync<local>();
#pragma unroll
    for (int r = 0; r < Cfg::C; ++r) {
        const int e = spos<Cfg>(inv_elem<Cfg, RFROM + 1>(tid, r));
#pragma unroll
        for (int p = 0; p < Cfg::NP; ++p) x[p][r] = sm[p * Cfg::SW + e];
    }
}

// ---- whole transforms -----------------------------------------------------------
// forward: x holds the round-0 layout (element tid + r*T) on entry and the
// last-round layout (element tid*C + r, contiguous) on exit.
template <class Cfg, int R = 0, bool HALF = false>
__device__ __forceinline__ void fwd_transform(uint64_t (&x)[Cfg::NP][Cfg::C], uint64_t *sm,
                                              const ulonglong2 *__restrict__ tw, const ulonglong2 *__restrict__ twr,
                                              uint64_t q, int tid, int tmul = 1)
{
    fwd_round<Cfg, R, HALF>(x, tw, twr, q, tid, tmul);
    if constexpr (R + 1 < Cfg::NROUNDS) {
        fwd_exchange<Cfg, R>(x, sm, tid);
        fwd_transform<Cfg, R + 1, HALF>(x, sm, tw, twr, q, tid, tmul);
    }
}

struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// inverse: x holds element tid*C + r (contiguous) on entry, canonical values
// < q; on exit the last-round layout (element tid + r'*T for the slot order of
// inv_elem), canonical.  The first exchange synchronises the warp only: since
// the caller's last CTA barrier, no thread may have accessed shared memory
// outside its own warp's block of 32*C elements (every caller's last accesses
// are its reads of the round-0 layout, element tid*C + r).  hook() runs (in every thread) right before the last
// round, once this transform has finished with shared memory: after its last
// exchange, or after the caller's reads when there is one round only.
template <class Cfg, int R = 0, class Hook = NoHook, bool HALF = false>
__device__ __forceinline__ void inv_transform(uint64_t (&x)[Cfg::NP][Cfg::C], uint64_t *sm,
                                              const LimbConst &lc, const ulonglong2 *__restrict__ tw,
                                              int tid, const Hook &hook = Hook{}, int tmul = 1)
{
    if constexpr (R + 1 == Cfg::NROUNDS) hook();
    inv_round<Cfg, R, HALF>(x, lc, tw, tid, tmul);
    if constexpr (R + 1 < Cfg::NROUNDS) {
        inv_exchange<Cfg, R>(x, sm, tid);
        inv_transform<Cfg, R + 1, Hook, HALF>(x, sm, lc, tw, tid, hook, tmul);
    }
}

}  // namespace hc
