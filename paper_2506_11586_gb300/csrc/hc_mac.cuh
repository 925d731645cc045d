// hc_mac.cuh -- the blocked NTT-domain convolution MAC (Sec. 6.2) as one CTA
// task, shared by the stand-alone MAC kernel and the fused persistent
// convolution kernel:
//   Y[m*B+b][c] = sum_g W[m*G+g] . X[g*B+b][c]      (slot-wise, mod q_limb)
//
// A task owns one chunk of KC slots of one limb for every input ciphertext
// and the output channels [m0, m1).  The input chunk (G*2B rows of KC slots)
// is fetched once into shared memory by TMA bulk copies; the weight slices
// stream through a ring of kMacStages shared-memory stages of MS channels
// each (MS*G rows of KC slots), refilled while the other stages are in use.
// Each weight slot is therefore read from memory once and each input slot
// once per channel group.  Per stage the CTA computes MS*2B output rows of
// KC slots: thread (k, h) owns slot k0 + k and the rows j = h (mod H), row
// j = m*2B + p for channel m of the stage and component pair p = 2b + c.
//
// The ring's mbarriers live for the whole CTA; a MacRing carries their
// phase counters from one task to the next.  Waits are bounded: a wait that
// runs out sets err = 2, drains the task's copies in flight (bounded) and
// makes the task return false.
#pragma once

#include <type_traits>

#include "hc_arith.cuh"
#include "hc_async.cuh"
#include "hc_internal.h"

namespace hc {

constexpr int kMacStages = 3;
constexpr int kMacKC = 64;

struct MacRing {
    uint32_t gi;    // weight stages loaded and consumed so far by this CTA
    uint32_t xuse;  // input chunks loaded so far by this CTA
};

// bars: 1 + kMacStages mbarriers initialised with count 1.  The caller has
// synchronised the CTA since its last generic shared-memory access.
template <int KC, int NT>
__device__ __forceinline__ bool mac_task(const MacSeg &sg, uint32_t chunk, uint32_t limb, uint32_t m0, uint32_t m1,
                                         uint64_t *dsm, uint64_t *bars, MacRing &ring, int *err)
{
    constexpr int H = NT / KC;
    constexpr uint32_t ROW_BYTES = KC * sizeof(uint64_t);
    static_assert(NT % KC == 0 && KC % 32 == 0, "whole warps per row group");
    const uint32_t N = sg.N, L = sg.L, G = sg.G, B = sg.B, MS = sg.MS;
    const uint32_t P = 2 * B, rows = G * P, SR = MS * G;
    uint64_t *xs = dsm;                          // [rows][KC]
    uint64_t *ws = dsm + (size_t)rows * KC;      // [kMacStages][SR][KC]
    const uint32_t k0 = chunk * KC;
    const uint32_t nm = m1 > m0 ? m1 - m0 : 0;
    const uint32_t nst = (nm + MS - 1) / MS;     // stages of this task
    const size_t LN = (size_t)L * N;
    const uint64_t *xsrc = sg.X + (size_t)limb * N + k0;   // input row r at xsrc + r*LN
    const uint64_t *wsrc = sg.W + (size_t)limb * N + k0;   // weight poly j at wsrc + j*LN
    const int tid = threadIdx.x;
    const uint32_t g0 = ring.gi;

    auto issue_w = [&](uint32_t i) {  // channels m0 + i*MS ... into ring slot (g0 + i) % kMacStages
        const uint32_t st = (g0 + i) % kMacStages, c0 = m0 + i * MS;
        const uint32_t nr = min(MS, m1 - c0) * G;
        mbar_arrive_expect_tx(&bars[1 + st], nr * ROW_BYTES);
        const uint64_t *src = wsrc + (size_t)c0 * G * LN;
        uint64_t *dst = ws + (size_t)st * SR * KC;
        const uint64_t pol = l2_evict_first_policy();  // each weight slot is read once per layer
        for (uint32_t r = 0; r < nr; ++r) bulk_g2s_stream(dst + (size_t)r * KC, src + r * LN, ROW_BYTES, &bars[1 + st], pol);
    };
    if (tid == 0) {
        fence_proxy_async();  // earlier generic accesses to this shared memory before the copies
        mbar_arrive_expect_tx(&bars[0], rows * ROW_BYTES);
        for (uint32_t r = 0; r < rows; ++r) bulk_g2s(xs + (size_t)r * KC, xsrc + r * LN, ROW_BYTES, &bars[0]);
        for (uint32_t i = 0; i < (uint32_t)kMacStages && i < nst; ++i) issue_w(i);
    }

    const LimbConst &lc = sg.limbs[limb];
    const uint64_t q = lc.q, nq = 0ull - q, r64 = lc.r64, r64_s = lc.r64_s;
    const uint32_t ones = (uint32_t)lc.one_s;
    // inputs are canonical forward-NTT outputs (< q < 2^50), so with at most 16 terms
    // per row the special-form reduction applies whenever q = 2^50 - c, c small
    const uint32_t sc = (uint32_t)lc.special_c;
    const bool special = sc != 0 && G <= 16;
    const uint32_t k = tid % KC, h = tid / KC;  // h is warp-uniform
    const uint32_t xstep = P * KC;
    bool ok = mbar_wait(&bars[0], ring.xuse & 1);
    uint32_t i = 0;
    for (; i < nst; ++i) {
        const uint32_t st = (g0 + i) % kMacStages;
        ok = mbar_wait(&bars[1 + st], ((g0 + i) / kMacStages) & 1) && ok;
        ok = __syncthreads_and(ok);  // also: every thread has finished stage i - 1
        if (!ok) break;
        if (tid == 0 && i >= 1 && i - 1 + kMacStages < nst) {
            fence_proxy_async();
            issue_w(i - 1 + kMacStages);  // into the slot that stage i - 1 used
        }
        const uint32_t c0 = m0 + i * MS, cnt = min(MS, m1 - c0);
        const uint64_t *wst = ws + (size_t)st * SR * KC + k;
        uint64_t *yk = sg.Y + (size_t)limb * N + k0 + k + (size_t)c0 * P * LN;
        // one output row: sum over the G channel groups (two chains for latency hiding)
        auto row = [&](const uint64_t *xp, const uint64_t *wk, uint64_t *yp) {
            MacAcc acc0, acc1;
            mac_zero(acc0);
            mac_zero(acc1);
            uint32_t g = 0;
            for (; g + 1 < G; g += 2) {
                mac_add(acc0, xp[0], wk[g * KC]);
                mac_add(acc1, xp[xstep], wk[(g + 1) * KC]);
                xp += 2 * xstep;
            }
            if (g < G) mac_add(acc0, xp[0], wk[g * KC]);
            mac_merge(acc0, acc1);
            *yp = special ? mac_reduce_special(acc0, q, sc) : mac_reduce(acc0, q, nq, r64, r64_s, ones);
        };
        // CR channels x RR rows (rows p and p + H) at once: each input slot and each
        // weight slot read from shared memory once per tile instead of once per term
        auto tile = [&](auto cr, auto rr, const uint64_t *xp, const uint64_t *wk, uint64_t *yp, uint32_t cs) {
            constexpr int CR = decltype(cr)::value, RR = decltype(rr)::value;
            MacAcc acc[CR][RR];
#pragma unroll
            for (int c = 0; c < CR; ++c)
#pragma unroll
                for (int r = 0; r < RR; ++r) mac_zero(acc[c][r]);
            for (uint32_t g = 0; g < G; ++g, xp += xstep, wk += KC) {
                uint64_t xv[RR], wv[CR];
#pragma unroll
                for (int r = 0; r < RR; ++r) xv[r] = xp[r * H * KC];
#pragma unroll
                for (int c = 0; c < CR; ++c) wv[c] = wk[(size_t)c * cs * G * KC];
#pragma unroll
                for (int c = 0; c < CR; ++c)
#pragma unroll
                    for (int r = 0; r < RR; ++r) mac_add(acc[c][r], xv[r], wv[c]);
            }
#pragma unroll
            for (int c = 0; c < CR; ++c)
#pragma unroll
                for (int r = 0; r < RR; ++r)
                    yp[(size_t)c * cs * P * LN + (size_t)r * H * LN] =
                        special ? mac_reduce_special(acc[c][r], q, sc) : mac_reduce(acc[c][r], q, nq, r64, r64_s, ones);
        };
        using I1 = std::integral_constant<int, 1>;
        using I2 = std::integral_constant<int, 2>;
        const uint64_t *xk = xs + k;
        if (P >= (uint32_t)H) {  // every row group has work in every channel
            uint32_t ml = 0;
            for (; ml + 1 < cnt; ml += 2) {  // channel pairs
                const uint64_t *wk = wst + (size_t)ml * G * KC;
                uint64_t *ym = yk + (size_t)ml * P * LN;
                uint32_t p = h;
                for (; p + H < P; p += 2 * H) tile(I2{}, I2{}, xk + p * KC, wk, ym + p * LN, 1);
                if (p < P) tile(I2{}, I1{}, xk + p * KC, wk, ym + p * LN, 1);
            }
            if (ml < cnt) {  // the last channel alone
                const uint64_t *wk = wst + (size_t)ml * G * KC;
                uint64_t *ym = yk + (size_t)ml * P * LN;
                uint32_t p = h;
                for (; p + H < P; p += 2 * H) tile(I1{}, I2{}, xk + p * KC, wk, ym + p * LN, 1);
                if (p < P) row(xk + p * KC, wk, ym + p * LN);
            }
        } else if (H % P == 0) {  // few rows per channel: row p = h mod P of channels h/P, h/P + H/P, ...
            const uint32_t p = h % P, cs = H / P;
            uint32_t ml = h / P;
            for (; ml + cs < cnt; ml += 2 * cs)  // channel pairs (ml, ml + cs) share the input loads
                tile(I2{}, I1{}, xk + p * KC, wst + (size_t)ml * G * KC, yk + ((size_t)ml * P + p) * LN, cs);
            if (ml < cnt) row(xk + p * KC, wst + (size_t)ml * G * KC, yk + ((size_t)ml * P + p) * LN);
        } else {                 // few rows per channel: spread (channel, row) pairs over the groups
            const uint32_t jobs = cnt * P;
            uint32_t ml = h / P, p = h % P;
            for (uint32_t j = h; j < jobs; j += H) {
                row(xk + p * KC, wst + (size_t)ml * G * KC, yk + (size_t)j * LN);
                p += H;
                while (p >= P) {
                    p -= P;
                    ++ml;
                }
            }
        }
    }
    ok = __syncthreads_and(ok);  // uniform across the CTA even when the task has no stage
    if (!ok) {
        if (tid == 0) {
            atomicExch(err, 2);
            // drain this task's bulk copies still in flight before the shared memory is reused
            mbar_wait(&bars[0], ring.xuse & 1);
            const uint32_t last = i == 0 ? min(nst, (uint32_t)kMacStages) : min(nst, i - 1 + kMacStages);
            for (uint32_t j = i; j < last; ++j)
                mbar_wait(&bars[1 + (g0 + j) % kMacStages], ((g0 + j) / kMacStages) & 1);
        }
        return false;
    }
    ring.gi = g0 + nst;
    ring.xuse += 1;
    return true;
}

}  // namespace hc
