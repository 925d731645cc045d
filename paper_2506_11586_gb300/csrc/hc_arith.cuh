// hc_arith.cuh -- uint64 modular arithmetic on the integer pipes.
//
// Residues live in 64-bit words with q < 2^50, which leaves 14 bits of head
// room: butterflies run lazily (no conditional subtraction inside the
// transforms) and reductions happen once, at the end.
//
// Shoup multiplication (V. Shoup, NTL; D. Harvey, "Faster arithmetic for
// number-theoretic transforms", JSC 2014): for a constant w < q with
// companion w' = floor(w * 2^64 / q), and ANY y < 2^64,
//     y*w - floor(y*w' / 2^64) * q   lies in [0, 2q)
// and is congruent to y*w mod q.  All arithmetic is mod 2^64.
#pragma once

#include <cstdint>

namespace hc {

__device__ __forceinline__ uint64_t shoup_mul(uint64_t y, uint64_t w, uint64_t wp, uint64_t q)
{
    return y * w - __umul64hi(y, wp) * q;
}

__device__ __forceinline__ uint64_t csub(uint64_t x, uint64_t m)
{
    return x >= m ? x - m : x;
}

// 128-bit accumulator (hi:lo) += a * b
__device__ __forceinline__ void mac128(uint64_t &lo, uint64_t &hi, uint64_t a, uint64_t b)
{
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
        "madc.hi.u64 %1, %2, %3, %1;"
        : "+l"(lo), "+l"(hi)
        : "l"(a), "l"(b));
}

// (hi * 2^64 + lo) mod q, canonical, for any hi, lo < 2^64:
// hi*2^64 = hi * (2^64 mod q), both halves by Shoup into [0, 2q), sum < 4q.
__device__ __forceinline__ uint64_t reduce128(uint64_t lo, uint64_t hi, uint64_t q, uint64_t r64,
                                              uint64_t r64_s, uint64_t one_s)
{
    uint64_t a = shoup_mul(hi, r64, r64_s, q);   // [0, 2q)
    uint64_t b = lo - __umul64hi(lo, one_s) * q;  // lo*1 by Shoup: [0, 2q)
    uint64_t s = a + b;                           // [0, 4q)
    s = csub(s, 2 * q);
    return csub(s, q);
}

// x mod q for x < 2^64 (one Shoup step then one correction)
__device__ __forceinline__ uint64_t reduce64(uint64_t x, uint64_t q, uint64_t one_s)
{
    return csub(x - __umul64hi(x, one_s) * q, q);
}

}  // namespace hc
