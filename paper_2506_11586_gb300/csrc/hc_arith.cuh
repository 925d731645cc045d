// hc_arith.cuh -- uint64 modular arithmetic on the integer pipes, built from
// 32-bit partial products.
//
// Residues live in 64-bit words with q < 2^50, leaving 14 bits of head room:
// butterflies run lazily and reductions happen once, at the end.
//
// Cost model (measured on GB300): a 32x32->64 multiply-add (mad.wide.u32)
// issues at the same rate as a 32-bit multiply-add, while the high half
// alone (mad.hi.u32) costs twice as much, and the compiler's 64-bit mul.lo /
// mul.hi cost about 4 and 8 multiply-adds.  So every product below is formed
// from wide 32-bit multiply-adds, and high halves are taken from the wide
// results instead of being computed separately.
//
// Shoup multiplication (V. Shoup; D. Harvey, "Faster arithmetic for
// number-theoretic transforms", JSC 2014): for a constant w < q with
// companion w' = floor(w * 2^64 / q) and any y < 2^64,
//     y*w - floor(y*w' / 2^64) * q   lies in [0, 2q).
// shoup_lazy drops the lowest partial product y_lo*w'_lo and the carry of
// the two middle ones from the quotient, which makes the quotient at most 2
// too small: the result is congruent to y*w and lies in [0, 4q).
#pragma once

#include <cstdint>

namespace hc {

// y*w mod q, lazily: result in [0, 4q) for any y < 2^64, w < q < 2^62,
// wp = floor(w*2^64/q), nq = 2^64 - q.
__device__ __forceinline__ uint64_t shoup_lazy(uint64_t y, uint64_t w, uint64_t wp, uint64_t nq)
{
    uint64_t r;
    asm("{\n\t"
        ".reg .u32 yl, yh, wl, wh, pl, ph, nl, nh, al, ah, bl, bh, ql, qh, rl, rh, h, c;\n\t"
        ".reg .u64 a, b, t;\n\t"
        "mov.b64 {yl, yh}, %1;\n\t"
        "mov.b64 {wl, wh}, %2;\n\t"
        "mov.b64 {pl, ph}, %3;\n\t"
        "mov.b64 {nl, nh}, %4;\n\t"
        "mul.wide.u32 a, yh, pl;\n\t"
        "mul.wide.u32 b, yl, ph;\n\t"
        "mov.b64 {al, ah}, a;\n\t"
        "mov.b64 {bl, bh}, b;\n\t"
        "add.cc.u32 al, ah, bh;\n\t"       // hi(a) + hi(b): 33 bits
        "addc.u32 c, 0, 0;\n\t"
        "mov.b64 t, {al, c};\n\t"
        "mad.wide.u32 t, yh, ph, t;\n\t"   // quotient estimate Q
        "mov.b64 {ql, qh}, t;\n\t"
        "mul.wide.u32 a, yl, wl;\n\t"      // low 64 bits of y*w + Q*nq
        "mad.wide.u32 a, ql, nl, a;\n\t"
        "mul.lo.u32 h, yl, wh;\n\t"
        "mad.lo.u32 h, yh, wl, h;\n\t"
        "mad.lo.u32 h, ql, nh, h;\n\t"
        "mad.lo.u32 h, qh, nl, h;\n\t"
        "mov.b64 {rl, rh}, a;\n\t"
        "add.u32 rh, rh, h;\n\t"
        "mov.b64 %0, {rl, rh};\n\t"
        "}"
        : "=l"(r)
        : "l"(y), "l"(w), "l"(wp), "l"(nq));
    return r;
}

// y mod q, lazily: result in [0, 3q) for any y < 2^64.  ones = floor(2^64/q)
// (< 2^32 since q > 2^32); the quotient floor(y_hi * ones / 2^32) is at most
// one below floor(y * ones / 2^64).
__device__ __forceinline__ uint64_t reduce_lazy(uint64_t y, uint32_t ones, uint64_t nq)
{
    uint64_t r;
    asm("{\n\t"
        ".reg .u32 yl, yh, nl, nh, ql, qh, rl, rh, h;\n\t"
        ".reg .u64 a;\n\t"
        "mov.b64 {yl, yh}, %1;\n\t"
        "mov.b64 {nl, nh}, %3;\n\t"
        "mul.wide.u32 a, yh, %2;\n\t"
        "mov.b64 {ql, qh}, a;\n\t"          // Q = qh
        "mad.wide.u32 a, qh, nl, %1;\n\t"   // y + Q*nq (low 64 bits)
        "mul.lo.u32 h, qh, nh;\n\t"
        "mov.b64 {rl, rh}, a;\n\t"
        "add.u32 rh, rh, h;\n\t"
        "mov.b64 %0, {rl, rh};\n\t"
        "}"
        : "=l"(r)
        : "l"(y), "r"(ones), "l"(nq));
    return r;
}

__device__ __forceinline__ uint64_t csub(uint64_t x, uint64_t m)
{
    return x >= m ? x - m : x;
}

// canonical residue of x < 3q
__device__ __forceinline__ uint64_t canon3(uint64_t x, uint64_t q)
{
    return csub(csub(x, 2 * q), q);
}

// canonical residue of x < 4q
__device__ __forceinline__ uint64_t canon4(uint64_t x, uint64_t q)
{
    return csub(csub(x, 2 * q), q);
}

// Multiply-accumulate of products x*w with x < 2^56, w < 2^50, as three
// partial sums of 32x32 products:
//   V = s0 + 2^64 c0 + 2^32 s1 + 2^64 s2,
//   s0 = sum xl*wl (carries counted in c0), s1 = sum xl*wh + xh*wl, s2 = sum xh*wh.
// s1, s2 cannot overflow for fewer than 2^7 terms with x < 2^56 (2^13 with x < 2^50).
struct MacAcc {
    uint64_t s0, s1, s2;
    uint32_t c0;
};

__device__ __forceinline__ void mac_zero(MacAcc &a)
{
    a.s0 = a.s1 = a.s2 = 0;
    a.c0 = 0;
}

__device__ __forceinline__ void mac_add(MacAcc &a, uint64_t x, uint64_t w)
{
    asm("{\n\t"
        ".reg .u32 xl, xh, wl, wh;\n\t"
        ".reg .u64 p;\n\t"
        "mov.b64 {xl, xh}, %4;\n\t"
        "mov.b64 {wl, wh}, %5;\n\t"
        "mul.wide.u32 p, xl, wl;\n\t"
        "add.cc.u64 %0, %0, p;\n\t"
        "addc.u32 %3, %3, 0;\n\t"
        "mad.wide.u32 %1, xl, wh, %1;\n\t"
        "mad.wide.u32 %1, xh, wl, %1;\n\t"
        "mad.wide.u32 %2, xh, wh, %2;\n\t"
        "}"
        : "+l"(a.s0), "+l"(a.s1), "+l"(a.s2), "+r"(a.c0)
        : "l"(x), "l"(w));
}

// a += b (same representation; the s0 carry is counted in c0)
__device__ __forceinline__ void mac_merge(MacAcc &a, const MacAcc &b)
{
    asm("{\n\t"
        "add.cc.u64 %0, %0, %4;\n\t"
        "addc.u32 %3, %3, %7;\n\t"
        "add.u64 %1, %1, %5;\n\t"
        "add.u64 %2, %2, %6;\n\t"
        "}"
        : "+l"(a.s0), "+l"(a.s1), "+l"(a.s2), "+r"(a.c0)
        : "l"(b.s0), "l"(b.s1), "l"(b.s2), "r"(b.c0));
}

// V = lo + 2^64 hi of an accumulator: lo = s0 + 2^32 lo32(s1), hi = c0 + s2 + hi32(s1) + carry
__device__ __forceinline__ void mac_value(const MacAcc &a, uint64_t &lo, uint64_t &hi)
{
    asm("{\n\t"
        ".reg .u32 sl, sh, l0, l1, h0;\n\t"
        ".reg .u64 t;\n\t"
        "mov.b64 {sl, sh}, %3;\n\t"
        "mov.b64 {l0, l1}, %2;\n\t"
        "add.cc.u32 l1, l1, sl;\n\t"
        "addc.u32 h0, %5, sh;\n\t"          // c0 + hi32(s1) + carry (< 2^32)
        "mov.b64 %0, {l0, l1};\n\t"
        "cvt.u64.u32 t, h0;\n\t"
        "add.u64 %1, %4, t;\n\t"
        "}"
        : "=l"(lo), "=l"(hi)
        : "l"(a.s0), "l"(a.s1), "l"(a.s2), "r"(a.c0));
}

// canonical (lo + 2^64 hi) mod q for any hi < 2^64.  r64 = 2^64 mod q with companion r64_s.
__device__ __forceinline__ uint64_t reduce128(uint64_t lo, uint64_t hi, uint64_t q, uint64_t nq, uint64_t r64,
                                              uint64_t r64_s, uint32_t ones)
{
    const uint64_t x = shoup_lazy(hi, r64, r64_s, nq);  // < 4q
    const uint64_t y = reduce_lazy(lo, ones, nq);        // < 3q
    uint64_t s = x + y;                                  // < 7q
    s = csub(s, 4 * q);
    return canon4(s, q);
}

// canonical V mod q
__device__ __forceinline__ uint64_t mac_reduce(const MacAcc &a, uint64_t q, uint64_t nq, uint64_t r64,
                                               uint64_t r64_s, uint32_t ones)
{
    uint64_t lo, hi;
    mac_value(a, lo, hi);
    return reduce128(lo, hi, q, nq, r64, r64_s, ones);
}

// canonical V = lo + 2^64 hi mod q for q = 2^50 - c with 0 < c < 2^22, V < 2^104 (at most 16
// terms of products of residues below 2^50): with A = V >> 50 and
// B = V mod 2^50, V = A*2^50 + B = A*c + B (mod q); folding A*c (< 2^76) once
// more the same way leaves B + B2 + A2*c < 2.25 * 2^50 < 3q.  Three wide
// 32-bit products instead of the generic reduction's Shoup step.
__device__ __forceinline__ uint64_t reduce128_special(uint64_t lo, uint64_t hi, uint64_t q, uint32_t c)
{
    constexpr uint64_t M50 = (1ull << 50) - 1;
    const uint64_t A = (hi << 14) | (lo >> 50);  // < 2^54
    const uint64_t B = lo & M50;
    const uint64_t p0 = (uint64_t)(uint32_t)A * c;          // < 2^54
    const uint64_t p1 = (uint64_t)(uint32_t)(A >> 32) * c;  // < 2^44
    const uint64_t plo = p0 + (p1 << 32);
    const uint64_t phi = (p1 >> 32) + (plo < p0 ? 1 : 0);
    const uint64_t A2 = (phi << 14) | (plo >> 50);          // < 2^26
    const uint64_t r = B + (plo & M50) + (uint64_t)(uint32_t)A2 * c;
    return canon3(r, q);
}

__device__ __forceinline__ uint64_t mac_reduce_special(const MacAcc &a, uint64_t q, uint32_t c)
{
    uint64_t lo, hi;
    mac_value(a, lo, hi);
    return reduce128_special(lo, hi, q, c);
}

}  // namespace hc
