// hc_mac_tc.cu -- the NTT-domain convolution MAC (Sec. 6.2) on the 5th-generation
// tensor cores:  Y[m*B+b][c] = sum_g W[m*G+g] . X[g*B+b][c]  (slot-wise, mod q).
//
// For one limb and one NTT slot the MAC is the small dense product
// Y_k = W_k X_k of an M x G matrix by a G x P matrix (P = 2B).  Residues are
// below 2^50, so each is split into seven 8-bit limbs, w = sum_i w_i 2^(8i),
// x = sum_j x_j 2^(8j), and
//     Y = sum_t 2^(8t) S_t,   S_t = sum_g sum_(i+j=t) w_(g,i) x_(g,j),   t = 0..12.
// Every S_t is an exact dot product of small integers, which the tensor core
// computes in fp32 from f16 operands (kind::f16, fp32 accumulator in tensor
// memory):
//     D[m][(p,t)] = sum_(i',g) A[m][(i',g)] B[(p,t)][(i',g)],   i' = 7 - i,
//     A[m][(i',g)] = w_(m,g,7-i'),   B[(p,t)][(i',g)] = x_(g,p,t-7+i')  (0 outside 0..6).
// Exactness: a product is below 2^16 and a column t has at most 7G nonzero
// terms, so for G <= 8 every partial sum of the accumulation stays below 2^22:
// integers that fp32 represents exactly in any order of the additions.  A first
// MMA on two constant tiles (2048 and 4096 at K = 0) seeds every accumulator
// with 2^23, so D lies in [2^23, 2^24) and its fp32 bit pattern is 0x4B000000 +
// S_t; the epilogue shifts and adds the 13 S_t into V < 2^104 and reduces V mod
// q, so the result equals the integer MAC's bit for bit.
//
// Tiles: the MMA is M = 128 rows, N = 16 P columns (column 16p + t), K = 16 per
// instruction.  A unit is one limb, two consecutive slots and a block of 64
// output channels: rows 0-63 hold slot k0's channels, rows 64-127 slot k0+1's,
// and the contraction runs over two K-blocks of 64 -- slot k0's (i', g) against
// rows 0-63, slot k0+1's against rows 64-127 -- with the off-diagonal blocks
// zero.  A is K-major with the 128-byte swizzle, 24 KB: [slot k0 rows | zeros |
// slot k0+1 rows], K-block 0 = the first 16 KB, K-block 1 = the last 16 KB,
// sharing the zero block.  B is K-major without swizzle (core matrices of 8 rows
// x 16 bytes, 16 bytes apart along K and 128 bytes apart along N): row 16p + t
// starts 16 (16p + t) bytes into the slot's array and its chunk i' lies 16 i'
// further, so with K ordered by i' the array of chunks C[16p + 7 + j] = limb j
// of (x_(g,p), g = 0..7) makes the hardware read exactly the shifted rows of B
// -- 7 chunks per (slot, p) instead of 13 rows of 8.
//
// Per CTA (one per SM): 16 worker warps and one issuing warp.  The issuer copies
// stages of four slots (two units) -- the channel block's weights as G blocks of
// 64 channel rows and the input rows, by 2-D tensor copies (32-byte swizzle) --
// and issues each unit's MMAs once the workers have built its operands; the
// workers build A (limbs of the weights, byte-gathered into f16 chunks) and the
// B arrays from the stage, read the previous unit's accumulator, and stage the
// results in shared memory, written to Y in full 32-byte sectors every two
// units.  Two operand buffers and two accumulators overlap unit u's MMAs with
// the workers' work on units u - 1 and u + 1.
//
// Waits are bounded: a wait that runs out sets the context's error word (5),
// drains (bounded) and the CTA frees its tensor memory and returns.
#include <atomic>

#include <cuda.h>

#include "hc_arith.cuh"
#include "hc_async.cuh"
#include "hc_internal.h"
#include "hc_tc.cuh"

namespace hc {

namespace {

constexpr int kTcWorkers = 512;              // warps 0-15
constexpr int kTcThreads = kTcWorkers + 32;  // + the issuing warp
constexpr uint32_t kTcA = 24 * 1024;  // A image
constexpr uint32_t kTcKB = 144 * 16;   // one slot's B chunk array (16 P + 7 chunks used, P <= 8)
constexpr uint32_t kTcBuf = kTcA + 5 * 1024;  // A image + B arrays (4.5 KB), 1024-byte multiple
constexpr uint32_t kTcCols = 256;                // two accumulators of 128 columns

// swizzled byte offset of 16-byte chunk c of row r in a K-block
__device__ __forceinline__ uint32_t chunk_off(uint32_t r, uint32_t c)
{
    return (r >> 3) * 1024u + (r & 7u) * 128u + ((c ^ (r & 7u)) << 4);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

}  // namespace

__device__ __forceinline__ uint64_t ld_shared_u64(uint32_t addr)
{
    uint64_t v;
    asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ void ld_shared_2u64(uint32_t addr, uint64_t &x, uint64_t &y)
{
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(x), "=l"(y) : "r"(addr) : "memory");
}

__device__ __forceinline__ void st_shared_u64(uint32_t addr, uint64_t v)
{
    asm volatile("st.shared.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

// One launch: the layer's units for limbs [limb0, limb0 + Lc); CTA c takes units
// [c * per, (c + 1) * per) (per even): consecutive slot pairs of one limb and
// channel block, in the order (limb, channel block, slot pair).
struct TcMacArgs {
    CUtensorMap wmap;   // W as [M rows][G*L*N], boxes of 4 slots x 64 channels, 32-byte swizzle
    CUtensorMap xmap;   // X as [G*P rows][L*N], one box of 4 slots x G*P rows
    uint64_t *Y;        // [M*P][L][N]; X is [G*P][L][N] and W [M*G][L][N]
    const LimbConst *limbs;
    uint32_t N, L, G, P, M, CB, limb0, Lc, units, per;
};

// position of a unit, advanced without divisions
struct TcPos {
    uint32_t limb, cb, k0;
    __device__ __forceinline__ void next(const TcMacArgs &a)
    {
        k0 += 2;
        if (k0 == a.N) {
            k0 = 0;
            if (++cb == a.CB) {
                cb = 0;
                ++limb;
            }
        }
    }
};

// Shared memory: two operand buffers (A image, B arrays), two input stages (for
// four slots -- two units: the weights of a channel block as G blocks of 64
// channel rows, [g][channel], and the input rows; 32 bytes a row, copied by 2-D
// tensor copies with the 32-byte swizzle: the 16-byte half c of row r sits at
// c ^ (r / 4 % 2)), two output stages (each the 64 P results of two units, row
// (p, channel) at a 48-byte pitch; written out while the other fills).
constexpr uint32_t kTcXOff = 16 * 1024;            // input rows of a stage
constexpr uint32_t kTcStage = kTcXOff + 64 * 32;   // 18 KB
constexpr uint32_t kTcRow = 48;                    // output stage pitch
constexpr uint32_t kTcYStage = 512 * kTcRow;
constexpr uint32_t kTcStageOff = 2 * kTcBuf;
constexpr uint32_t kTcYOff = kTcStageOff + 2 * kTcStage;
// the accumulator seed: A and B tiles (K-major, no swizzle, 128 rows, K = 16) whose
// only nonzero is 2048 and 4096 at K = 0, so that one MMA sets every D to 2^23
constexpr uint32_t kTcSeedOff = kTcYOff + 2 * kTcYStage;
constexpr uint32_t kTcSeed = 4096;  // one tile: 16 core matrices of 8 rows x 16 bytes, twice along K
constexpr uint32_t kTcSmem = kTcSeedOff + 2 * kTcSeed + 1024;

// byte offset of 16-byte half c of row r in a stage region
__device__ __forceinline__ uint32_t stage_off(uint32_t r, uint32_t c)
{
    return r * 32u + ((c ^ ((r >> 2) & 1u)) << 4);
}

// What one thread does in every unit (fixed for the whole launch).
//   A (tid < 256, warps 0-7): row (slot, channel) = 32 (w / 2) + lane of the 128
//     MMA rows; half-word hw = w % 2 of the row's G weights: the high words give
//     chunks 1-3 (limbs 6-4; chunk 0, limb 7, is zero), the low words chunks 4-7.
//   B: tid < 16 P: (slot, column block p) = tid / 8, limb j = tid % 8 < 7: chunk
//     7 + j of the pair's array.
//   Epilogue: TMEM lane 32 (w % 4) + lane = row (slot, channel), column blocks
//     p = w / 4 and w / 4 + 4.
struct TcRole {
    uint32_t a_ok, a_hw, a_slot, a_ml;
    uint32_t b_ok, b_p, b_j, b_slot, b_soff;
    uint32_t e_slot, e_ml;
};

__device__ __forceinline__ TcRole tc_role(const TcMacArgs &a, int tid)
{
    TcRole r{};
    const uint32_t t = (uint32_t)tid, w = t >> 5;
    if (t < 256) {
        const uint32_t row = 32 * (w >> 1) + (t & 31);
        r.a_ok = 1;
        r.a_hw = w & 1;
        r.a_slot = row >> 6;
        r.a_ml = row & 63;
    }
    if (t < 16 * a.P && (t & 7) < 7) {
        const uint32_t pair = t >> 3;
        r.b_ok = 1;
        r.b_slot = pair & 1;
        r.b_p = pair >> 1;
        r.b_j = t & 7;
        r.b_soff = r.b_slot * kTcKB + (16 * r.b_p + 7 + r.b_j) * 16;
    }
    const uint32_t row = 32 * (w & 3) + (t & 31);
    r.e_slot = row >> 6;
    r.e_ml = row & 63;
    return r;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// the tensor copies of one stage (slots k0 .. k0 + 3), issued by one thread after its
// expect_tx of tc_stage_bytes; channels beyond the tensor read as zero
__device__ __forceinline__ void tc_stage_copy(const TcMacArgs &a, const TcPos &u, uint32_t stage, uint64_t *full)
{
    const int x = (int)(u.limb * a.N + u.k0);
    const int LN = (int)(a.L * a.N);
    for (uint32_t g = 0; g < a.G; ++g) tma_load_2d(stage + g * 2048u, &a.wmap, (int)g * LN + x, (int)(u.cb * 64), full);
    tma_load_2d(stage + kTcXOff, &a.xmap, x, 0, full);
}

__device__ __forceinline__ uint32_t tc_stage_bytes(const TcMacArgs &a)
{
    return (64 * a.G + a.G * a.P) * 32;
}

__device__ __forceinline__ uint32_t ld_shared_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// the 16-byte chunk of f16 values {byte b of v[g], g = 0..7}: word k holds groups
// 2k, 2k + 1; vw[g] is the 32-bit half of v[g] that holds byte b, bs = b % 4
__device__ __forceinline__ void gather_chunk(const uint32_t (&vw)[8], uint32_t bs, uint32_t &c0, uint32_t &c1,
                                             uint32_t &c2, uint32_t &c3)
{
    const uint32_t sel = bs | ((4u + bs) << 8);  // byte bs of the first word -> 0, of the second -> 2
    uint32_t c[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t t = (__byte_perm(vw[2 * k], vw[2 * k + 1], sel) & 0x00FF00FFu) | 0x64006400u;
        asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(c[k]) : "r"(t), "r"(0x64006400u));
    }
    c0 = c[0];
    c1 = c[1];
    c2 = c[2];
    c3 = c[3];
}

// operands of the unit in half h (0, 1) of the stage at `stage`.  K = (i', g) with
// i' = 7 - i: chunk i' of a row holds limb 7 - i' of the G (<= 8) values.
__device__ __forceinline__ void tc_build(const TcMacArgs &a, const TcRole &r, uint32_t stage, uint32_t h,
                                         uint32_t sA, uint32_t sB)
{
    const uint32_t G = a.G, P = a.P;
    if (r.a_ok) {  // A: chunks of row (slot, channel) from one half-word of each weight
        const uint32_t off = stage_off(r.a_ml, h) + r.a_slot * 8 + r.a_hw * 4;
        uint32_t vw[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) vw[g] = (uint32_t)g < G ? ld_shared_u32(stage + g * 2048u + off) : 0u;
        const uint32_t ab = sA + r.a_slot * 16384u;
        uint32_t c0, c1, c2, c3;
        if (r.a_hw) {  // limbs 6, 5, 4 (bytes 2, 1, 0 of the high word) -> chunks 1, 2, 3
#pragma unroll
            for (uint32_t c = 1; c < 4; ++c) {
                gather_chunk(vw, 3 - c, c0, c1, c2, c3);
                st_shared_v4(ab + chunk_off(r.a_ml, c), c0, c1, c2, c3);
            }
        } else {  // limbs 3..0 (bytes 3..0 of the low word) -> chunks 4..7
#pragma unroll
            for (uint32_t c = 4; c < 8; ++c) {
                gather_chunk(vw, 7 - c, c0, c1, c2, c3);
                st_shared_v4(ab + chunk_off(r.a_ml, c), c0, c1, c2, c3);
            }
        }
    }
    if (r.b_ok) {  // B: chunk 7 + j of the (slot, p) array = limb j of x_(g,p), g = 0..7
        uint32_t vw[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            vw[g] = 0;
            if ((uint32_t)g < G) {
                const uint64_t x = ld_shared_u64(stage + kTcXOff + stage_off(g * P + r.b_p, h) + r.b_slot * 8);
                vw[g] = r.b_j >= 4 ? (uint32_t)(x >> 32) : (uint32_t)x;
            }
        }
        uint32_t c0, c1, c2, c3;
        gather_chunk(vw, r.b_j & 3, c0, c1, c2, c3);
        st_shared_v4(sB + r.b_soff, c0, c1, c2, c3);
    }
}

// u = raw bits of D = 2^23 + S_t (t = 0..12): V = sum_t S_t 2^(8t) = lo + 2^64 hi.
// a_k = sum_b u_(4k+b) 2^(8b) - K4 (K4 = the 2^23 terms' share, K = 0x4B000000),
// a_3 = u_12 - K, each below 2^47; V = a0 + 2^32 a1 + 2^64 a2 + 2^96 a3.
__device__ __forceinline__ void tc_combine(const uint32_t (&u)[16], uint64_t &lo, uint64_t &hi)
{
    constexpr uint64_t K = 0x4B000000ull;
    constexpr uint64_t NEG_K4 = 0ull - (K + (K << 8) + (K << 16) + (K << 24));
    asm("{\n\t.reg .u64 a0, a1, a2;\n\t.reg .u32 a0l, a0h, a1l, a1h, a2l, a2h, a3, l1, h0, h1;\n\t"
        "mad.wide.u32 a0, %2, 1, %15;\n\t"
        "mad.wide.u32 a0, %3, 256, a0;\n\t"
        "mad.wide.u32 a0, %4, 65536, a0;\n\t"
        "mad.wide.u32 a0, %5, 16777216, a0;\n\t"
        "mad.wide.u32 a1, %6, 1, %15;\n\t"
        "mad.wide.u32 a1, %7, 256, a1;\n\t"
        "mad.wide.u32 a1, %8, 65536, a1;\n\t"
        "mad.wide.u32 a1, %9, 16777216, a1;\n\t"
        "mad.wide.u32 a2, %10, 1, %15;\n\t"
        "mad.wide.u32 a2, %11, 256, a2;\n\t"
        "mad.wide.u32 a2, %12, 65536, a2;\n\t"
        "mad.wide.u32 a2, %13, 16777216, a2;\n\t"
        "sub.u32 a3, %14, 0x4B000000;\n\t"
        "mov.b64 {a0l, a0h}, a0;\n\t"
        "mov.b64 {a1l, a1h}, a1;\n\t"
        "mov.b64 {a2l, a2h}, a2;\n\t"
        "add.cc.u32 l1, a0h, a1l;\n\t"
        "addc.cc.u32 h0, a2l, a1h;\n\t"
        "addc.u32 h1, a2h, a3;\n\t"
        "mov.b64 %0, {a0l, l1};\n\t"
        "mov.b64 %1, {h0, h1};\n\t}"
        : "=l"(lo), "=l"(hi)
        : "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(u[4]), "r"(u[5]), "r"(u[6]), "r"(u[7]), "r"(u[8]),
          "r"(u[9]), "r"(u[10]), "r"(u[11]), "r"(u[12]), "l"(NEG_K4));
}

// canonical V mod q for V = lo + 2^64 hi < 2^104 and q = 2^50 - c, 0 < c < 2^22:
// V = A 2^50 + B = B + A c (mod q) with A < 2^54, then R = B + A c < 2^77 folds
// once more the same way to below 2^50 + 2^49 < 2q, and one subtraction finishes.
__device__ __forceinline__ uint64_t reduce104_special(uint64_t lo, uint64_t hi, uint64_t q, uint32_t c)
{
    uint64_t r;
    asm("{\n\t.reg .u32 l0, l1, h0, h1, A0, A1, b1, r0, r1, r2, t0, t1, R1, R0h;\n\t"
        ".reg .u64 s, t, B, v;\n\t.reg .pred ge;\n\t"
        "mov.b64 {l0, l1}, %1;\n\t"
        "mov.b64 {h0, h1}, %2;\n\t"
        "shf.r.clamp.b32 A0, l1, h0, 18;\n\t"  // V bits 50..81
        "shf.r.clamp.b32 A1, h0, h1, 18;\n\t"  // V bits 82..103
        "and.b32 b1, l1, 0x3FFFF;\n\t"
        "mov.b64 B, {l0, b1};\n\t"             // V mod 2^50
        "mad.wide.u32 s, A0, %4, B;\n\t"       // < 2^55
        "mul.wide.u32 t, A1, %4;\n\t"          // < 2^44, weight 2^32
        "mov.b64 {r0, r1}, s;\n\t"
        "mov.b64 {t0, t1}, t;\n\t"
        "add.cc.u32 r1, r1, t0;\n\t"
        "addc.u32 r2, t1, 0;\n\t"              // R = r0 + 2^32 r1 + 2^64 r2 < 2^77
        "shf.r.clamp.b32 R1, r1, r2, 18;\n\t"  // R >> 50 < 2^27
        "and.b32 R0h, r1, 0x3FFFF;\n\t"
        "mov.b64 v, {r0, R0h};\n\t"
        "mad.wide.u32 v, R1, %4, v;\n\t"       // < 2^50 + 2^49
        "setp.ge.u64 ge, v, %3;\n\t"
        "@ge sub.u64 v, v, %3;\n\t"
        "mov.b64 %0, v;\n\t}"
        : "=l"(r)
        : "l"(lo), "l"(hi), "l"(q), "r"(c));
    return r;
}

// results of the unit in half par of its output group into the output stage ys
__device__ __forceinline__ void tc_epilogue(const TcMacArgs &a, const TcRole &r, const TcPos &u, uint32_t acc,
                                            uint32_t ys, uint32_t par, int tid)
{
    const uint32_t w = (uint32_t)tid >> 5, qd = w & 3;
    const LimbConst &lc = a.limbs[u.limb];
    const uint64_t q = lc.q;
    const uint32_t sc = (uint32_t)lc.special_c;
    const uint32_t p0 = w >> 2, p1 = p0 + 4;  // warp-uniform; P <= 8
    uint32_t v0[16], v1[16];
    const uint32_t ta = acc + ((32 * qd) << 16);
    if (p0 < a.P) tmem_ld16(ta + 16 * p0, v0);
    if (p1 < a.P) tmem_ld16(ta + 16 * p1, v1);
    tmem_ld_wait();
    const uint32_t yo = ys + r.e_ml * kTcRow + (2 * par + r.e_slot) * 8;
    auto out = [&](const uint32_t(&v)[16], uint32_t p) {  // v[t] = bits of 2^23 + S_t
        uint64_t lo, hi;
        tc_combine(v, lo, hi);
        const uint64_t y = sc ? reduce104_special(lo, hi, q, sc)
                              : reduce128(lo, hi, q, 0ull - q, lc.r64, lc.r64_s, (uint32_t)lc.one_s);
        st_shared_u64(yo + p * 64 * kTcRow, y);
    };
    if (p0 < a.P) out(v0, p0);
    if (p1 < a.P) out(v1, p1);
}

// the output stage (stage row p * 64 + channel, four slots from k0) to Y in 16-byte pieces
__device__ __forceinline__ void tc_flush(const TcMacArgs &a, const TcPos &u, uint32_t ys, int tid)
{
    const size_t LN = (size_t)a.L * a.N, off = (size_t)u.limb * a.N + u.k0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const uint32_t i = (uint32_t)tid + kTcWorkers * j, row = i >> 1, half = i & 1;
        const uint32_t p = row >> 6, m = u.cb * 64 + (row & 63);
        if (p < a.P && m < a.M) {
            uint64_t y0, y1;
            ld_shared_2u64(ys + row * kTcRow + half * 16, y0, y1);
            *reinterpret_cast<ulonglong2 *>(a.Y + (size_t)(m * a.P + p) * LN + off + 2 * half) = make_ulonglong2(y0, y1);
        }
    }
}

__device__ __forceinline__ void mbar_arrive1(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar)) : "memory");
}

// the 512 worker threads only (the issuing warp does not take part)
__device__ __forceinline__ void workers_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kTcWorkers) : "memory");
}

// Warps 0-15 (workers) build operands, wait for each unit's MMAs and finish the
// results; warp 16 (issuer) copies the stages and issues the MMAs.  They meet
// only on mbarriers: ready[b] (one arrival per worker warp: the operands of the
// unit in buffer b are written and the accumulator b is read out), done[b]
// (tcgen05 commit: the unit's MMAs completed), full[s] (a stage's copies landed).
__global__ void __launch_bounds__(kTcThreads, 1) k_mac_tc(const __grid_constant__ TcMacArgs a, int *err)
{
    extern __shared__ __align__(16) uint8_t tc_smem[];
    __shared__ __align__(8) uint64_t bars[6];  // 0, 1: done; 2, 3: full; 4, 5: ready
    __shared__ uint32_t tbase_s;
    const int tid = threadIdx.x;
    const uint32_t raw = smem_addr(tc_smem);
    const uint32_t sbase = (raw + 1023u) & ~1023u;  // swizzle atoms on 1024-byte boundaries
    const uint32_t stage0 = sbase + kTcStageOff, ys0 = sbase + kTcYOff;
    for (uint32_t o = (uint32_t)tid * 16; o < 2 * kTcBuf; o += kTcThreads * 16) st_shared_v4(sbase + o, 0, 0, 0, 0);
    const uint32_t seedA = sbase + kTcSeedOff, seedB = seedA + kTcSeed;
    for (uint32_t o = (uint32_t)tid * 16; o < 2 * kTcSeed; o += kTcThreads * 16) {
        // row r of a tile sits at (r / 8) * 128 + (r % 8) * 16 in its first 2 KB (K = 0..7)
        const uint32_t lead = o < kTcSeed ? 0x00006800u : 0x00006C00u;  // f16 2048 / 4096 at K = 0
        st_shared_v4(seedA + o, (o % kTcSeed) < 2048 ? lead : 0u, 0, 0, 0);
    }
    fence_proxy_async();
    const uint32_t u0 = blockIdx.x * a.per, u1 = min(a.units, u0 + a.per);
    const uint32_t n = u1 - u0, nst = n / 2;  // units and stages (two units each) of this CTA
    const uint32_t pairs = a.N >> 1, rest = u0 / pairs;
    const TcPos start{a.limb0 + rest / a.CB, rest % a.CB, (u0 - rest * pairs) * 2};
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
        mbar_init(&bars[4], kTcWorkers / 32);
        mbar_init(&bars[5], kTcWorkers / 32);
        mbar_fence_init();
    }
    if (tid < 32) {
        tmem_alloc(&tbase_s, kTcCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tbase_s;
    bool bad = false;
    uint32_t c = 0, issued = 0;  // issuer: units issued, stages issued
    if (tid >= kTcWorkers) {
        if (tid == kTcWorkers) {  // ---- issuer ----
            TcPos sp = start;
            for (; issued < 2 && issued < nst; ++issued) {
                mbar_arrive_expect_tx(&bars[2 + issued], tc_stage_bytes(a));
                tc_stage_copy(a, sp, stage0 + issued * kTcStage, &bars[2 + issued]);
                sp.next(a);
                sp.next(a);
            }
            const uint32_t idesc = tc_idesc_f16(128, 16 * a.P);
            for (; c < n; ++c) {
                const uint32_t b = c & 1, j = c >> 1, sb = j & 1;
                if (!mbar_wait(&bars[4 + b], (c >> 1) & 1)) {
                    bad = true;
                    break;
                }
                tc_fence_after();
                if ((c & 1) && issued < nst) {  // stage j is read: copy stage j + 2 into it
                    fence_proxy_async();
                    mbar_arrive_expect_tx(&bars[2 + sb], tc_stage_bytes(a));
                    tc_stage_copy(a, sp, stage0 + sb * kTcStage, &bars[2 + sb]);
                    sp.next(a);
                    sp.next(a);
                    ++issued;
                }
                const uint32_t sA = sbase + b * kTcBuf, sB = sA + kTcA;
                tc_mma_f16(tbase + 128 * b, tc_desc_plain(seedA, 2048, 128), tc_desc_plain(seedB, 2048, 128), idesc,
                           0);  // D = 2^23
#pragma unroll
                for (uint32_t k = 0; k < 2; ++k)  // K-block k: slot k0 + k
#pragma unroll
                    for (uint32_t ks = 0; ks < 4; ++ks)
                        tc_mma_f16(tbase + 128 * b, tc_desc_sw128(sA + k * 8192 + ks * 32, 1024),
                                   tc_desc_plain(sB + k * kTcKB + ks * 32, 16, 128), idesc, 1);
                tc_commit(&bars[b]);
            }
        }
    } else {  // ---- workers ----
        const TcRole role = tc_role(a, tid);
        const uint32_t lane = tid & 31;
        TcPos cur = start, prev = start;
        for (uint32_t u = 0; u < n; ++u) {
            const uint32_t h = u & 1, j = u >> 1, sb = j & 1, b = u & 1;
            if (h == 0 && !bad && !__all_sync(0xffffffffu, mbar_wait(&bars[2 + sb], (j >> 1) & 1))) bad = true;
            const uint32_t sA = sbase + b * kTcBuf, sB = sA + kTcA;
            tc_build(a, role, stage0 + sb * kTcStage, h, sA, sB);
            fence_proxy_async();  // this thread's operand writes before the MMAs read them
            tc_fence_before();    // and its reads of accumulator b (unit u - 2) before the MMAs write it
            __syncwarp();
            if (lane == 0) mbar_arrive1(&bars[4 + b]);
            if (u >= 1) {  // the previous unit
                const uint32_t e = u - 1, pb = e & 1;
                const bool ok = !bad && __all_sync(0xffffffffu, mbar_wait(&bars[pb], (e >> 1) & 1));
                tc_fence_after();
                const uint32_t ys = ys0 + ((e >> 1) & 1) * kTcYStage;
                if (ok) tc_epilogue(a, role, prev, tbase + 128 * pb, ys, e & 1, tid);
                else bad = true;
                tc_fence_before();
                if (e & 1) {  // the output stage holds two units: write it out
                    workers_sync();
                    TcPos g = prev;
                    g.k0 -= 2;
                    tc_flush(a, g, ys, tid);
                }
            }
            prev = cur;
            cur.next(a);
        }
        if (n >= 1) {  // the last unit (odd: n is even)
            const uint32_t e = n - 1, pb = e & 1;
            const bool ok = !bad && __all_sync(0xffffffffu, mbar_wait(&bars[pb], (e >> 1) & 1));
            tc_fence_after();
            const uint32_t ys = ys0 + ((e >> 1) & 1) * kTcYStage;
            if (ok) tc_epilogue(a, role, prev, tbase + 128 * pb, ys, e & 1, tid);
            else bad = true;
            tc_fence_before();
            workers_sync();
            TcPos g = prev;
            g.k0 -= 2;
            tc_flush(a, g, ys, tid);
        }
    }
    bad = __syncthreads_or(bad);
    if (bad) {
        if (tid == kTcWorkers) {
            atomicExch(err, 5);
            // MMAs and copies that may still run: wait (bounded) before the CTA's memory is released
            for (uint32_t k = c >= 2 ? c - 2 : 0; k < c; ++k) mbar_wait(&bars[k & 1], (k >> 1) & 1);
            for (uint32_t k = issued >= 2 ? issued - 2 : 0; k < issued; ++k) mbar_wait(&bars[2 + (k & 1)], (k >> 1) & 1);
        }
        tc_fence_before();
        __syncthreads();
    }
    tc_fence_after();
    if (tid < 32) tmem_dealloc(tbase, kTcCols);
}

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once through the runtime
EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// a [rows][LN] uint64 matrix at base (row pitch LN words), boxes of 4 columns x box_rows rows
hc_status encode_rows(CUtensorMap *map, const uint64_t *base, uint64_t rows, uint64_t LN, uint32_t box_rows)
{
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return set_error(HC_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t dims[2] = {LN, rows};
    const cuuint64_t strides[1] = {LN * sizeof(uint64_t)};
    const cuuint32_t box[2] = {4, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(HC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return HC_OK;
}

}  // namespace

bool mac_tc_fits(uint32_t G, uint32_t B)
{
    return G >= 1 && G <= 8 && B >= 1 && 2 * B <= 8;
}

hc_status launch_mac_tc(const hc_ctx *ctx, const uint64_t *x, const uint64_t *w, uint64_t *y, uint32_t G, uint32_t B,
                        uint32_t M, uint32_t limb0, uint32_t Lc, cudaStream_t s)
{
    if (!mac_tc_fits(G, B)) return set_error(HC_ERR_UNSUPPORTED, "tensor-core MAC: G = %u, B = %u", G, B);
    if (Lc == 0) Lc = ctx->L;
    if (M == 0 || Lc == 0) return HC_OK;
    static std::atomic<uint32_t> attr_done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(attr_done.load() & (1u << (dev & 31)))) {
        cudaError_t e = cudaFuncSetAttribute(k_mac_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(k_mac_tc)");
        attr_done.fetch_or(1u << (dev & 31));
    }
    TcMacArgs a{};
    a.Y = y;
    a.limbs = ctx->d_limbs;
    a.N = ctx->N;
    a.L = ctx->L;
    a.G = G;
    a.P = 2 * B;
    a.M = M;
    a.CB = (M + 63) / 64;
    a.limb0 = limb0;
    a.Lc = Lc;
    a.units = Lc * a.CB * (ctx->N / 2);
    const uint64_t LN = (uint64_t)ctx->L * ctx->N;
    hc_status st = encode_rows(&a.wmap, w, M, G * LN, 64);
    if (st == HC_OK) st = encode_rows(&a.xmap, x, (uint64_t)G * 2 * B, LN, G * 2 * B);
    if (st != HC_OK) return st;
    const uint32_t ctas = a.units < ctx->sms ? a.units : ctx->sms;  // one resident CTA per SM
    a.per = (a.units + ctas - 1) / ctas;
    a.per += a.per & 1;  // whole stages of two units
    const uint32_t grid = (a.units + a.per - 1) / a.per;
    ProfileScope ps("k_mac_tc", s);
    k_mac_tc<<<grid, kTcThreads, kTcSmem, s>>>(a, timeout_flag(ctx));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HC_OK : cuda_error(e, "k_mac_tc");
}

}  // namespace hc
