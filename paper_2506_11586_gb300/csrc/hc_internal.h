// hc_internal.h -- internal types of libhconv (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "hconv.h"

namespace hc {

constexpr uint32_t kMaxLimbs = 8;
constexpr uint32_t kMagicCtx = 0x48435458u;      // 'HCTX'
constexpr uint32_t kMagicWeights = 0x48435754u;  // 'HCWT'
constexpr uint32_t kMagicPlan = 0x4843504Cu;     // 'HCPL'
constexpr uint32_t kMagicServer = 0x48435352u;   // 'HCSR'
constexpr uint32_t kMagicGaloisKey = 0x4843474Bu;  // 'HCGK'
constexpr uint32_t kMagicDead = 0xDEADDEADu;

// Per-limb constants and twiddle tables, device-resident, read through the
// read-only path.  Every Shoup companion w' = floor(w * 2^64 / q).
struct LimbConst {
    uint64_t q;
    uint64_t r64, r64_s;      // 2^64 mod q, companion
    uint64_t one_s;           // companion of 1: floor(2^64 / q)
    uint64_t ninv, ninv_s;    // N^-1 mod q, companion
    uint64_t ninvw, ninvw_s;  // N^-1 * psi^-rev(1) mod q, companion (last GS stage)
    const ulonglong2 *tw_f;   // [N] {psi^rev(k), companion}, rev over log2 N bits
    const ulonglong2 *tw_i;   // [N] {psi^-rev(k), companion}
    uint64_t delta, delta_s;  // BFV scale floor(Q/t) mod q (Q = product of all limbs), companion
    uint64_t special_c;       // c when q = 2^50 - c with 0 < c < 2^22 (cheaper MAC reduction), else 0
    // Twiddles of the register rounds in which every thread needs its own ones,
    // rearranged so that the threads of a warp read consecutive entries, for
    // transforms with 2^LOGC residues per thread (T = N >> LOGC threads): table
    // tw_r + (3*d + LOGC - 3)*N, d = 0 inverse (first round), d = 1 forward (last
    // round); layouts in hc_ntt.cuh.  Tables with LOGC >= log2 N stay unset.
    const ulonglong2 *tw_r;
    uint64_t pad_[2];         // 128-byte stride
};
static_assert(sizeof(LimbConst) == 128, "LimbConst is 128 bytes");

// Kernel families whose launch shape is selectable per context.
enum KernelKind {
    KK_FWD = 0, KK_INV = 1, KK_MAC = 2, KK_PROD = 3, KK_FWDCT = 4, KK_INVCT = 5, KK_MACB = 6,
    KK_CONV = 7,  // convolution launch form: 0 three launches per degree, 1 one fused persistent launch,
                  // 2 three launches per limb, the limbs' chains on parallel streams
    KK_COUNT = 8
};
constexpr int kNumVariants = 3;
// the blocked convolution MAC has one more: the tensor-core MAC (hc_mac_tc.cu)
constexpr int kMacTcVariant = 3;
constexpr int kind_variants(int kind)
{
    return kind == KK_MACB ? kNumVariants + 1 : kNumVariants;
}

// One output slot of a layer's output ciphertext: coefficient k holds output
// row n of the ciphertext's No packed rows at block-local position (i, j).
struct SlotEntry {
    uint16_t k, n, i, j;
};

// The inverse transform of a layer's NTT-domain outputs y [O][2][L][N] with the
// server step's epilogue: c1 stored in full to c1 [O][L][N]; c0 reduced to its
// S output slots minus Delta * mask into slots [O][L][S] (0 outside the output
// map or past M).  Output ct o = m'*B + b, block b = bh*Bw + bw.
struct ExtractArgs {
    const uint64_t *y;
    uint64_t *c1;
    uint64_t *slots;
    const uint64_t *mask;     // [M][Ho][Wo] residues in [0, t), or null
    const SlotEntry *table;   // [S]
    uint32_t O, S, B, Bw, oh, ow, Ho, Wo, No, M;
    uint32_t limb0 = 0, Lc = 0;  // limbs [limb0, limb0 + Lc) only (Lc = 0: all L)
};

}  // namespace hc

struct hc_ctx {
    uint32_t magic;
    uint32_t N, logN, L;
    uint64_t t;
    uint32_t flags;
    int device;
    uint32_t sms;             // streaming multiprocessors of `device` (grid sizing)
    uint64_t q[hc::kMaxLimbs];
    uint64_t psi[hc::kMaxLimbs];
    hc::LimbConst *d_limbs;   // [L]
    void *d_tables;           // twiddle storage (owned)
    size_t table_bytes;
    int *d_flag;              // device error flag for checked mode (owned)
    uint8_t variant[hc::KK_COUNT];  // launch-shape variant per kernel family
};

// A linear layer is held as a stride-1 convolution without output packing
// restrictions: `desc` is that convolution (for a strided layer the layer of
// the phase-split input, for a fully connected layer a 1x1 convolution on a
// 1x1 image) with its resolved partition; `No` output channels share one
// output polynomial at coefficient shifts of Cw*Hw*Ww, so Mp = ceil(M/No)
// output polynomials per spatial block.  Convolutions have No = 1, Mp = M.
enum LayerKind : uint32_t { LAYER_CONV = 0, LAYER_FC = 1 };

// The stride-1 layer computed for a caller's layer, and its geometry.
struct LayerGeom {
    hc_conv_desc eff;
    uint32_t No, Mp, pa, pb, G, B, I, P, O;
};

struct hc_weights {
    uint32_t magic;
    const hc_ctx *ctx;
    int device;
    hc_conv_desc desc;        // the stride-1 layer computed, resolved partition
    hc_conv_desc user;        // the layer as described by the caller (stride, pad, C/H/W/kh/kw of its tensors)
    uint32_t kind;            // LayerKind
    uint32_t No, Mp;          // output channels per output polynomial, output polynomials per block
    uint32_t pa, pb;          // row and column phases of a strided layer (1, 1 for stride 1)
    uint32_t G, B, I, P, O;   // P = Mp*G, O = Mp*B
    uint32_t mode;            // hc_weights_mode
    uint64_t *d_pt;           // [P][L][N] NTT domain (offline mode) or coefficient domain (online mode), owned
    int8_t *d_k;              // [M][C][kh][kw] (no-NTT mode), owned
    hc::SlotEntry *d_slot_table;  // [No*oh*ow] output slots of one output ciphertext (owned)
    uint32_t *d_terms;        // CSR of output terms (owned): see mac kernels
    uint32_t *d_term_ptr;     // [O+1]
};

namespace hc {

// inverse transform with the server step's output epilogue (ExtractArgs)
hc_status launch_inv_extract(const hc_ctx *ctx, const ExtractArgs &ex, cudaStream_t s);
// the output slot table of w (built once per weights handle)
hc_status build_slot_table(hc_weights *w);

// Geometry of a Z_P convolution (hc_zp_conv*): zero-padded image of Hp x Wp slots
// (Hp*Wp <= N/2), Y = ceil(M/2) output ciphertexts, rotation steps 1 (within a
// kernel row) and Wp - kw + 1 (to the next kernel row)
struct ZpConvGeom {
    uint32_t Hp, Wp, Ho, Wo, Y, step_row;
};
hc_status zp_conv_geometry(const hc_conv_desc *d, uint32_t N, ZpConvGeom *g);

// frees a Galois key handle (hc_rotate.cu)
void galois_key_destroy(hc_galois_key *k);

// keep freed per-call scratch cached in the device's default memory pool
void keep_scratch_cached(int device);

// Geometry of a layer from the caller's descriptor (kind LAYER_CONV: any stride;
// LAYER_FC: the 1x1 convolution {C,1,1,M,1,1,1,0,Cw,1,1} with No rows per output)
// with an explicit partition, as saved weights store it.
hc_status layer_geometry(const hc_conv_desc &user, uint32_t kind, uint32_t No, uint32_t N, LayerGeom *out);

// ---- error reporting ------------------------------------------------------
hc_status set_error(hc_status s, const char *fmt, ...);
hc_status cuda_error(cudaError_t e, const char *what);

#define HC_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t e__ = (expr);                           \
        if (e__ != cudaSuccess) return hc::cuda_error(e__, #expr); \
    } while (0)

// ---- allocation -------------------------------------------------------------
void *dev_alloc(size_t bytes, cudaStream_t s);            // per-call scratch, stream ordered
void dev_free(void *p, cudaStream_t s);
void *dev_alloc_persistent(size_t bytes);                 // handle-owned memory
void dev_free_persistent(void *p);

// ---- device guard -------------------------------------------------------------
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};

// ---- per-thread launch overrides ------------------------------------------------
// Side streams (and their fork / join events) for launch form 2's per-limb chains.
struct SidePool {
    std::vector<cudaStream_t> st;
    std::vector<cudaEvent_t> ev;  // [0]: fork, [1 + i]: join of side stream i
    int priority = 0;             // CUDA stream priority of the side streams made
};
// Word that the bounded device waits of the calling thread's launches report a
// timeout into: the context's device flag, unless a LaunchScope on this thread
// names another one.
int *timeout_flag(const hc_ctx *ctx);
// While alive, the calling thread's launches report timeouts into `flag` and run
// per-limb chains on `side` (either may be null: the defaults).  The request
// loop gives every stream slot its own flag and side streams, so that batches in
// flight on different slots neither share an error word nor serialise on
// shared side streams.
struct LaunchScope {
    LaunchScope(int *flag, SidePool *side);
    ~LaunchScope();
    LaunchScope(const LaunchScope &) = delete;
    LaunchScope &operator=(const LaunchScope &) = delete;

  private:
    int *prev_flag_;
    SidePool *prev_side_;
};
SidePool *side_override();

// ---- tracing: CUDA events around one launch when hc_profile_enable(1) ----------
bool profile_enabled();
class ProfileScope {
   public:
    ProfileScope(const char *name, cudaStream_t s);
    ~ProfileScope();
    ProfileScope(const ProfileScope &) = delete;
    ProfileScope &operator=(const ProfileScope &) = delete;

   private:
    const char *name_;
    cudaStream_t s_;
    cudaEvent_t start_ = nullptr, stop_ = nullptr;
    bool active_ = false;
};

// ---- host-side number theory (independent of any test code) -----------------
bool is_prime_u64(uint64_t n);
uint64_t mulmod_u64(uint64_t a, uint64_t b, uint64_t q);
uint64_t powmod_u64(uint64_t a, uint64_t e, uint64_t q);
uint64_t min_primitive_2n_root(uint64_t q, uint32_t N);
// floor(prod(moduli) / t) mod q_i for every limb (exact multi-precision)
void delta_residues(const uint64_t *moduli, uint32_t L, uint64_t t, uint64_t *out);
uint64_t shoup_companion(uint64_t w, uint64_t q);
uint32_t bit_reverse(uint32_t k, uint32_t logn);

// ---- kernel launchers (hc_kernels.cu) -------------------------------------------
struct MacTerms {
    const uint32_t *term_ptr;  // [n_out + 1] CSR offsets into terms
    const uint32_t *terms;     // pairs (ct index, pt index), 2 per term
};

// one batch of a multi-segment transform launch: n_groups CTAs per limb (in
// ciphertexts for the *_SEGS kinds), CTAs [cta_begin, cta_begin + n_groups * L)
struct NttSeg {
    const uint64_t *in;
    uint64_t *out;
    const LimbConst *limbs;
    uint32_t L, n_groups, cta_begin;
    uint32_t Lc = 0, limb0 = 0;  // limbs [limb0, limb0 + Lc) only (Lc = 0: all L); L stays the layout stride
};
__host__ __device__ inline uint32_t seg_limbs(const NttSeg &s) { return s.Lc ? s.Lc : s.L; }
constexpr int kMaxSegs = 48;
template <int NS>
struct NttSegsT {
    uint32_t n;
    NttSeg s[NS];
};
using NttSegs = NttSegsT<kMaxSegs>;  // multi-layer launches
using NttSegs1 = NttSegsT<1>;        // one segment: a small kernel-parameter block
// one layer of a multi-layer blocked-MAC launch (see k_mac_conv)
struct MacSeg {
    const uint64_t *X;
    const uint64_t *W;
    uint64_t *Y;
    const LimbConst *limbs;
    uint32_t N, L, G, B, M, MB, MS, KC, chunks, groups, cta_begin;
    uint32_t Lc = 0, limb0 = 0;  // limbs [limb0, limb0 + Lc) only (Lc = 0: all L); L stays the layout stride
};
__host__ __device__ inline uint32_t seg_limbs(const MacSeg &s) { return s.Lc ? s.Lc : s.L; }
template <int NS>
struct MacSegsT {
    uint32_t n;
    MacSeg s[NS];
};
using MacSegs = MacSegsT<kMaxSegs>;  // multi-layer launches
using MacSegs1 = MacSegsT<1>;        // one layer: a small kernel-parameter block
struct MacLayer {
    const uint64_t *x;
    const uint64_t *w;
    uint64_t *y;
    uint32_t G, B, M;
    uint32_t Lc = 0, limb0 = 0;  // limbs [limb0, limb0 + Lc) only (Lc = 0: all)
};
bool mac_conv_fits(uint32_t G, uint32_t B);
// tensor-core MAC of one layer, limbs [limb0, limb0 + Lc) (Lc = 0: all): shapes with
// G <= 8 and 2B <= 8 (mac_tc_fits)
bool mac_tc_fits(uint32_t G, uint32_t B);
hc_status launch_mac_tc(const hc_ctx *ctx, const uint64_t *x, const uint64_t *w, uint64_t *y, uint32_t G, uint32_t B,
                        uint32_t M, uint32_t limb0, uint32_t Lc, cudaStream_t s);
// MAC task geometry of one layer (channels per stage from the context's variant)
// (kc = 0: the chunk width of the context's variant; 32 or 64 forces it; waves:
// CTAs for about that many waves of the layer's work over all limbs)
MacSeg make_mac_seg(const hc_ctx *ctx, const uint64_t *x, const uint64_t *w, uint64_t *y, uint32_t G, uint32_t B,
                    uint32_t M, uint32_t kc = 0, uint32_t waves = 4);
size_t mac_seg_smem(const MacSeg &sg);
// blocked MACs of n layers (layer i on ctxs[i]) in ceil(n / kMaxSegs) launches
hc_status launch_mac_conv_layers(const hc_ctx *const *ctxs, const MacLayer *layers, size_t n, cudaStream_t s);

void plan_destroy(hc_plan *p);
hc_status launch_wait_selftest(const hc_ctx *ctx, uint32_t limit, cudaStream_t s);
void server_destroy(hc_server *s);

// one conv layer of a batched launch sequence
struct ConvJob {
    const hc_ctx *ctx;
    const hc_weights *w;
    const uint64_t *in;   // [I][2][L][N] coefficient domain
    uint64_t *out;        // [O][2][L][N] coefficient domain
    uint64_t *ntt;        // scratch: NTT-domain inputs [I][2][L][N]
    bool blocked;         // blocked MAC fits (else fused MAC + inverse NTT)
    const uint64_t *wpt = nullptr;  // NTT-domain weights [P][L][N]; nullptr: the resident ones
    const ExtractArgs *ex = nullptr;  // set: out is the NTT-domain MAC result and the inverse
                                      // transform is the server step's epilogue (limb chains only)
};
inline const uint64_t *job_weights(const ConvJob &c) { return c.wpt ? c.wpt : c.w->d_pt; }
bool conv_job_blocked(const hc_ctx *c, const hc_weights *w);
// launch form 2 for the blocked jobs of one degree: one forward -> MAC -> inverse
// chain per limb on parallel streams, joined back into s
hc_status launch_limb_chains(const ConvJob *jobs, size_t n, uint32_t logN, cudaStream_t s);
// The batched launch sequence of n conv jobs in stream order on s.  Per ring
// degree, when the first job's context selects the fused form (KK_CONV) and
// ctr holds enough words (conv_jobs_counter_words): one persistent fused
// launch; otherwise forward NTTs (one launch per degree), MACs (one launch),
// inverse NTTs (one launch per degree), at most kMaxSegs jobs per launch.
hc_status launch_conv_jobs(const ConvJob *jobs, size_t n, cudaStream_t s, uint32_t *ctr = nullptr,
                           size_t ctr_words = 0);
// counter words the fused form of these jobs needs (the largest degree's)
size_t conv_jobs_counter_words(const ConvJob *jobs, size_t n);

// one conv layer of a fused persistent launch (see k_conv_fused)
struct FusedLayer {
    MacSeg mac;               // X = NTT-domain scratch, W, Y, limbs and the MAC task geometry
    const uint64_t *in;       // coefficient-domain inputs [I][2][L][N]
    uint32_t I, O;
    uint32_t t_fwd, t_mac, t_inv;  // first task of each phase (numbered over the whole launch)
    uint32_t c_fwd, c_mac;         // counter offsets: c_fwd + limb; c_mac + group * L + limb
};
template <int NS>
struct FusedLayersT {
    uint32_t n, total;             // layers, tasks
    FusedLayer s[NS];
};
constexpr int kFusedMaxLayers = 32;
// counter words a fused launch over these jobs needs (one degree), 0 if none
size_t fused_counter_words(const ConvJob *jobs, size_t n, uint32_t logN);
// one fused launch over the blocked jobs of degree 2^logN (at most kFusedMaxLayers);
// ctr: zero-initialised by this call on s
hc_status launch_conv_fused(const ConvJob *jobs, size_t n, uint32_t logN, uint32_t *ctr, cudaStream_t s);

// one standalone product of a mixed-degree batch (see k_product_mixed)
struct MixItem {
    const uint64_t *ct;       // [2][L][N] coefficient domain
    const uint64_t *pt;       // [L][N] NTT domain
    uint64_t *out;            // [2][L][N] coefficient domain
    const LimbConst *limbs;
    uint32_t L, logN;
};
// work unit code: item << 4 | limb << 1 | component
constexpr uint32_t mix_unit(uint32_t item, uint32_t limb, uint32_t comp) { return item << 4 | limb << 1 | comp; }
// components per unit at ring degree 2^logN (2: both in one unit, 1: one unit per component)
constexpr uint32_t mix_comps_per_unit(uint32_t logN) { return logN >= 14 ? 1 : 2; }
// persistent launch over n_units units (sorted by cost, most expensive first);
// *next must be 0 when the launch starts
hc_status launch_product_mixed(const MixItem *items, const uint32_t *units, uint32_t n_units, uint32_t *next,
                               cudaStream_t s);

// transform kinds that take a segment table (pseudo-kinds, variant of FWDCT / INVCT),
// and the inverse transform with the server step's output epilogue (variant of INV)
constexpr int KK_FWDCT_SEGS = 100, KK_INVCT_SEGS = 101, KK_INV_EXTRACT = 102;


// arguments of one launch of a kernel family (unused fields ignored)
struct LaunchArgs {
    const NttSegs *segs;
    const uint64_t *in;
    uint64_t *out;
    const uint64_t *pt;
    MacTerms terms;
    const uint32_t *out_index;
    size_t n;
    bool accumulate;
    const ExtractArgs *ex;
};
template <int LOGN>
hc_status launch_n(const hc_ctx *ctx, int kind, int variant, const LaunchArgs &a, cudaStream_t s);

// default launch variant of a kernel family at ring degree 2^logn
int default_variant(int kind, uint32_t logn);

// in-place / out-of-place forward NTT of n_polys polys [n][L][N] (canonical in, canonical out)
hc_status launch_ntt_fwd(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_polys,
                         cudaStream_t s);
hc_status launch_ntt_inv(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_polys,
                         cudaStream_t s);
// inverse NTT of n_ct ciphertexts [n][2][L][N] (canonical NTT domain in, coefficients out)
hc_status launch_ntt_inv_ct(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_ct, cudaStream_t s);
// multi-segment forward / inverse transforms of ciphertexts (all segments share
// ctx's N and launch variant; n_groups counts ciphertexts)
hc_status launch_ntt_ct_segs(const hc_ctx *ctx, const NttSegs &segs, bool inverse, cudaStream_t s);
// conv MAC blocked over coefficient chunks: Y[m*B+b] = sum_g W[m*G+g] . X[g*B+b] (NTT domain)
hc_status launch_mac_conv(const hc_ctx *ctx, const uint64_t *x_ntt, const uint64_t *w_ntt, uint64_t *y,
                          uint32_t G, uint32_t B, uint32_t M, cudaStream_t s);
// forward NTT of n_ct ciphertexts [n][2][L][N] into out (both components per CTA)
hc_status launch_ntt_fwd_ct(const hc_ctx *ctx, const uint64_t *in, uint64_t *out, size_t n_ct,
                            cudaStream_t s);
// out[o] = INTT(sum_t ct_ntt[terms.ct] . pt_ntt[terms.pt]) for o < n_out
hc_status launch_mac_intt(const hc_ctx *ctx, const uint64_t *ct_ntt, const uint64_t *pt_ntt,
                          MacTerms terms, uint64_t *out, size_t n_out, cudaStream_t s);
// out[j] (+)= INTT(NTT(ct[j]) . pt_ntt[j]) for j < n (standalone products)
hc_status launch_product(const hc_ctx *ctx, const uint64_t *ct, const uint64_t *pt_ntt,
                         const uint32_t *out_index, uint64_t *out, size_t n, bool accumulate,
                         cudaStream_t s);
// weights: lift int8 packed polys [P][N] to [P][L][N] residues
hc_status launch_lift_int8(const hc_ctx *ctx, const int8_t *packed, uint64_t *out, size_t n_polys,
                           cudaStream_t s);
// checked mode: set *flag if any of count residues of [n][L][N] is >= its q
hc_status launch_range_check(const hc_ctx *ctx, const uint64_t *p, size_t n_polys, int *flag,
                             cudaStream_t s);

// one convolution layer on the device (Sec. 6.2): NTT of the inputs into
// scratch ([I][2][L][N]), NTT-domain MAC into d_out, inverse NTT of d_out in
// place; falls back to the fused MAC + inverse NTT kernel for layers whose
// input chunk does not fit the blocked MAC's shared memory
hc_status conv_layer(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_in, uint64_t *d_out,
                     uint64_t *scratch, size_t scratch_words, cudaStream_t s, const uint64_t *wpt = nullptr);
// one layer in the weights' preprocessing mode (offline NTT, online NTT, no NTT)
hc_status conv_any(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_in, uint64_t *d_out, cudaStream_t s);
hc_status launch_conv_direct(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_in, uint64_t *d_out,
                             cudaStream_t s);
// scratch words conv_layer uses at most (NTT-domain inputs + fused-form counters)
size_t conv_scratch_words(const hc_ctx *ctx, const hc_weights *w);
// an upper bound of the fused form's counter words for one layer (any MAC variant)
size_t conv_counter_bound(const hc_ctx *ctx, const hc_weights *w);

// checked mode only: HC_ERR_RANGE if a residue is >= its q_i (synchronises s); HC_OK otherwise
hc_status check_inputs(const hc_ctx *ctx, const uint64_t *p, size_t n_polys, cudaStream_t s);

}  // namespace hc
