/*
 * hconv.h -- C ABI of the GB300 (sm_103a) library for the homomorphic
 * convolution hot path of SecONNds (arXiv 2506.11586): RLWE ciphertext x
 * plaintext polynomial products computed as forward NTT -> NTT-domain
 * multiply-accumulate -> inverse NTT over RNS limbs (Sec. 6.2, App. C.1).
 *
 * Conventions shared by every call
 *   - Status: every call returns hc_status (HC_OK == 0); none aborts, throws
 *     or exits.  hc_last_error() returns a thread-local detail string for the
 *     most recent failing call on the calling thread.
 *   - Pointers prefixed d_ are device memory, h_ are host memory.  Buffers
 *     passed in are owned by the caller; handles (hc_ctx, hc_weights,
 *     hc_plan) are owned by the library and released only by hc_free().
 *   - Layout: little-endian uint64 residues, [item][component][limb][coeff];
 *     a ciphertext is [2][L][N] (components c0, c1), a plaintext [L][N].
 *     Coefficient-domain arrays are in natural order.  NTT-domain arrays hold
 *     slot k = a(psi_i^(2*rev(k)+1)) mod q_i, where rev reverses log2(N) bits
 *     and psi_i is the smallest primitive 2N-th root of unity mod q_i.
 *   - Ranges: inputs must be canonical residues in [0, q_i); outputs are
 *     canonical.  Inputs are not range-checked unless the context was created
 *     with HC_CTX_CHECKED, in which case an out-of-range input makes the call
 *     return HC_ERR_RANGE (the call then also synchronises the stream).
 *   - Asynchrony: compute calls are enqueued on the given cudaStream_t
 *     (passed as void*, NULL = legacy default stream) and return before the
 *     GPU finishes; launch errors are reported by the call, execution errors
 *     by a later call or by stream synchronisation.
 *   - Supported parameters: N in {4096, 8192, 16384}; 1 <= L <= 8 distinct
 *     primes 2^32 < q_i < 2^50 with q_i = 1 (mod 2N).
 *   - A context is immutable after creation and may be used from several
 *     streams and host threads at once; weights likewise.  A plan is not
 *     thread-safe: run one plan on one stream at a time.
 */
#ifndef HCONV_H
#define HCONV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hc_ctx hc_ctx;
typedef struct hc_weights hc_weights;
typedef struct hc_plan hc_plan;

typedef enum {
    HC_OK = 0,
    HC_ERR_INVALID_ARG = 1,  /* null pointer, zero/oversized count, bad shape */
    HC_ERR_BAD_MODULUS = 2,  /* not prime, outside (2^32, 2^50), != 1 mod 2N, duplicate */
    HC_ERR_RANGE = 3,        /* checked mode: an input residue >= q_i */
    HC_ERR_OOM = 4,          /* device or host allocation failed */
    HC_ERR_BUDGET = 5,       /* admission: request exceeds the memory budget */
    HC_ERR_TIMEOUT = 6,      /* a bounded device-side wait expired */
    HC_ERR_CUDA = 7,         /* a CUDA runtime call failed (see hc_last_error) */
    HC_ERR_UNSUPPORTED = 8   /* valid but not supported for these arguments (e.g. a plan with online weights) */
} hc_status;

/* Context flags. */
#define HC_CTX_CHECKED 1u    /* range-check every input residue (debug mode) */

/* ---------------------------------------------------------------- context --
 * The RLWE ring R_Q = Z_Q[X]/(X^N+1) with Q = prod q_i in RNS form
 * (Sec. 2.1, App. C), plus the plaintext modulus t (informational; the
 * server-side hot path never reduces mod t).
 *
 * hc_ctx_create: validates (N, moduli[0..L), t) on the host, then builds and
 * uploads per-limb twiddle tables (psi^rev(k), psi^-rev(k) with Shoup
 * companions) and constants.  moduli is a host array, copied.  *out receives
 * a new handle; on failure *out is set to NULL.
 * Errors: HC_ERR_INVALID_ARG (null out/moduli, N unsupported, L == 0 or > 8,
 * t < 2), HC_ERR_BAD_MODULUS, HC_ERR_OOM, HC_ERR_CUDA. */
hc_status hc_ctx_create(uint32_t N, const uint64_t *moduli, uint32_t L, uint64_t t,
                        hc_ctx **out);
hc_status hc_ctx_create_ex(uint32_t N, const uint64_t *moduli, uint32_t L, uint64_t t,
                           uint32_t flags, hc_ctx **out);

/* Host-only validation of hc_ctx_create's arguments; touches no GPU. */
hc_status hc_ctx_validate(uint32_t N, const uint64_t *moduli, uint32_t L, uint64_t t);

/* Ring parameters of a context.  Any output pointer may be NULL; moduli_out
 * and psi_out (host arrays of L entries) receive q_i and the psi_i used. */
hc_status hc_ctx_info(const hc_ctx *ctx, uint32_t *N, uint32_t *L, uint64_t *t,
                      uint64_t *moduli_out, uint64_t *psi_out);

/* Self-test of device-side failure detection (no counterpart in the paper).
 * Launches one CTA that waits on an mbarrier nothing arrives at, with the
 * same bounded wait the pipelined kernels use but at most `limit` (1..2^20)
 * attempts; the wait runs out, the CTA records a timeout in the context's
 * device flag and exits, leaving the device usable.  A following
 * hc_ctx_device_status returns HC_ERR_TIMEOUT (and clears the flag).
 * Errors: HC_ERR_INVALID_ARG, HC_ERR_CUDA. */
hc_status hc_selftest_wait_timeout(const hc_ctx *ctx, uint32_t limit, void *cuda_stream);

/* Launch-shape tuning (no counterpart in the paper: a GPU scheduling knob).
 * Kernel families (kind): 0 forward NTT, 1 inverse NTT, 2 fused NTT-domain
 * MAC + inverse NTT, 3 fused standalone product, 4 forward NTT of whole
 * ciphertexts, 5 inverse NTT of whole ciphertexts, 6 blocked convolution MAC,
 * 7 convolution launch form.  variant (0..2) selects, for kinds 0-5, the radix
 * per register round, the polynomials per CTA and the CTAs per SM for the
 * context's N; variant 2 of the inverse kinds is a persistent kernel (TMA-fed
 * at N = 4096, prefetching into its exchange buffer at N >= 8192; with fewer
 * limbs than resident CTAs there, one cluster of two CTAs per limb) and
 * variant 2 of the forward kinds at N >= 8192 transforms each limb with a
 * cluster of two CTAs.  For kind 6 variants 0..2 select the weight rows per pipeline
 * stage (about 8, 16 or 32) of the integer MAC, and variant 3 the tensor-core MAC
 * (residues split into 8-bit limbs, exact f16 products summed in fp32 by
 * tcgen05 MMAs, recombined and reduced mod q; layers with G <= 8 channel groups
 * and 2B <= 8 rows per group, the others keep the integer MAC with 16-row
 * stages).  For kind 7: three launches per ring degree (forward NTTs,
 * MACs, inverse NTTs: variant 0), one persistent launch whose CTAs take the
 * layers' NTT, MAC and INTT tasks in order and wait on per-limb completion
 * counters (variant 1), or three launches per limb, the limbs' chains on
 * parallel streams (variant 2).  Every variant computes the same bits, only
 * speed differs.  hc_ctx_create picks defaults: variant 2 for kinds 0, 1, 4
 * and 5 at N >= 8192, variant 0 otherwise.
 * Changing a variant while other threads use the context is a data race.
 * Errors: HC_ERR_INVALID_ARG (bad handle, kind or variant: 0..3 for kind 6,
 * 0..2 otherwise). */
hc_status hc_ctx_set_variant(hc_ctx *ctx, uint32_t kind, uint32_t variant);
hc_status hc_ctx_get_variant(const hc_ctx *ctx, uint32_t kind, uint32_t *variant);

/* Device-side status of a context's kernels (no counterpart in the paper).
 * Kernels that wait on asynchronous copies bound every wait; a wait that runs
 * out records a flag in the context instead of hanging the GPU, and that
 * kernel's output is then unspecified.  hc_ctx_device_status synchronises
 * cuda_stream, reads and clears the flag, and returns HC_ERR_TIMEOUT if it was
 * set (HC_OK otherwise).  hc_conv_ct_pt_host performs this check itself. */
hc_status hc_ctx_device_status(const hc_ctx *ctx, void *cuda_stream);

/* -------------------------------------------------------------- transforms --
 * Negacyclic NTT over each RNS limb (App. C.1): the point-value form in which
 * the ring product becomes the slot-wise product (App. C.1).
 *
 * hc_ntt_fwd: in place on d_polys, n_polys polynomials of layout [n][L][N];
 * coefficient domain (natural order) in, NTT domain (order above) out.
 * hc_ntt_inv: the exact inverse, N^-1 folded in.
 * n_polys == 0 is a no-op.  Errors: HC_ERR_INVALID_ARG (null ctx, null
 * d_polys with n_polys > 0), HC_ERR_RANGE (checked mode), HC_ERR_CUDA. */
hc_status hc_ntt_fwd(const hc_ctx *ctx, uint64_t *d_polys, size_t n_polys, void *cuda_stream);
hc_status hc_ntt_inv(const hc_ctx *ctx, uint64_t *d_polys, size_t n_polys, void *cuda_stream);

/* ------------------------------------------------------------ convolution --
 * Cheetah-style coefficient-encoded convolution (Sec. 2.3, Sec. 6.1) with
 * weights NTT-preprocessed offline (Sec. 6.2, Sec. 7).  The paper prints no
 * packing; the library's packing of a stride-1 convolution with zero padding
 * `pad` is:
 *   channel groups of Cw, spatial blocks of Hw x Ww over the padded input,
 *   overlapping by kh-1 rows and kw-1 columns; G = ceil(C/Cw) groups,
 *   B = Bh*Bw blocks with Bh = ceil(Ho/(Hw-kh+1)), Bw = ceil(Wo/(Ww-kw+1));
 *   input ct  i = g*B + b : coeff [c*Hw*Ww + i*Ww + j] = x_pad[g*Cw+c][i0+i][j0+j]
 *   weight pt p = m*G + g : coeff [O - c*Hw*Ww - l*Ww - l'] = K[m][g*Cw+c][l][l']
 *                           (int8 lifted to w mod q_i), O = (Cw-1)HwWw + (kh-1)Ww + kw-1
 *   output ct o = m*B + b : coeff [O + i*Ww + j] encrypts y[m][i0+i][j0+j]
 *   with block b = bh*Bw + bw at padded origin (i0, j0) = (bh(Hw-kh+1), bw(Ww-kw+1)).
 * Cw = Hw = Ww = 0 in the descriptor selects the canonical partition: the
 * one minimising 2I + P + 2O polynomials moved (I = G*B inputs, P = M*G
 * weights, O = M*B outputs), ties to larger Hw*Ww, then larger Cw, then
 * larger Ww, over Cw <= C, kh <= Hw <= H+2pad, kw <= Ww <= W+2pad,
 * Cw*Hw*Ww <= N.
 *
 * Strided layers (the stride-2 convolutions of SqueezeNet-1.1 and ResNet-50,
 * Sec. 8.1).  A stride-s convolution with padding p is computed as the
 * stride-1 convolution without padding of the phase-split input
 *   x'[(a*pb + b)*C + c][i][j] = x_pad[c][s*i + a][s*j + b]   (0 past x_pad)
 * with kernel K'[m][(a*pb + b)*C + c][u][v] = K[m][c][s*u + a][s*v + b]
 * (0 past kh, kw), for phases a < pa = min(s, kh), b < pb = min(s, kw):
 * C' = pa*pb*C channels, kernel kh' = ceil(kh/s) x kw' = ceil(kw/s), input
 * H' = Ho + kh' - 1 by W' = Wo + kw' - 1 where Ho = (H + 2p - kh)/s + 1,
 * Wo = (W + 2p - kw)/s + 1 are the strided output sizes.  The library
 * splits K itself; the client packs x' (not x) with the stride-1 packing
 * above, using the descriptor hc_conv_partition returns.  Outputs are the
 * strided layer's Ho x Wo map.  An explicit Cw/Hw/Ww in a strided
 * descriptor is a partition of that stride-1 layer. */
typedef struct {
    uint32_t C, H, W;       /* input channels, height, width */
    uint32_t M;             /* output channels */
    uint32_t kh, kw;        /* kernel height, width */
    uint32_t stride, pad;   /* stride >= 1, zero padding on every side */
    uint32_t Cw, Hw, Ww;    /* 0,0,0 = canonical partition */
} hc_conv_desc;

/* Host-only: resolve the partition of `desc` for ring degree N.  *resolved
 * gets the stride-1 layer computed, with Cw/Hw/Ww filled in: desc itself for
 * stride 1, the phase-split layer above (stride 1, pad 0) otherwise; counts
 * may be NULL.  Errors: HC_ERR_INVALID_ARG (null desc/resolved, zero dims,
 * stride 0, kernel larger than the padded input, a given partition with
 * Cw*Hw*Ww > N). */
hc_status hc_conv_partition(const hc_conv_desc *desc, uint32_t N, hc_conv_desc *resolved,
                            uint32_t *n_in_ct, uint32_t *n_pt, uint32_t *n_out_ct);

/* Fully connected layers (ResNet-50's classifier, Sec. 8.1): y = W x with W
 * int8 [M][C], by matrix-vector coefficient packing.  With Cw inputs per input
 * polynomial and No output rows per output polynomial (No*Cw <= N):
 *   input ct  g = 0..G-1      : coeff [c] = x[g*Cw + c]            (G = ceil(C/Cw))
 *   weight pt p = m'*G + g    : coeff [r*Cw + Cw-1 - c] = W[m'*No + r][g*Cw + c]
 *   output ct m' = 0..Mp-1    : coeff [r*Cw + Cw-1] encrypts y[m'*No + r]   (Mp = ceil(M/No))
 * A product term lands at r*Cw + Cw-1 + (c_in - c) with |c_in - c| < Cw, so
 * rows never mix and no wrapped term reaches an output coefficient.  The
 * layer is the 1x1 convolution on a 1x1 image with partition (Cw, 1, 1) and
 * No output channels sharing an output ciphertext: every call that takes
 * weights takes FC weights too (I = G inputs, O = Mp outputs, [..][2][L][N]).
 * Cw = No = 0 selects the canonical partition: minimal 2I + P + 2O, then
 * fewer P, then larger Cw, then smaller No. */
typedef struct {
    uint32_t C, M;          /* inputs, outputs */
    uint32_t Cw, No;        /* 0,0 = canonical partition */
} hc_fc_desc;

/* Host-only: resolve the partition of a fully connected layer for ring
 * degree N (counts may be NULL).  Errors: HC_ERR_INVALID_ARG (null desc or
 * resolved, zero dims, a given partition with Cw > C, No > M or
 * Cw*No > N). */
hc_status hc_fc_partition(const hc_fc_desc *desc, uint32_t N, hc_fc_desc *resolved,
                          uint32_t *n_in_ct, uint32_t *n_pt, uint32_t *n_out_ct);

/* Offline weight preprocessing (Sec. 6.2, Sec. 8.1): pack h_K (host int8,
 * [M][C][kh][kw], copied) into P = M*G plaintext polynomials, lift to every
 * q_i, forward-NTT and keep them resident on the device in a new handle
 * (*out).  Enqueued on cuda_stream; the handle is usable by later calls on
 * any stream once that work completes (the call synchronises the stream
 * before returning, so it is immediately usable).
 * Errors: HC_ERR_INVALID_ARG, HC_ERR_OOM, HC_ERR_CUDA. */
hc_status hc_weights_preprocess(const hc_ctx *ctx, const hc_conv_desc *desc, const int8_t *h_K,
                                hc_weights **out, void *cuda_stream);

/* Output-channel shard of a convolution layer (no counterpart in the paper:
 * the layer's output channels are independent, so a layer splits across GPUs
 * by output channel, each GPU holding the weights of its channels and a copy
 * of the 2*I*L input limbs).  desc and h_K describe the WHOLE layer (M output
 * channels, h_K host int8 [M][C][kh][kw]); the handle holds channels
 * [m0, m1) only, under the whole layer's partition (desc's Cw, Hw, Ww, or the
 * canonical one when they are 0).  hc_conv_ct_pt with it, on the whole
 * layer's input ciphertexts, writes (m1 - m0)*B output ciphertexts equal bit
 * for bit to output ciphertexts [m0*B, m1*B) of the whole layer (B spatial
 * blocks, from hc_conv_geometry).  Stride-1 and strided convolutions.
 * Errors: as hc_weights_preprocess, and HC_ERR_INVALID_ARG unless
 * m0 < m1 <= M. */
hc_status hc_weights_preprocess_range(const hc_ctx *ctx, const hc_conv_desc *desc, const int8_t *h_K,
                                      uint32_t m0, uint32_t m1, hc_weights **out, void *cuda_stream);

/* NTT preprocessing modes (the paper's linear layers run "with online,
 * offline or no NTT preprocessing", Sec. 9; Sec. 6.2 describes the offline
 * one).  HC_WEIGHTS_NTT_OFFLINE (what hc_weights_preprocess does): packed,
 * lifted and NTT'd once, resident in the NTT domain.  HC_WEIGHTS_NTT_ONLINE:
 * packed and lifted, resident in the coefficient domain, NTT'd again by every
 * hc_conv_ct_pt call (P*L*N*8 more bytes of scratch per call).
 * HC_WEIGHTS_NO_NTT: the int8 kernel is kept as given and hc_conv_ct_pt
 * computes every output coefficient as a direct negacyclic product sum in the
 * coefficient domain (no transform at all).  All three give the same bits.
 * Plans, the server, hc_conv_ct_pt_plain and hc_weights_data/export take
 * offline weights only (online weights also export, in the coefficient
 * domain); hc_conv_ct_pt_noalloc takes offline and no-NTT weights; the others
 * return HC_ERR_UNSUPPORTED. */
typedef enum {
    HC_WEIGHTS_NTT_OFFLINE = 0,
    HC_WEIGHTS_NTT_ONLINE = 1,
    HC_WEIGHTS_NO_NTT = 2
} hc_weights_mode;
hc_status hc_weights_preprocess_ex(const hc_ctx *ctx, const hc_conv_desc *desc, const int8_t *h_K,
                                   uint32_t mode, hc_weights **out, void *cuda_stream);

/* Preprocessed weights of a fully connected layer: h_W host int8 [M][C]
 * (copied), mode as in hc_weights_preprocess_ex.  Errors: as
 * hc_weights_preprocess_ex. */
hc_status hc_weights_preprocess_fc(const hc_ctx *ctx, const hc_fc_desc *desc, const int8_t *h_W,
                                   uint32_t mode, hc_weights **out, void *cuda_stream);

/* Layout of preprocessed weights: *computed = the stride-1 layer computed
 * (with its partition; for FC weights the 1x1 convolution {C,1,1,M,1,1,1,0,
 * Cw,1,1}), *kind = 0 convolution / 1 fully connected, *No = output channels
 * per output ciphertext (1 for convolutions), *n_slots = output slots per
 * output ciphertext and limb of hc_conv_server_step,
 * No*(Hw-kh+1)*(Ww-kw+1) of *computed.  Any output pointer may be NULL. */
hc_status hc_weights_layout(const hc_weights *w, hc_conv_desc *computed, uint32_t *kind,
                            uint32_t *No, uint32_t *n_slots);

/* Geometry of preprocessed weights.  Any output pointer may be NULL. */
hc_status hc_conv_geometry(const hc_weights *w, uint32_t *n_in_ct, uint32_t *n_out_ct,
                           uint32_t *Cw, uint32_t *Hw, uint32_t *Ww);

/* Read-only view of the resident NTT-domain weights, [P][L][N] (p = m*G+g).
 * The pointer stays owned by the handle. */
hc_status hc_weights_data(const hc_weights *w, const uint64_t **d_pt_ntt, size_t *n_pt);

/* Copy the resident NTT-domain weights ([P][L][N]) into the caller's device
 * buffer d_dst (P*L*N words), enqueued on cuda_stream.  Lets a server save
 * preprocessed weights or inspect them.  Errors: HC_ERR_INVALID_ARG,
 * HC_ERR_CUDA. */
hc_status hc_weights_export(const hc_weights *w, uint64_t *d_dst, void *cuda_stream);

/* Online server computation of one convolution layer (Sec. 6.2): NTT every
 * input ciphertext, run all multiply-accumulates in the NTT domain, inverse
 * NTT only the final sums:
 *   d_ct_out[m*B+b] = INTT( sum_g NTT(d_ct_in[g*B+b]) . pt_ntt[m*G+g] )
 * for both components and every limb.  d_ct_in: [I][2][L][N] coefficient
 * domain (not modified); d_ct_out: [O][2][L][N] coefficient domain, fully
 * overwritten.  The buffers must not overlap.  Device scratch of
 * I*2*L*N*8 bytes is taken from the allocator (hc_set_allocator) on the
 * stream and returned after the work is enqueued.
 * Errors: HC_ERR_INVALID_ARG (null args, ctx/weights mismatch),
 * HC_ERR_RANGE (checked mode), HC_ERR_OOM, HC_ERR_CUDA. */
hc_status hc_conv_ct_pt(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_ct_in,
                        uint64_t *d_ct_out, void *cuda_stream);

/* The same result computed the plain way: one kernel launch per ct x pt
 * product (forward NTT of the ciphertext, slot-wise product, inverse NTT,
 * add into the output), no fusion and no batching.  Comparison path. */
hc_status hc_conv_ct_pt_plain(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_ct_in,
                              uint64_t *d_ct_out, void *cuda_stream);

/* hc_conv_ct_pt on HOST buffers: copies h_ct_in ([I][2][L][N]) to the
 * device, runs the layer, copies the result to h_ct_out ([O][2][L][N]) and
 * synchronises the stream before returning.  With offline weights the layer
 * runs in up to eight blocks of output channels and each block's outputs are
 * copied back on a second stream while the next block is computed.  Pinned
 * host memory gives the fastest copies (and the overlap); pageable memory
 * works.  Device buffers come from the allocator.  Errors as hc_conv_ct_pt. */
hc_status hc_conv_ct_pt_host(const hc_ctx *ctx, const hc_weights *w, const uint64_t *h_ct_in,
                             uint64_t *h_ct_out, void *cuda_stream);

/* hc_conv_ct_pt without any device allocation.  The paper has no counterpart:
 * this is a deployment variant for callers that must not allocate device
 * memory -- e.g. a service whose device memory is reserved up front by
 * another framework's caching allocator, or a latency-critical loop where
 * cudaMalloc / cudaFree would synchronise the device.  Same arguments, same
 * result, bit for bit, as hc_conv_ct_pt.  Its scratch (the NTT'd inputs,
 * I*2*L*N*8 bytes) lives in one static device array of 16 MiB that every GPU
 * loading the library keeps until the process exits; a larger layer is
 * rejected with HC_ERR_BUDGET.  The first call on a device looks up that
 * array's device address (once per device, with the context's device
 * current); make that first call before any stream capture.  All calls share
 * the one array: calls whose GPU work overlaps (other streams, other threads)
 * race on it and must be serialised by the caller.  Every scratch word read
 * is first written by the same call, so leftovers from earlier calls are
 * harmless.  Errors: as hc_conv_ct_pt, plus HC_ERR_BUDGET. */
hc_status hc_conv_ct_pt_noalloc(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_ct_in,
                                uint64_t *d_ct_out, void *cuda_stream);

/* The server's whole step of one linear layer (Sec. 7: the server adds its own
 * activation share to the client's ciphertexts, runs the convolution with the
 * NTT-preprocessed weights and applies a random mask; Sec. 6.2: the results
 * are sparse and only the output coefficients are returned).  With
 * Delta = floor(Q/t) (Q the product of the context's moduli, t its plaintext
 * modulus):
 *   1. c0 += Delta * pack(d_share), packed like the input ciphertexts
 *      (d_share: device [C][H][W] residues in [0, t) of the caller's layer --
 *      the library applies a strided layer's phase split itself; [C] for a
 *      fully connected layer -- or NULL to skip);
 *   2. d_ct_out = hc_conv_ct_pt of the result (full [O][2][L][N]; its c1
 *      components are what the client needs beside the slots);
 *   3. d_c0_slots[o][l][s] = c0[k] - Delta * r[m][row][col] mod q_l, where,
 *      with the stride-1 layer computed (hc_weights_layout) and oh = Hw-kh+1,
 *      ow = Ww-kw+1: output ct o = m'*B + b, slot s = (n*oh + i)*ow + j,
 *      k = n*Cw*Hw*Ww + offset + i*Ww + j, m = m'*No + n, (row, col) =
 *      (i0+i, j0+j); r = d_mask (device [M][Ho][Wo] in [0, t) -- [M] for a
 *      fully connected layer -- or NULL for r = 0); 0 for slots outside the
 *      Ho x Wo output map or with m >= M.  S = No*oh*ow slots per ciphertext
 *      and limb (convolutions: No = 1; FC: oh = ow = 1, slot n holds y[m'*No+n]).
 * The client decrypts slot s of output o from (d_c0_slots, c1 of d_ct_out) as
 * layer(x_c + x_s) - r mod t.  Share and mask values must lie in [0, t).
 * Device scratch of (2I)*2*L*N*8 bytes plus small counters comes from the
 * allocator.  Errors: as hc_conv_ct_pt. */
hc_status hc_conv_server_step(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_ct_in,
                              const uint64_t *d_share, const uint64_t *d_mask, uint64_t *d_ct_out,
                              uint64_t *d_c0_slots, void *cuda_stream);

/* The same step returning only what the client needs (Sec. 6.2: the results
 * are sparse and only the output coefficients go back; Sec. 7): d_c1_out
 * [O][L][N] gets the full c1 of every output ciphertext and d_c0_slots
 * [O][L][S] the masked output slots of c0, bit for bit what
 * hc_conv_server_step returns.  c0 is never stored in full: the inverse NTT
 * of the outputs writes the slots directly, so the layer's output writes drop
 * from O*2*L*N to O*L*(N + S) words.  Device scratch of (I + 2*O)*L*N*8*2
 * bytes (plus P*L*N*8 for online weights) comes from the allocator.
 * Errors: as hc_conv_server_step. */
hc_status hc_conv_server_step_sparse(const hc_ctx *ctx, const hc_weights *w, const uint64_t *d_ct_in,
                                     const uint64_t *d_share, const uint64_t *d_mask, uint64_t *d_c1_out,
                                     uint64_t *d_c0_slots, void *cuda_stream);

/* Checkpoint / resume of preprocessed weights (the paper's server keeps its
 * NTT-preprocessed weights until the model changes, Sec. 8.1).  hc_weights_save
 * writes w (any preprocessing mode) with its ring parameters and an integrity
 * hash to the file `path` (synchronous).  hc_weights_load reads it back for a
 * context with the same N, moduli and t and returns a handle that computes the
 * same bits as the saved one.  Errors: HC_ERR_INVALID_ARG (bad handle or path,
 * unreadable, truncated, corrupt or foreign file, other ring parameters),
 * HC_ERR_OOM, HC_ERR_CUDA. */
hc_status hc_weights_save(const hc_weights *w, const char *path);
hc_status hc_weights_load(const hc_ctx *ctx, const char *path, hc_weights **out);

/* --------------------------------------------------- generic ct x pt MAC --
 * The NTT-domain multiply-accumulate of Sec. 6.2 for arbitrary products:
 *   d_out[s] = sum_{j : h_slot[j] == s} INTT( NTT(d_ct[j]) . d_pt_ntt[j] )
 * for every s < n_out (slots with no product are set to zero).
 * d_ct: [n][2][L][N] coefficient domain; d_pt_ntt: [n][L][N] NTT domain;
 * h_slot: host array of n slot indices (< n_out); d_out: [n_out][2][L][N]
 * coefficient domain, fully overwritten, must not overlap the inputs.
 * Device scratch of n*2*L*N*8 bytes (only when some slot has more than one
 * product) plus a small work list come from the allocator.
 * Errors: HC_ERR_INVALID_ARG (null args, slot >= n_out), HC_ERR_RANGE
 * (checked mode), HC_ERR_OOM, HC_ERR_CUDA. */
hc_status hc_ctpt_mac(const hc_ctx *ctx, const uint64_t *d_ct, const uint64_t *d_pt_ntt,
                      const uint32_t *h_slot, size_t n, uint64_t *d_out, size_t n_out,
                      void *cuda_stream);

/* ------------------------------------------- Z_P layers: slot rotations --
 * SecONNds-P runs its linear layers with HELiKs' kernels over Z_P^N (Sec. 6.1):
 * each iteration multiplies the input ciphertext by an NTT-preprocessed weight
 * plaintext, accumulates, and rotates the accumulator by one SIMD slot;
 * rotations need key switching with public evaluation keys (Sec. 2.1).
 *
 * A rotation applies the Galois automorphism sigma_g (X -> X^g, g odd < 2N;
 * g = 5 rotates both slot rows of a BFV-SIMD plaintext left by one) and
 * switches the key back with one special prime p_sp and one digit per limb:
 *   d = sigma_g(c1), D_j = d mod q_j;  u = sum_j D_j * k_j over Q*p_sp;
 *   v = (u - [u]_{p_sp}) / p_sp over Q ([.] centered);  out = (sigma_g(c0) + v0, v1).
 * The Galois key k_j = (b_j, a_j), j < L, is made by the secret-key holder:
 *   b_j = -a_j s + e_j + p_sp * (Q/q_j) * [(Q/q_j)^-1]_{q_j} * sigma_g(s)  over Q*p_sp.
 *
 * hc_galois_key_create: h_key is host [L][2][L+1][N] coefficient-domain
 * residues (digit j: b_j then a_j, limbs q_0 .. q_{L-1}, p_sp), copied and
 * kept in the NTT domain.  special_prime must be a prime < 2^50, = 1 mod 2N,
 * distinct from the context's moduli (it gets a context of its own, L + 1 <=
 * 8).  Errors: HC_ERR_INVALID_ARG, HC_ERR_BAD_MODULUS, HC_ERR_OOM, HC_ERR_CUDA.
 * Freed by hc_free. */
typedef struct hc_galois_key hc_galois_key;
hc_status hc_galois_key_create(const hc_ctx *ctx, uint64_t special_prime, uint32_t galois_elt,
                               const uint64_t *h_key, hc_galois_key **out, void *cuda_stream);

/* Rotate n_ct ciphertexts d_ct_in [n][2][L][N] (coefficient domain, residues
 * < q_i) into d_ct_out (same layout, must not overlap the input).  Scratch of
 * n*(L+1)*(L+2)*N*8 bytes comes from the allocator.  Errors: HC_ERR_INVALID_ARG,
 * HC_ERR_RANGE (checked mode), HC_ERR_OOM, HC_ERR_CUDA. */
hc_status hc_ct_rotate(const hc_ctx *ctx, const hc_galois_key *key, const uint64_t *d_ct_in,
                       uint64_t *d_ct_out, size_t n_ct, void *cuda_stream);

/* The multiply-accumulate-rotate iteration: for the ciphertext d_ct [2][L][N]
 * and n NTT-domain plaintexts d_w_ntt [n][L][N] (hc_zp_plain_preprocess),
 *   acc = d_ct * w_{n-1};  for i = n-2 .. 0: acc = rotate(acc) + d_ct * w_i;
 * d_out [2][L][N] = acc (coefficient domain; must not overlap d_ct).  Decrypts
 * to sum_i rot^i(m * w_i) slot-wise mod P.  The n products run first, in one
 * launch; scratch of (n + 1) ciphertexts plus one rotation's comes from the
 * allocator.  Errors as hc_ct_rotate. */
hc_status hc_mac_rotate(const hc_ctx *ctx, const hc_galois_key *key, const uint64_t *d_ct,
                        const uint64_t *d_w_ntt, uint32_t n, uint64_t *d_out, void *cuda_stream);

/* The same iteration for m ciphertexts d_ct [m][2][L][N] that share the n
 * plaintexts (e.g. m client vectors through one matrix-vector layer), run in
 * lockstep: the m*n products in one launch, then n - 1 rotations of all m
 * accumulators at once.  d_out [m][2][L][N] (must not overlap d_ct); scratch
 * of (m*n + m) ciphertexts plus one rotation of m.  hc_mac_rotate is m = 1.
 * Errors as hc_ct_rotate. */
hc_status hc_mac_rotate_many(const hc_ctx *ctx, const hc_galois_key *key, const uint64_t *d_ct, uint32_t m,
                             const uint64_t *d_w_ntt, uint32_t n, uint64_t *d_out, void *cuda_stream);

/* Weight preprocessing for the iteration: n plaintext polynomials h_plain
 * [n][N] with coefficients in [0, P) (BFV-SIMD encoded by the caller), lifted
 * centered ((P-1)/2 < v -> v - P) into every q_i and forward-NTT'd into the
 * device buffer d_out [n][L][N]; synchronises the stream.  Errors:
 * HC_ERR_INVALID_ARG, HC_ERR_RANGE (a coefficient >= P), HC_ERR_CUDA. */
hc_status hc_zp_plain_preprocess(const hc_ctx *ctx, uint64_t P, const uint64_t *h_plain, size_t n,
                                 uint64_t *d_out, void *cuda_stream);

/* ------------------------------------- Z_P layers: SIMD encoding, matvec --
 * Plaintext vectors of SecONNds-P's linear layers live in Z_P^N (Sec. 6.1),
 * P a prime = 1 mod 2N, in the BFV batching layout: slot (r, c), r in {0, 1},
 * c < N/2, of a polynomial p is p(zeta^e) with e = 5^c (r = 0) or -5^c (r = 1)
 * mod 2N, zeta the smallest primitive 2N-th root mod P; sigma_5 (the Galois
 * element of hc_ct_rotate) rotates both rows left by one slot.
 *
 * ctx_p is a context with the single modulus P: hc_ctx_create(N, &P, 1, P, ...)
 * (so 2^32 < P < 2^50).
 *
 * hc_zp_encode: d_slots [n][2][N/2] values in [0, P) -> d_poly [n][N]
 * coefficients in [0, P) with those slots (scatter to the slots' NTT indices,
 * inverse NTT mod P).  hc_zp_decode: the inverse map.  Device buffers, must
 * not overlap; decoding takes n*N*8 bytes of scratch from the allocator.
 * Errors: HC_ERR_INVALID_ARG (not a one-modulus context, null or overlapping
 * buffers), HC_ERR_RANGE (checked mode, a value >= P), HC_ERR_OOM, HC_ERR_CUDA. */
hc_status hc_zp_encode(const hc_ctx *ctx_p, const uint64_t *d_slots, size_t n, uint64_t *d_poly,
                       void *cuda_stream);
hc_status hc_zp_decode(const hc_ctx *ctx_p, const uint64_t *d_poly, size_t n, uint64_t *d_slots,
                       void *cuda_stream);

/* Device-side form of hc_zp_plain_preprocess: d_poly [n][N] in [0, P) lifted
 * centered ((P-1)/2 < v -> v - P) into every q_i of ctx and forward-NTT'd
 * into d_out [n][L][N].  P must be odd and below every q_i.  Asynchronous.
 * Errors: HC_ERR_INVALID_ARG, HC_ERR_CUDA. */
hc_status hc_zp_lift_ntt(const hc_ctx *ctx, uint64_t P, const uint64_t *d_poly, size_t n, uint64_t *d_out,
                         void *cuda_stream);

/* Matrix-vector weights for hc_mac_rotate by the diagonal method (the
 * iterative multiply-accumulate-rotate kernel of HELiKs, Sec. 6.1).  h_W is
 * host [n_out][n_in] residues mod P = ctx_p's modulus.  With n the smallest
 * power of two >= max(n_out, n_in) (n <= N/2), a vector v of length n_in is
 * held periodically in both slot rows (slot (r, t) = v[t mod n], zero past
 * n_in); the n plaintexts w_i[r][t] = W[(t - i) mod n][t mod n] (W zero-padded
 * to n x n) are encoded on the device, lifted into ctx's q_i and NTT'd into
 * d_out [n][L][N] (out_words >= n*L*N); *n_terms = n.  hc_mac_rotate with
 * these n plaintexts then decrypts to W v, held the same way (slot (r, j) =
 * (W v)[j mod n]).  Synchronises the stream.  Errors: HC_ERR_INVALID_ARG
 * (different N, empty or too large matrix, d_out too small), HC_ERR_RANGE (an
 * entry >= P), HC_ERR_OOM, HC_ERR_CUDA. */
hc_status hc_zp_matvec_preprocess(const hc_ctx *ctx, const hc_ctx *ctx_p, const uint64_t *h_W, uint32_t n_out,
                                  uint32_t n_in, uint64_t *d_out, size_t out_words, uint32_t *n_terms,
                                  void *cuda_stream);

/* Convolution layers over Z_P (SecONNds-P runs its convolutions with HELiKs'
 * multiply-accumulate-rotate kernels over Z_P^N, Sec. 6.1 and Sec. 2.3; the
 * paper prints no packing, so this is the library's reading).  A stride-1
 * convolution (desc: C, H, W, M, kh, kw, pad; stride 0 or 1; the partition
 * fields are ignored) with Hp*Wp <= N/2, Hp = H + 2 pad, Wp = W + 2 pad:
 *   input channel c is one ciphertext whose two slot rows both hold its
 *   zero-padded image, row-major from slot 0 (zeros after it);
 *   output ciphertext y < Y = ceil(M/2) holds output channel 2y + r in slot
 *   row r, output pixel (i, j) at slot i*Wp + j (i < Hp - kh + 1, j < Wp - kw
 *   + 1; the other slots hold no output);
 *   kernel offset i = l*kw + l' is a rotation by delta_i = l*Wp + l' slots, and
 *   w_{y,i,c} is the plaintext whose slot row r is the constant
 *   K[2y + r][c][l][l'] (0 past M).  The layer runs the iteration
 *     P_i = sum_c x_c * w_{y,i,c};  acc = P_{kk-1};
 *     acc = rot^(delta_{i+1} - delta_i)(acc) + P_i,  i = kk-2 .. 0,
 *   which decrypts at slot (r, i*Wp + j) to conv(x, K)[2y + r][i][j] mod P.
 *
 * hc_zp_conv_preprocess: h_K host [M][C][kh][kw] residues mod P = ctx_p's
 * modulus; builds the Y*kh*kw*C weight plaintexts on the device (slot
 * vectors, SIMD encoding, centered lift into ctx's q_i, NTT) into d_out
 * [Y][kh*kw][C][L][N] (out_words >= that), in chunks of 1024 plaintexts of
 * allocator scratch.  Synchronises the stream.  Errors: HC_ERR_INVALID_ARG
 * (bad contexts, P not below every q_i, different N, image too large,
 * d_out too small), HC_ERR_UNSUPPORTED (stride > 1), HC_ERR_RANGE (an
 * entry >= P), HC_ERR_OOM, HC_ERR_CUDA.
 *
 * hc_zp_conv: d_ct_in [C][2][L][N] and d_ct_out [Y][2][L][N] coefficient
 * domain (not overlapping); d_w_ntt from hc_zp_conv_preprocess for the same
 * desc; key_1 a Galois key of element 5 (a one-slot rotation; unused when
 * kw = 1, may be NULL then) and key_row one of element 5^(Wp - kw + 1) mod 2N
 * (unused when kh = 1), both made for ctx.  Rotations: Y*(kh*kw - 1).
 * Scratch of (C + Y*kh*kw)*2*L*N*8 bytes plus the rotations' comes from the
 * allocator.  Errors: HC_ERR_INVALID_ARG (bad arguments or keys),
 * HC_ERR_UNSUPPORTED, HC_ERR_RANGE (checked mode), HC_ERR_OOM, HC_ERR_CUDA. */
hc_status hc_zp_conv_preprocess(const hc_ctx *ctx, const hc_ctx *ctx_p, const hc_conv_desc *desc,
                                const uint64_t *h_K, uint64_t *d_out, size_t out_words, void *cuda_stream);
hc_status hc_zp_conv(const hc_ctx *ctx, const hc_conv_desc *desc, const hc_galois_key *key_1,
                     const hc_galois_key *key_row, const uint64_t *d_w_ntt, const uint64_t *d_ct_in,
                     uint64_t *d_ct_out, void *cuda_stream);

/* ------------------------------------------------------------------ plans --
 * Batching across layers, products and ring degrees (Sec. 6.2; the paper's
 * closing remarks on accelerating composite HE operations).  A plan binds a
 * list of independent work items to their buffers once, then runs them all
 * with as few launches as the work allows:
 *   - the forward NTTs of every conv item of one ring degree in one launch,
 *   - the NTT-domain MACs of every conv item in one launch (all degrees),
 *   - the inverse NTTs of every conv item of one ring degree in one launch,
 *   - every standalone product of every degree in one persistent launch
 *     whose CTAs pull (product, limb) units from a global counter.
 * (At most 48 conv items share one launch; more items take more launches.)
 * hc_plan_run captures that launch sequence into a CUDA graph the first time
 * and replays the graph afterwards.  Results are identical, bit for bit, to
 * running every item alone with hc_conv_ct_pt / hc_ctpt_mac.
 *
 * Items are independent: no item's output may overlap another item's input
 * or output.  An item's output may coincide exactly with its own input
 * (in place).  The plan keeps the pointers; buffers, contexts and weights
 * must outlive it.  A plan owns device scratch for the conv items' NTT'd
 * inputs (sum of I*2*L*N*8 bytes) and its work tables, allocated when it is
 * created. */
typedef enum {
    HC_WORK_CONV = 0,     /* one conv layer: weights, d_ct_in [I][2][L][N], d_ct_out [O][2][L][N] */
    HC_WORK_PRODUCTS = 1  /* n standalone products: d_ct_out[j] = INTT(NTT(d_ct_in[j]) . d_pt_ntt[j]) */
} hc_work_kind;

typedef struct {
    uint32_t kind;              /* hc_work_kind */
    const hc_ctx *ctx;
    const hc_weights *weights;  /* HC_WORK_CONV: preprocessed for ctx */
    const uint64_t *d_ct_in;    /* coefficient domain */
    const uint64_t *d_pt_ntt;   /* HC_WORK_PRODUCTS: [n][L][N] NTT domain */
    uint64_t *d_ct_out;         /* coefficient domain, fully overwritten */
    size_t n;                   /* HC_WORK_PRODUCTS: number of products */
} hc_work_item;

/* Build a plan over n items (copied).  All contexts must live on the device
 * that is current at the call.  Errors: HC_ERR_INVALID_ARG (null/invalid
 * handle or buffer, weights of another context, overlapping items, more than
 * 2^28 products), HC_ERR_OOM, HC_ERR_CUDA. */
hc_status hc_plan_create(const hc_work_item *items, size_t n, hc_plan **out);

/* Run the plan on cuda_stream (graph replay after the first run; while
 * hc_profile_enable is on, the launches are issued directly instead so that
 * they can be timed).  Checked contexts range-check every input first.
 * Errors: HC_ERR_RANGE (checked mode), HC_ERR_CUDA, HC_ERR_TIMEOUT (a
 * bounded device wait expired in an earlier launch). */
hc_status hc_plan_run(hc_plan *plan, void *cuda_stream);

/* The same results the plain way: one kernel launch per ct x pt product
 * (forward NTT, slot-wise product, inverse NTT, accumulate), no batching and
 * no graph.  Comparison path for the batched form. */
hc_status hc_plan_run_plain(hc_plan *plan, void *cuda_stream);

/* Pick the fastest launch variant of each kernel family the plan uses, per
 * context, by timing the plan itself (CUDA events on cuda_stream, median of
 * several runs), and set it in the contexts (hc_ctx_set_variant).  Variants
 * change speed only, never results.  cache_path (NULL = no cache) names a
 * text file of earlier choices keyed by GPU, N, L, moduli and a signature of
 * the plan's work (its layer shapes and product counts); cached choices are
 * applied without timing and new ones are appended.  The plan's outputs
 * hold unspecified values afterwards.  Errors: as hc_plan_run, plus
 * HC_ERR_INVALID_ARG (unreadable cache lines are ignored, not errors). */
hc_status hc_plan_autotune(hc_plan *plan, const char *cache_path, void *cuda_stream);

/* Work in a plan: total ct x pt products, algorithmic HBM bytes of one run
 * (8*N*L*(2I + P + 2O) per conv item, 8*N*L*5 per product: read the inputs
 * and weights once, write the outputs once) and the kernel launches of one
 * batched run.  Any out pointer may be NULL. */
hc_status hc_plan_info(const hc_plan *plan, uint64_t *n_products, uint64_t *alg_bytes, uint32_t *n_launches);

/* ---------------------------------------------------------------- serving --
 * The server side of the paper's linear layers as a request loop (Sec. 6.2:
 * the server holds NTT-preprocessed weights and answers each client
 * ciphertext with NTT -> MAC -> INTT).  Layers (context + resident weights)
 * are registered once; requests -- one layer applied to one client's input
 * ciphertexts -- arrive at any time from any host thread.
 *
 * Continuous batching: a scheduler thread admits queued requests in arrival
 * order as soon as their device buffers fit in the memory budget, and each
 * time one of the max_inflight stream slots is free it launches the oldest
 * admitted request together with the admitted requests of the same ring
 * degree after it (up to max_batch) as one batch: host->device copies of the
 * inputs, then the batched launch sequence of hc_plan_run over all the
 * batch's layers, then device->host copies of the outputs that have a host
 * buffer.  Batches on different streams overlap on the device; a batch of a
 * smaller ring degree (shorter requests) runs on a stream of higher CUDA
 * priority, so its thread blocks are scheduled ahead of those of larger
 * batches already in flight (flag HC_SERVER_EQUAL_PRIORITY turns this off).
 * A completion thread retires batches, returns their memory to the budget
 * and wakes waiters.  Each request's result is bit-identical to
 * hc_conv_ct_pt on the same layer and input, whatever else is in flight.
 * Every stream slot has its own device error word: a bounded device wait of
 * the batch that ran out completes the batch's requests with HC_ERR_TIMEOUT
 * (their results are then unspecified and not counted in the products).
 *
 * Device memory: one pool of budget_bytes is reserved at creation; a request
 * takes (2*I + O)*2*L*N*8 bytes (input, NTT scratch, output) from it while in
 * flight.  Requests that can never fit are refused at submission. */
typedef struct hc_server hc_server;

#define HC_SERVER_EQUAL_PRIORITY 1u  /* hc_server_config.flags: every batch at the same stream priority */

typedef struct {
    size_t budget_bytes;      /* device pool for in-flight requests (0 = 32 GiB) */
    uint32_t max_batch;       /* most requests per batch (0 = 64, at most 4096) */
    uint32_t max_inflight;    /* batches on the device at once, one stream slot each (0 = 4, at most 16) */
    uint32_t flags;           /* HC_SERVER_* bits */
    uint32_t selftest_wait_limit; /* self-test of the timeout path (0 = off): every batch also runs one
                                     bounded wait that nothing completes, of at most this many attempts
                                     (<= 2^20), so its requests complete with HC_ERR_TIMEOUT */
} hc_server_config;

typedef struct {
    hc_status status;         /* HC_OK, or the error that failed the request's batch */
    uint32_t batch_size;      /* requests in the batch that carried it */
    double queue_ms;          /* submission -> its batch was enqueued */
    double latency_ms;        /* submission -> result ready (retired by the completion thread) */
} hc_request_info;

typedef struct {
    uint64_t submitted, completed, refused, batches, products;
    uint64_t pool_bytes, bytes_in_use, peak_bytes_in_use;
    uint32_t max_batch_seen;
} hc_server_stats;

/* Reserve the pool (on the current device) and start the scheduler and
 * completion threads.  cfg may be NULL (defaults).  Errors:
 * HC_ERR_INVALID_ARG, HC_ERR_OOM, HC_ERR_CUDA. */
hc_status hc_server_create(const hc_server_config *cfg, hc_server **out);

/* Register a layer: ctx and weights (preprocessed for ctx, on the server's
 * device) must outlive the server.  *layer_id receives its index.  Errors:
 * HC_ERR_INVALID_ARG. */
hc_status hc_server_add_layer(hc_server *srv, const hc_ctx *ctx, const hc_weights *w, uint32_t *layer_id);

/* Queue a request and return at once with its ticket.  h_ct_in: host
 * [I][2][L][N] (pinned gives asynchronous copies), read during the request
 * and kept valid by the caller until it completes.  h_ct_out: host
 * [O][2][L][N] that receives the result, or NULL to keep the result in the
 * pool (hc_server_result) until hc_server_release.  Errors:
 * HC_ERR_INVALID_ARG (bad layer or buffer), HC_ERR_BUDGET (the request alone
 * exceeds the pool), HC_ERR_INVALID_ARG after hc_server_shutdown. */
hc_status hc_server_submit(hc_server *srv, uint32_t layer_id, const uint64_t *h_ct_in, uint64_t *h_ct_out,
                           uint64_t *ticket);

/* Block until the request is done (timeout_s < 0: no limit) and fill *info
 * (may be NULL).  Errors: HC_ERR_INVALID_ARG (unknown or released ticket),
 * HC_ERR_TIMEOUT (not done within timeout_s). */
hc_status hc_server_wait(hc_server *srv, uint64_t ticket, double timeout_s, hc_request_info *info);

/* Non-blocking: *done = 1 and *info filled if the request is done. */
hc_status hc_server_poll(hc_server *srv, uint64_t ticket, int *done, hc_request_info *info);

/* Device pointer of a done request's result [O][2][L][N] kept in the pool
 * (submitted with h_ct_out == NULL), valid until hc_server_release.  Errors:
 * HC_ERR_INVALID_ARG (unknown ticket, not done, or copied to the host). */
hc_status hc_server_result(hc_server *srv, uint64_t ticket, const uint64_t **d_ct_out);

/* Copy a done request's pool-resident result to host memory h_ct_out
 * ([O][2][L][N]); returns when the copy is complete.  Errors: as
 * hc_server_result, HC_ERR_CUDA. */
hc_status hc_server_fetch(hc_server *srv, uint64_t ticket, uint64_t *h_ct_out);

/* Forget a done request and return its result memory to the pool.  Every
 * ticket is released once.  Errors: HC_ERR_INVALID_ARG (unknown or not done). */
hc_status hc_server_release(hc_server *srv, uint64_t ticket);

hc_status hc_server_stats_get(hc_server *srv, hc_server_stats *out);

/* Stop accepting requests, finish everything queued, join the threads.
 * hc_free(server) does this too. */
hc_status hc_server_shutdown(hc_server *srv);

/* ------------------------------------------------------------- allocation --
 * Device memory used by the library: handles' resident tables and weights,
 * and per-call scratch.  alloc(bytes, stream, user) must return device memory
 * usable in stream order on `stream` (NULL on failure); free(ptr, stream,
 * user) releases it in stream order.  Passing alloc == NULL restores the
 * default (cudaMallocAsync / cudaFreeAsync on the stream's device pool).
 * Not thread-safe with respect to concurrent library calls: set it once at
 * start-up. */
typedef void *(*hc_alloc_fn)(size_t bytes, void *cuda_stream, void *user);
typedef void (*hc_free_fn)(void *ptr, void *cuda_stream, void *user);
void hc_set_allocator(hc_alloc_fn alloc, hc_free_fn free_fn, void *user);

/* ---------------------------------------------------------------- tracing --
 * Per-kernel device timing.  While enabled, every kernel launch the library
 * enqueues is bracketed by CUDA events recorded on the launch's own stream.
 * hc_profile_collect synchronises on the recorded events, then reports for
 * each kernel name its launch count and summed device time (ms) since the
 * last collect, and clears the record.  entries: caller array of cap
 * elements; *n_out receives the number of kernel names (which may exceed
 * cap; only cap are written).  Not for use inside CUDA-graph capture. */
typedef struct {
    char name[48];
    uint64_t launches;
    double total_ms;
} hc_kernel_time;
void hc_profile_enable(int on);
hc_status hc_profile_collect(hc_kernel_time *entries, size_t cap, size_t *n_out);

/* Integer-pipe throughput probe (no counterpart in the paper: the roofline of
 * the integer-bound kernels needs the multiply pipe's rate on the device at
 * hand).  Runs long independent chains of one arithmetic form on every SM of
 * ctx's device (eight chains per thread, 4 CTAs of 256 threads per SM), one
 * untimed launch then one timed with CUDA events on `cuda_stream`, and
 * synchronises.  form 0: lazy Shoup multiplications (the NTT butterfly's
 * product), 1: 32-bit multiply-adds, 2: 32x32->64-bit multiply-adds.
 * *ops_per_s receives operations per second, *ms the timed launch's duration,
 * *imad_eq_per_op the operation's cost in 32-bit multiply-adds (14, 1, 2).
 * Any output may be NULL.  A scratch buffer of one word per thread comes from
 * the allocator.  Errors: HC_ERR_INVALID_ARG (bad context, form > 2, iters
 * outside [1, 2^24]), HC_ERR_OOM, HC_ERR_CUDA. */
hc_status hc_probe_int_rate(const hc_ctx *ctx, uint32_t form, uint32_t iters, void *cuda_stream,
                            double *ops_per_s, double *ms, double *imad_eq_per_op);

/* Release a handle of any kind (context, weights, plan, server).  NULL is a no-op.
 * A handle must not be in use by queued GPU work when it is freed. */
void hc_free(void *handle);

const char *hc_status_str(hc_status s);
const char *hc_last_error(void);

/* Library version, for diagnostics. */
const char *hc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HCONV_H */
