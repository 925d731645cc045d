// hc_io.cu -- checkpoint and resume of preprocessed weights.  The paper's
// server preprocesses its weights once and reuses them until the model changes
// (Sec. 8.1); saving the NTT-domain plaintexts lets a restarted server resume
// without repacking and re-transforming them.
//
// File layout (little-endian): the 8-byte tag "HCWTS002"; a header of u32 N,
// L, mode, kind, No, G, B, I, P, O; the 11 u32 of the caller's hc_conv_desc
// (any stride; a fully connected layer as its 1x1 convolution) with the
// resolved partition; u64 t and the L moduli; u64 sizes of the four payloads
// (NTT-domain plaintexts, int8 kernel of the stride-1 layer, term pointers,
// terms); the payloads; a u64 FNV-1a hash of every byte before it.  Loading
// derives the layer's geometry from the descriptor again and refuses a file
// whose counts disagree with it.
#include <cstdio>
#include <cstring>
#include <vector>

#include "hc_internal.h"

using namespace hc;

namespace {

constexpr char kTag[8] = {'H', 'C', 'W', 'T', 'S', '0', '0', '2'};

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n)
    {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
};

struct Writer {
    FILE *f;
    Fnv fnv;
    bool ok = true;
    void put(const void *p, size_t n)
    {
        if (!n || !ok) return;
        ok = fwrite(p, 1, n, f) == n;
        fnv.add(p, n);
    }
};

struct Reader {
    FILE *f;
    Fnv fnv;
    bool ok = true;
    void get(void *p, size_t n)
    {
        if (!n || !ok) return;
        ok = fread(p, 1, n, f) == n;
        if (ok) fnv.add(p, n);
    }
};

size_t k_bytes_of(const hc_weights *w)
{
    return w->mode == HC_WEIGHTS_NO_NTT ? (size_t)w->desc.M * w->desc.C * w->desc.kh * w->desc.kw : 0;
}

}  // namespace

extern "C" {

hc_status hc_weights_save(const hc_weights *w, const char *path)
{
    if (!w || w->magic != kMagicWeights || !path) return set_error(HC_ERR_INVALID_ARG, "invalid weights or path");
    const hc_ctx *c = w->ctx;
    DeviceGuard g(w->device);
    const size_t pt_words = w->d_pt ? (size_t)w->P * c->L * c->N : 0;
    const size_t kb = k_bytes_of(w);
    const size_t n_tp = w->d_term_ptr ? (size_t)w->O + 1 : 0, n_t = w->d_terms ? (size_t)2 * w->O * w->G : 0;
    std::vector<uint64_t> pt(pt_words);
    std::vector<int8_t> kk(kb);
    std::vector<uint32_t> tp(n_tp), tm(n_t);
    cudaError_t e = cudaSuccess;
    if (pt_words) e = cudaMemcpy(pt.data(), w->d_pt, pt_words * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && kb) e = cudaMemcpy(kk.data(), w->d_k, kb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && n_tp) e = cudaMemcpy(tp.data(), w->d_term_ptr, n_tp * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && n_t) e = cudaMemcpy(tm.data(), w->d_terms, n_t * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "reading weights for saving");
    FILE *f = fopen(path, "wb");
    if (!f) return set_error(HC_ERR_INVALID_ARG, "cannot open %s for writing", path);
    Writer wr{f};
    wr.put(kTag, sizeof kTag);
    const uint32_t hdr[10] = {c->N, c->L, w->mode, w->kind, w->No, w->G, w->B, w->I, w->P, w->O};
    wr.put(hdr, sizeof hdr);
    wr.put(&w->user, sizeof(hc_conv_desc));
    wr.put(&c->t, sizeof c->t);
    wr.put(c->q, sizeof(uint64_t) * c->L);
    const uint64_t sizes[4] = {pt_words, kb, n_tp, n_t};
    wr.put(sizes, sizeof sizes);
    wr.put(pt.data(), pt_words * 8);
    wr.put(kk.data(), kb);
    wr.put(tp.data(), n_tp * 4);
    wr.put(tm.data(), n_t * 4);
    const uint64_t h = wr.fnv.h;
    if (wr.ok) wr.ok = fwrite(&h, 1, sizeof h, f) == sizeof h;
    const bool closed = fclose(f) == 0;
    if (!wr.ok || !closed) return set_error(HC_ERR_INVALID_ARG, "writing %s failed", path);
    return HC_OK;
}

hc_status hc_weights_load(const hc_ctx *ctx, const char *path, hc_weights **out)
{
    if (!out) return set_error(HC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx || ctx->magic != kMagicCtx || !path) return set_error(HC_ERR_INVALID_ARG, "invalid context or path");
    FILE *f = fopen(path, "rb");
    if (!f) return set_error(HC_ERR_INVALID_ARG, "cannot open %s", path);
    Reader rd{f};
    char tag[8];
    uint32_t hdr[10];
    hc_conv_desc user;
    uint64_t t = 0, q[kMaxLimbs] = {}, sizes[4] = {};
    rd.get(tag, sizeof tag);
    rd.get(hdr, sizeof hdr);
    rd.get(&user, sizeof user);
    rd.get(&t, sizeof t);
    const uint32_t L = hdr[1];
    bool ok = rd.ok && memcmp(tag, kTag, sizeof tag) == 0 && L >= 1 && L <= kMaxLimbs;
    if (ok) rd.get(q, sizeof(uint64_t) * L);
    if (ok) rd.get(sizes, sizeof sizes);
    ok = ok && rd.ok;
    if (!ok) {
        fclose(f);
        return set_error(HC_ERR_INVALID_ARG, "%s is not a saved weights file", path);
    }
    if (hdr[0] != ctx->N || L != ctx->L || t != ctx->t || memcmp(q, ctx->q, sizeof(uint64_t) * L) != 0) {
        fclose(f);
        return set_error(HC_ERR_INVALID_ARG, "%s was saved for other ring parameters", path);
    }
    const uint32_t mode = hdr[2], kind = hdr[3], No = hdr[4];
    LayerGeom lg{};
    if (mode > HC_WEIGHTS_NO_NTT || layer_geometry(user, kind, No, ctx->N, &lg) != HC_OK) {
        fclose(f);
        return set_error(HC_ERR_INVALID_ARG, "%s describes no valid layer", path);
    }
    const hc_conv_desc &desc = lg.eff;
    const size_t want_pt = mode == HC_WEIGHTS_NO_NTT ? 0 : (size_t)lg.P * ctx->L * ctx->N;
    const size_t want_k = mode == HC_WEIGHTS_NO_NTT ? (size_t)desc.M * desc.C * desc.kh * desc.kw : 0;
    if (sizes[0] != want_pt || sizes[1] != want_k ||
        (mode != HC_WEIGHTS_NO_NTT && (sizes[2] != (size_t)lg.O + 1 || sizes[3] != (size_t)2 * lg.O * lg.G)) ||
        hdr[5] != lg.G || hdr[6] != lg.B || hdr[7] != lg.I || hdr[8] != lg.P || hdr[9] != lg.O) {
        fclose(f);
        return set_error(HC_ERR_INVALID_ARG, "%s has inconsistent sizes", path);
    }
    std::vector<uint64_t> pt(sizes[0]);
    std::vector<int8_t> kk(sizes[1]);
    std::vector<uint32_t> tp(sizes[2]), tm(sizes[3]);
    rd.get(pt.data(), pt.size() * 8);
    rd.get(kk.data(), kk.size());
    rd.get(tp.data(), tp.size() * 4);
    rd.get(tm.data(), tm.size() * 4);
    uint64_t h = 0;
    const uint64_t want_h = rd.fnv.h;
    const bool read_ok = rd.ok && fread(&h, 1, sizeof h, f) == sizeof h;
    fclose(f);
    if (!read_ok || h != want_h) return set_error(HC_ERR_INVALID_ARG, "%s is truncated or corrupt", path);

    DeviceGuard g(ctx->device);
    hc_weights *w = new (std::nothrow) hc_weights();
    if (!w) return set_error(HC_ERR_OOM, "host allocation failed");
    w->magic = kMagicWeights;
    w->ctx = ctx;
    w->device = ctx->device;
    w->desc = desc;
    w->user = user;
    w->kind = kind;
    w->No = lg.No;
    w->Mp = lg.Mp;
    w->pa = lg.pa;
    w->pb = lg.pb;
    w->G = lg.G;
    w->B = lg.B;
    w->I = lg.I;
    w->P = lg.P;
    w->O = lg.O;
    w->mode = mode;
    auto up = [&](void **dst, const void *src, size_t bytes) -> bool {
        if (!bytes) return true;
        *dst = dev_alloc_persistent(bytes);
        return *dst && cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (!up((void **)&w->d_pt, pt.data(), pt.size() * 8) || !up((void **)&w->d_k, kk.data(), kk.size()) ||
        !up((void **)&w->d_term_ptr, tp.data(), tp.size() * 4) || !up((void **)&w->d_terms, tm.data(), tm.size() * 4)) {
        cudaGetLastError();
        hc_free(w);
        return set_error(HC_ERR_OOM, "uploading loaded weights failed");
    }
    const hc_status st = build_slot_table(w);
    if (st != HC_OK) {
        hc_free(w);
        return st;
    }
    *out = w;
    return HC_OK;
}

}  // extern "C"
