"""Thin ctypes binding of libhconv's C ABI (include/hconv.h).

Every function here has the name of the C entry point it wraps and only
marshals arguments: device buffers are torch CUDA tensors (int64 or uint64,
contiguous; their bytes are the uint64 residues), host buffers are numpy
arrays or pinned CPU tensors, streams are torch.cuda.Stream objects (None =
torch's current stream).  Every step of the computation runs in libhconv's
kernels; there is no Python or CPU fallback.  A non-OK status raises HcError.

The library must have been built (``paper_2506_11586_gb300.build.build()``);
if it is missing, loading fails loudly.
"""
import ctypes as C
import os

import numpy as np

from .build import LIB

HC_OK = 0
HC_ERR_INVALID_ARG = 1
HC_ERR_BAD_MODULUS = 2
HC_ERR_RANGE = 3
HC_ERR_OOM = 4
HC_ERR_BUDGET = 5
HC_ERR_TIMEOUT = 6
HC_ERR_CUDA = 7
HC_ERR_UNSUPPORTED = 8
HC_CTX_CHECKED = 1

STATUS_NAMES = {0: "HC_OK", 1: "HC_ERR_INVALID_ARG", 2: "HC_ERR_BAD_MODULUS", 3: "HC_ERR_RANGE",
                4: "HC_ERR_OOM", 5: "HC_ERR_BUDGET", 6: "HC_ERR_TIMEOUT", 7: "HC_ERR_CUDA",
                8: "HC_ERR_UNSUPPORTED"}


class HcError(RuntimeError):
    def __init__(self, status, detail):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), detail))


class hc_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_uint64), ("total_ms", C.c_double)]


class hc_conv_desc(C.Structure):
    _fields_ = [(n, C.c_uint32) for n in ("C", "H", "W", "M", "kh", "kw", "stride", "pad", "Cw", "Hw", "Ww")]


class hc_fc_desc(C.Structure):
    _fields_ = [(n, C.c_uint32) for n in ("C", "M", "Cw", "No")]


class hc_work_item(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("ctx", C.c_void_p), ("weights", C.c_void_p), ("d_ct_in", C.c_void_p),
                ("d_pt_ntt", C.c_void_p), ("d_ct_out", C.c_void_p), ("n", C.c_size_t)]


HC_WORK_CONV = 0
HC_WORK_PRODUCTS = 1


class hc_server_config(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("max_batch", C.c_uint32), ("max_inflight", C.c_uint32),
                ("flags", C.c_uint32), ("selftest_wait_limit", C.c_uint32)]


class hc_request_info(C.Structure):
    _fields_ = [("status", C.c_int), ("batch_size", C.c_uint32), ("queue_ms", C.c_double),
                ("latency_ms", C.c_double)]


class hc_server_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("submitted", "completed", "refused", "batches", "products",
                                          "pool_bytes", "bytes_in_use", "peak_bytes_in_use")] + \
               [("max_batch_seen", C.c_uint32)]

_lib = None

# name -> (restype, argtypes); mirrors include/hconv.h
_P = C.c_void_p
_SIGS = {
    "hc_ctx_create": (C.c_int, [C.c_uint32, _P, C.c_uint32, C.c_uint64, C.POINTER(_P)]),
    "hc_ctx_create_ex": (C.c_int, [C.c_uint32, _P, C.c_uint32, C.c_uint64, C.c_uint32, C.POINTER(_P)]),
    "hc_ctx_validate": (C.c_int, [C.c_uint32, _P, C.c_uint32, C.c_uint64]),
    "hc_ctx_device_status": (C.c_int, [_P, _P]),
    "hc_ctx_set_variant": (C.c_int, [_P, C.c_uint32, C.c_uint32]),
    "hc_selftest_wait_timeout": (C.c_int, [_P, C.c_uint32, _P]),
    "hc_ctx_get_variant": (C.c_int, [_P, C.c_uint32, C.POINTER(C.c_uint32)]),
    "hc_probe_int_rate": (C.c_int, [_P, C.c_uint32, C.c_uint32, _P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    "hc_ctx_info": (C.c_int, [_P, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint64), _P, _P]),
    "hc_ntt_fwd": (C.c_int, [_P, _P, C.c_size_t, _P]),
    "hc_ntt_inv": (C.c_int, [_P, _P, C.c_size_t, _P]),
    "hc_conv_partition": (C.c_int, [C.POINTER(hc_conv_desc), C.c_uint32, C.POINTER(hc_conv_desc),
                                    C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "hc_weights_preprocess": (C.c_int, [_P, C.POINTER(hc_conv_desc), _P, C.POINTER(_P), _P]),
    "hc_weights_preprocess_ex": (C.c_int, [_P, C.POINTER(hc_conv_desc), _P, C.c_uint32, C.POINTER(_P), _P]),
    "hc_weights_preprocess_range": (C.c_int, [_P, C.POINTER(hc_conv_desc), _P, C.c_uint32, C.c_uint32,
                                              C.POINTER(_P), _P]),
    "hc_fc_partition": (C.c_int, [C.POINTER(hc_fc_desc), C.c_uint32, C.POINTER(hc_fc_desc),
                                  C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "hc_weights_preprocess_fc": (C.c_int, [_P, C.POINTER(hc_fc_desc), _P, C.c_uint32, C.POINTER(_P), _P]),
    "hc_weights_layout": (C.c_int, [_P, C.POINTER(hc_conv_desc), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                    C.POINTER(C.c_uint32)]),
    "hc_conv_geometry": (C.c_int, [_P] + [C.POINTER(C.c_uint32)] * 5),
    "hc_weights_data": (C.c_int, [_P, C.POINTER(_P), C.POINTER(C.c_size_t)]),
    "hc_weights_export": (C.c_int, [_P, _P, _P]),
    "hc_weights_save": (C.c_int, [_P, C.c_char_p]),
    "hc_weights_load": (C.c_int, [_P, C.c_char_p, C.POINTER(_P)]),
    "hc_conv_ct_pt": (C.c_int, [_P, _P, _P, _P, _P]),
    "hc_conv_ct_pt_plain": (C.c_int, [_P, _P, _P, _P, _P]),
    "hc_conv_ct_pt_host": (C.c_int, [_P, _P, _P, _P, _P]),
    "hc_conv_ct_pt_noalloc": (C.c_int, [_P, _P, _P, _P, _P]),
    "hc_ctpt_mac": (C.c_int, [_P, _P, _P, _P, C.c_size_t, _P, C.c_size_t, _P]),
    "hc_galois_key_create": (C.c_int, [_P, C.c_uint64, C.c_uint32, _P, C.POINTER(_P), _P]),
    "hc_ct_rotate": (C.c_int, [_P, _P, _P, _P, C.c_size_t, _P]),
    "hc_mac_rotate": (C.c_int, [_P, _P, _P, _P, C.c_uint32, _P, _P]),
    "hc_mac_rotate_many": (C.c_int, [_P, _P, _P, C.c_uint32, _P, C.c_uint32, _P, _P]),
    "hc_zp_plain_preprocess": (C.c_int, [_P, C.c_uint64, _P, C.c_size_t, _P, _P]),
    "hc_zp_encode": (C.c_int, [_P, _P, C.c_size_t, _P, _P]),
    "hc_zp_decode": (C.c_int, [_P, _P, C.c_size_t, _P, _P]),
    "hc_zp_lift_ntt": (C.c_int, [_P, C.c_uint64, _P, C.c_size_t, _P, _P]),
    "hc_zp_matvec_preprocess": (C.c_int, [_P, _P, _P, C.c_uint32, C.c_uint32, _P, C.c_size_t,
                                          C.POINTER(C.c_uint32), _P]),
    "hc_zp_conv_preprocess": (C.c_int, [_P, _P, C.POINTER(hc_conv_desc), _P, _P, C.c_size_t, _P]),
    "hc_zp_conv": (C.c_int, [_P, C.POINTER(hc_conv_desc), _P, _P, _P, _P, _P, _P]),
    "hc_conv_server_step": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "hc_conv_server_step_sparse": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "hc_plan_create": (C.c_int, [_P, C.c_size_t, C.POINTER(_P)]),
    "hc_plan_run": (C.c_int, [_P, _P]),
    "hc_plan_run_plain": (C.c_int, [_P, _P]),
    "hc_plan_autotune": (C.c_int, [_P, C.c_char_p, _P]),
    "hc_plan_info": (C.c_int, [_P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]),
    "hc_server_create": (C.c_int, [C.POINTER(hc_server_config), C.POINTER(_P)]),
    "hc_server_add_layer": (C.c_int, [_P, _P, _P, C.POINTER(C.c_uint32)]),
    "hc_server_submit": (C.c_int, [_P, C.c_uint32, _P, _P, C.POINTER(C.c_uint64)]),
    "hc_server_wait": (C.c_int, [_P, C.c_uint64, C.c_double, C.POINTER(hc_request_info)]),
    "hc_server_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(C.c_int), C.POINTER(hc_request_info)]),
    "hc_server_result": (C.c_int, [_P, C.c_uint64, C.POINTER(_P)]),
    "hc_server_release": (C.c_int, [_P, C.c_uint64]),
    "hc_server_fetch": (C.c_int, [_P, C.c_uint64, _P]),
    "hc_server_stats_get": (C.c_int, [_P, C.POINTER(hc_server_stats)]),
    "hc_server_shutdown": (C.c_int, [_P]),
    "hc_set_allocator": (None, [_P, _P, _P]),
    "hc_profile_enable": (None, [C.c_int]),
    "hc_profile_collect": (C.c_int, [_P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "hc_free": (None, [_P]),
    "hc_status_str": (C.c_char_p, [C.c_int]),
    "hc_last_error": (C.c_char_p, []),
    "hc_version": (C.c_char_p, []),
}


def lib():
    """Load libhconv.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libhconv.so is not built (%s); run paper_2506_11586_gb300.build.build()" % LIB)
        L = C.CDLL(LIB)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != HC_OK:
        raise HcError(status, lib().hc_last_error().decode(errors="replace"))


def _dptr(t):
    """Device pointer of a contiguous CUDA tensor of 8-byte integers."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if t.element_size() != 8:
        raise ValueError("expected 8-byte integer elements (int64/uint64)")
    return C.c_void_p(t.data_ptr())


def _hptr(a):
    """Host pointer of a C-contiguous numpy array or CPU tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous array")
        return C.c_void_p(a.ctypes.data)
    if a.is_cuda or not a.is_contiguous():
        raise ValueError("expected a contiguous CPU tensor")
    return C.c_void_p(a.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class _Handle:
    """Owns a library handle; hc_free on close()/garbage collection."""

    def __init__(self, ptr, keep=None):
        self.ptr = ptr
        self._keep = keep

    def close(self):
        if self.ptr:
            lib().hc_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ctx(_Handle):
    def __init__(self, ptr, N, moduli, t):
        super().__init__(ptr)
        self.N, self.moduli, self.t = N, tuple(moduli), t
        self.L = len(moduli)


class Weights(_Handle):
    """Preprocessed weights.  desc: the caller's layer with its partition;
    computed: the stride-1 layer the library computes (hc_weights_layout);
    kind 0 convolution / 1 fully connected; No output channels per output
    ciphertext; n_slots server-step slots per output ciphertext and limb;
    products: ct x pt products of one call."""

    def __init__(self, ptr, ctx, resolved, I, O):
        super().__init__(ptr, keep=ctx)
        self.ctx, self.desc, self.I, self.O = ctx, resolved, I, O
        comp, kind, no, slots = hc_conv_desc(), C.c_uint32(), C.c_uint32(), C.c_uint32()
        _check(lib().hc_weights_layout(self.ptr, C.byref(comp), C.byref(kind), C.byref(no), C.byref(slots)))
        self.computed, self.kind, self.No, self.n_slots = comp, kind.value, no.value, slots.value
        self.products = -(-comp.M // self.No) * I


# ---------------------------------------------------------------- context ---

def hc_ctx_validate(N, moduli, t):
    """Host-only validation; returns the hc_status code (no exception)."""
    m = np.ascontiguousarray(moduli, dtype=np.uint64)
    return lib().hc_ctx_validate(N, C.c_void_p(m.ctypes.data), m.size, t)


def hc_ctx_create(N, moduli, t, flags=0):
    m = np.ascontiguousarray(moduli, dtype=np.uint64)
    out = C.c_void_p()
    _check(lib().hc_ctx_create_ex(N, C.c_void_p(m.ctypes.data), m.size, t, flags, C.byref(out)))
    return Ctx(out, N, [int(x) for x in m], t)


(KIND_NTT_FWD, KIND_NTT_INV, KIND_MAC_INTT, KIND_PRODUCT, KIND_NTT_FWD_CT, KIND_NTT_INV_CT, KIND_MAC_CONV,
 KIND_CONV_FORM) = range(8)
N_VARIANTS = 3


def hc_ctx_device_status(ctx, stream=None):
    """Synchronise the stream; raise HcError(HC_ERR_TIMEOUT) if a bounded device wait ran out."""
    _check(lib().hc_ctx_device_status(ctx.ptr, _stream(stream)))


def hc_selftest_wait_timeout(ctx, limit=256, stream=None):
    _check(lib().hc_selftest_wait_timeout(ctx.ptr, limit, _stream(stream)))


def hc_probe_int_rate(ctx, form, iters, stream=None):
    """(operations/s, ms, IMAD-equivalents per operation) of the integer-pipe probe."""
    r, ms, eq = C.c_double(), C.c_double(), C.c_double()
    _check(lib().hc_probe_int_rate(ctx.ptr, form, iters, _stream(stream), C.byref(r), C.byref(ms), C.byref(eq)))
    return r.value, ms.value, eq.value


def hc_ctx_set_variant(ctx, kind, variant):
    _check(lib().hc_ctx_set_variant(ctx.ptr, kind, variant))


def hc_ctx_get_variant(ctx, kind):
    v = C.c_uint32()
    _check(lib().hc_ctx_get_variant(ctx.ptr, kind, C.byref(v)))
    return v.value


def hc_ctx_info(ctx):
    N, L, t = C.c_uint32(), C.c_uint32(), C.c_uint64()
    q = np.zeros(8, dtype=np.uint64)
    psi = np.zeros(8, dtype=np.uint64)
    _check(lib().hc_ctx_info(ctx.ptr, C.byref(N), C.byref(L), C.byref(t), C.c_void_p(q.ctypes.data),
                             C.c_void_p(psi.ctypes.data)))
    n = L.value
    return {"N": N.value, "L": n, "t": t.value, "moduli": [int(x) for x in q[:n]],
            "psi": [int(x) for x in psi[:n]]}


# ------------------------------------------------------------- transforms ---

def _npolys(ctx, t):
    per = ctx.L * ctx.N
    if t.numel() % per:
        raise ValueError("tensor size is not a multiple of L*N")
    return t.numel() // per


def hc_ntt_fwd(ctx, polys, stream=None):
    _check(lib().hc_ntt_fwd(ctx.ptr, _dptr(polys), _npolys(ctx, polys), _stream(stream)))


def hc_ntt_inv(ctx, polys, stream=None):
    _check(lib().hc_ntt_inv(ctx.ptr, _dptr(polys), _npolys(ctx, polys), _stream(stream)))


# ------------------------------------------------------------ convolution ---

def make_desc(C_, H, W, M, kh, kw, pad=0, stride=1, Cw=0, Hw=0, Ww=0):
    return hc_conv_desc(C_, H, W, M, kh, kw, stride, pad, Cw, Hw, Ww)


def hc_conv_partition(desc, N):
    """Host-only: (resolved desc, n_in_ct, n_pt, n_out_ct)."""
    res = hc_conv_desc()
    i, p, o = C.c_uint32(), C.c_uint32(), C.c_uint32()
    _check(lib().hc_conv_partition(C.byref(desc), N, C.byref(res), C.byref(i), C.byref(p), C.byref(o)))
    return res, i.value, p.value, o.value


HC_WEIGHTS_NTT_OFFLINE, HC_WEIGHTS_NTT_ONLINE, HC_WEIGHTS_NO_NTT = 0, 1, 2


def hc_weights_preprocess(ctx, desc, K, stream=None):
    return hc_weights_preprocess_ex(ctx, desc, K, HC_WEIGHTS_NTT_OFFLINE, stream)


def hc_weights_preprocess_ex(ctx, desc, K, mode, stream=None):
    K = np.ascontiguousarray(K, dtype=np.int8)
    if K.size != desc.M * desc.C * desc.kh * desc.kw:
        raise ValueError("K must have M*C*kh*kw entries")
    out = C.c_void_p()
    _check(lib().hc_weights_preprocess_ex(ctx.ptr, C.byref(desc), C.c_void_p(K.ctypes.data), mode, C.byref(out),
                                          _stream(stream)))
    i, o, cw, hw, ww = (C.c_uint32() for _ in range(5))
    _check(lib().hc_conv_geometry(out, C.byref(i), C.byref(o), C.byref(cw), C.byref(hw), C.byref(ww)))
    res = hc_conv_desc(desc.C, desc.H, desc.W, desc.M, desc.kh, desc.kw, desc.stride, desc.pad,
                       cw.value, hw.value, ww.value)
    return Weights(out, ctx, res, i.value, o.value)


def hc_weights_preprocess_range(ctx, desc, K, m0, m1, stream=None):
    """Weights of output channels [m0, m1) of the whole layer desc (K: its whole int8 kernel),
    under the whole layer's partition."""
    K = np.ascontiguousarray(K, dtype=np.int8)
    if K.size != desc.M * desc.C * desc.kh * desc.kw:
        raise ValueError("K must have M*C*kh*kw entries")
    out = C.c_void_p()
    _check(lib().hc_weights_preprocess_range(ctx.ptr, C.byref(desc), C.c_void_p(K.ctypes.data), m0, m1,
                                             C.byref(out), _stream(stream)))
    i, o, cw, hw, ww = (C.c_uint32() for _ in range(5))
    _check(lib().hc_conv_geometry(out, C.byref(i), C.byref(o), C.byref(cw), C.byref(hw), C.byref(ww)))
    res = hc_conv_desc(desc.C, desc.H, desc.W, m1 - m0, desc.kh, desc.kw, desc.stride, desc.pad,
                       cw.value, hw.value, ww.value)
    return Weights(out, ctx, res, i.value, o.value)


def make_fc_desc(C_, M, Cw=0, No=0):
    return hc_fc_desc(C_, M, Cw, No)


def hc_fc_partition(desc, N):
    """Host-only: (resolved fc desc, n_in_ct, n_pt, n_out_ct)."""
    res = hc_fc_desc()
    i, p, o = C.c_uint32(), C.c_uint32(), C.c_uint32()
    _check(lib().hc_fc_partition(C.byref(desc), N, C.byref(res), C.byref(i), C.byref(p), C.byref(o)))
    return res, i.value, p.value, o.value


def hc_weights_preprocess_fc(ctx, desc, Wm, mode=HC_WEIGHTS_NTT_OFFLINE, stream=None):
    """Fully connected layer y = Wm x, Wm int8 [M][C]; the handle's desc is its 1x1 convolution form."""
    Wm = np.ascontiguousarray(Wm, dtype=np.int8)
    if Wm.size != desc.M * desc.C:
        raise ValueError("Wm must have M*C entries")
    out = C.c_void_p()
    _check(lib().hc_weights_preprocess_fc(ctx.ptr, C.byref(desc), C.c_void_p(Wm.ctypes.data), mode, C.byref(out),
                                          _stream(stream)))
    i, o, cw, hw, ww = (C.c_uint32() for _ in range(5))
    _check(lib().hc_conv_geometry(out, C.byref(i), C.byref(o), C.byref(cw), C.byref(hw), C.byref(ww)))
    res = hc_conv_desc(desc.C, 1, 1, desc.M, 1, 1, 1, 0, cw.value, 1, 1)
    return Weights(out, ctx, res, i.value, o.value)


def hc_conv_geometry(w):
    i, o, cw, hw, ww = (C.c_uint32() for _ in range(5))
    _check(lib().hc_conv_geometry(w.ptr, C.byref(i), C.byref(o), C.byref(cw), C.byref(hw), C.byref(ww)))
    return i.value, o.value, cw.value, hw.value, ww.value


def hc_weights_data(w):
    """(device pointer as int, number of plaintext polys) of the resident NTT-domain weights."""
    p, n = C.c_void_p(), C.c_size_t()
    _check(lib().hc_weights_data(w.ptr, C.byref(p), C.byref(n)))
    return p.value, n.value


def hc_weights_save(w, path):
    _check(lib().hc_weights_save(w.ptr, str(path).encode()))


def hc_weights_load(ctx, path, like_desc=None):
    """Load saved weights for ctx; returns a Weights handle (its desc from the file's geometry)."""
    out = C.c_void_p()
    _check(lib().hc_weights_load(ctx.ptr, str(path).encode(), C.byref(out)))
    i, o, cw, hw, ww = (C.c_uint32() for _ in range(5))
    _check(lib().hc_conv_geometry(out, C.byref(i), C.byref(o), C.byref(cw), C.byref(hw), C.byref(ww)))
    d = like_desc
    if d is None:
        comp = hc_conv_desc()
        _check(lib().hc_weights_layout(out, C.byref(comp), None, None, None))
        d = comp
    res = hc_conv_desc(d.C, d.H, d.W, d.M, d.kh, d.kw, d.stride, d.pad, cw.value, hw.value, ww.value)
    return Weights(out, ctx, res, i.value, o.value)


def hc_weights_export(w, dst, stream=None):
    """Copy the resident NTT-domain weights [P][L][N] into the CUDA tensor dst."""
    if dst.numel() != w.ctx.L * w.ctx.N * hc_weights_data(w)[1]:
        raise ValueError("dst must hold P*L*N words")
    _check(lib().hc_weights_export(w.ptr, _dptr(dst), _stream(stream)))


def hc_conv_ct_pt(ctx, w, ct_in, ct_out, stream=None):
    _check(lib().hc_conv_ct_pt(ctx.ptr, w.ptr, _dptr(ct_in), _dptr(ct_out), _stream(stream)))


def hc_conv_ct_pt_plain(ctx, w, ct_in, ct_out, stream=None):
    _check(lib().hc_conv_ct_pt_plain(ctx.ptr, w.ptr, _dptr(ct_in), _dptr(ct_out), _stream(stream)))


def hc_conv_ct_pt_noalloc(ctx, w, ct_in, ct_out, stream=None):
    """hc_conv_ct_pt with its scratch in the library's static device array (no allocation)."""
    _check(lib().hc_conv_ct_pt_noalloc(ctx.ptr, w.ptr, _dptr(ct_in), _dptr(ct_out), _stream(stream)))


def hc_conv_ct_pt_host(ctx, w, h_in, h_out, stream=None):
    _check(lib().hc_conv_ct_pt_host(ctx.ptr, w.ptr, _hptr(h_in), _hptr(h_out), _stream(stream)))


def slot_count(w):
    """Output slots per output ciphertext and limb of hc_conv_server_step: No*(Hw-kh+1)*(Ww-kw+1)
    of the stride-1 layer computed."""
    return w.n_slots


def hc_conv_server_step(ctx, w, ct_in, share, mask, ct_out, c0_slots, stream=None):
    """share: device [C][H][W] or None; mask: device [M][Ho][Wo] or None; c0_slots: [O][L][S]."""
    _check(lib().hc_conv_server_step(ctx.ptr, w.ptr, _dptr(ct_in), _dptr(share) if share is not None else None,
                                     _dptr(mask) if mask is not None else None, _dptr(ct_out), _dptr(c0_slots),
                                     _stream(stream)))


def hc_conv_server_step_sparse(ctx, w, ct_in, share, mask, c1_out, c0_slots, stream=None):
    """share: device [C][H][W] or None; mask: device [M][Ho][Wo] or None; c1_out: [O][L][N]; c0_slots: [O][L][S]."""
    _check(lib().hc_conv_server_step_sparse(ctx.ptr, w.ptr, _dptr(ct_in),
                                            _dptr(share) if share is not None else None,
                                            _dptr(mask) if mask is not None else None, _dptr(c1_out),
                                            _dptr(c0_slots), _stream(stream)))


def hc_ctpt_mac(ctx, ct, pt_ntt, slots, out, stream=None):
    sl = np.ascontiguousarray(slots, dtype=np.uint32)
    n_out = _npolys(ctx, out) // 2
    _check(lib().hc_ctpt_mac(ctx.ptr, _dptr(ct), _dptr(pt_ntt), C.c_void_p(sl.ctypes.data), sl.size,
                             _dptr(out), n_out, _stream(stream)))


class GaloisKey(_Handle):
    def __init__(self, ptr, ctx, special, g):
        super().__init__(ptr, keep=ctx)
        self.ctx, self.special, self.g = ctx, special, g


def hc_galois_key_create(ctx, special_prime, galois_elt, h_key, stream=None):
    """h_key: host [L][2][L+1][N] coefficient-domain residues (digit j: b_j, a_j)."""
    k = np.ascontiguousarray(h_key, dtype=np.uint64)
    if k.size != ctx.L * 2 * (ctx.L + 1) * ctx.N:
        raise ValueError("key must have L*2*(L+1)*N words")
    out = C.c_void_p()
    _check(lib().hc_galois_key_create(ctx.ptr, int(special_prime), galois_elt, C.c_void_p(k.ctypes.data),
                                      C.byref(out), _stream(stream)))
    return GaloisKey(out, ctx, int(special_prime), galois_elt)


def hc_ct_rotate(ctx, key, ct_in, ct_out, stream=None):
    n = _npolys(ctx, ct_in) // 2
    _check(lib().hc_ct_rotate(ctx.ptr, key.ptr, _dptr(ct_in), _dptr(ct_out), n, _stream(stream)))


def hc_mac_rotate(ctx, key, ct, w_ntt, out, stream=None):
    n = _npolys(ctx, w_ntt)
    _check(lib().hc_mac_rotate(ctx.ptr, key.ptr, _dptr(ct), _dptr(w_ntt), n, _dptr(out), _stream(stream)))


def hc_mac_rotate_many(ctx, key, cts, w_ntt, out, stream=None):
    """cts: device [m][2][L][N]; w_ntt: device [n][L][N] shared by all m; out: device [m][2][L][N]."""
    m = _npolys(ctx, cts) // 2
    n = _npolys(ctx, w_ntt)
    _check(lib().hc_mac_rotate_many(ctx.ptr, key.ptr, _dptr(cts), m, _dptr(w_ntt), n, _dptr(out), _stream(stream)))


def hc_zp_plain_preprocess(ctx, P, h_plain, out, stream=None):
    """h_plain: host [n][N] coefficients in [0, P); out: device [n][L][N]."""
    h = np.ascontiguousarray(h_plain, dtype=np.uint64)
    n = h.size // ctx.N
    _check(lib().hc_zp_plain_preprocess(ctx.ptr, int(P), C.c_void_p(h.ctypes.data), n, _dptr(out), _stream(stream)))


def hc_zp_encode(ctx_p, slots, poly, stream=None):
    """slots: device [n][2][N/2] values in [0, P); poly: device [n][N] (ctx_p: the one-modulus P context)."""
    n = _npolys(ctx_p, slots)
    _check(lib().hc_zp_encode(ctx_p.ptr, _dptr(slots), n, _dptr(poly), _stream(stream)))


def hc_zp_decode(ctx_p, poly, slots, stream=None):
    n = _npolys(ctx_p, poly)
    _check(lib().hc_zp_decode(ctx_p.ptr, _dptr(poly), n, _dptr(slots), _stream(stream)))


def hc_zp_lift_ntt(ctx, P, poly, out, stream=None):
    """poly: device [n][N] in [0, P); out: device [n][L][N]."""
    n = poly.numel() // ctx.N
    _check(lib().hc_zp_lift_ntt(ctx.ptr, int(P), _dptr(poly), n, _dptr(out), _stream(stream)))


def hc_zp_matvec_preprocess(ctx, ctx_p, W, out, stream=None):
    """W: host [n_out][n_in] residues mod P; out: device tensor of at least n*L*N words.
    Returns n, the number of plaintexts written (the iteration's length)."""
    Wm = np.ascontiguousarray(W, dtype=np.uint64)
    n_out, n_in = Wm.shape
    nt = C.c_uint32()
    _check(lib().hc_zp_matvec_preprocess(ctx.ptr, ctx_p.ptr, C.c_void_p(Wm.ctypes.data), n_out, n_in, _dptr(out),
                                         out.numel(), C.byref(nt), _stream(stream)))
    return nt.value


def hc_zp_conv_preprocess(ctx, ctx_p, desc, K, out, stream=None):
    """K: host [M][C][kh][kw] residues mod P; out: device tensor of at least Y*kh*kw*C*L*N words
    (Y = ceil(M/2)), written [Y][kh*kw][C][L][N] in the NTT domain."""
    Km = np.ascontiguousarray(K, dtype=np.uint64)
    assert Km.shape == (desc.M, desc.C, desc.kh, desc.kw)
    _check(lib().hc_zp_conv_preprocess(ctx.ptr, ctx_p.ptr, C.byref(desc), C.c_void_p(Km.ctypes.data), _dptr(out),
                                       out.numel(), _stream(stream)))


def hc_zp_conv(ctx, desc, key_1, key_row, w_ntt, ct_in, ct_out, stream=None):
    """The Z_P convolution: ct_in device [C][2][L][N], ct_out device [ceil(M/2)][2][L][N]; key_1 /
    key_row the Galois keys of the one-slot and next-kernel-row rotations (None when unused)."""
    _check(lib().hc_zp_conv(ctx.ptr, C.byref(desc), key_1.ptr if key_1 is not None else None,
                            key_row.ptr if key_row is not None else None, _dptr(w_ntt), _dptr(ct_in), _dptr(ct_out),
                            _stream(stream)))


class Plan(_Handle):
    """A plan handle; keeps the contexts, weights and tensors it refers to alive."""


def work_conv(ctx, w, ct_in, ct_out):
    """Plan item: one conv layer (hc_conv_ct_pt's arguments)."""
    return (HC_WORK_CONV, ctx, w, ct_in, None, ct_out, 0)


def work_products(ctx, ct, pt_ntt, out):
    """Plan item: standalone products out[j] = INTT(NTT(ct[j]) . pt_ntt[j]), j < n."""
    n = _npolys(ctx, pt_ntt)
    if _npolys(ctx, ct) != 2 * n or _npolys(ctx, out) != 2 * n:
        raise ValueError("ct and out must hold 2*n polynomials, pt_ntt n")
    return (HC_WORK_PRODUCTS, ctx, None, ct, pt_ntt, out, n)


def hc_plan_create(items):
    """items: list of work_conv(...) / work_products(...) tuples."""
    arr = (hc_work_item * max(1, len(items)))()
    keep = []
    for i, (kind, ctx, w, ct_in, pt, ct_out, n) in enumerate(items):
        arr[i] = hc_work_item(kind, ctx.ptr, w.ptr if w is not None else None, _dptr(ct_in),
                              _dptr(pt) if pt is not None else None, _dptr(ct_out), n)
        keep.append((ctx, w, ct_in, pt, ct_out))
    h = C.c_void_p()
    _check(lib().hc_plan_create(C.cast(arr, C.c_void_p), len(items), C.byref(h)))
    return Plan(h, keep=keep)


def hc_plan_run(plan, stream=None):
    _check(lib().hc_plan_run(plan.ptr, _stream(stream)))


def hc_plan_run_plain(plan, stream=None):
    _check(lib().hc_plan_run_plain(plan.ptr, _stream(stream)))


def hc_plan_autotune(plan, cache_path=None, stream=None):
    _check(lib().hc_plan_autotune(plan.ptr, cache_path.encode() if cache_path else None, _stream(stream)))


def hc_plan_info(plan):
    """(products, algorithmic bytes, kernel launches) of one batched run."""
    a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint32()
    _check(lib().hc_plan_info(plan.ptr, C.byref(a), C.byref(b), C.byref(c)))
    return int(a.value), int(b.value), int(c.value)


class Server(_Handle):
    """A server handle; keeps its layers' contexts and weights alive."""


HC_SERVER_EQUAL_PRIORITY = 1


def hc_server_create(budget_bytes=0, max_batch=0, max_inflight=0, flags=0, selftest_wait_limit=0):
    cfg = hc_server_config(budget_bytes, max_batch, max_inflight, flags, selftest_wait_limit)
    h = C.c_void_p()
    _check(lib().hc_server_create(C.byref(cfg), C.byref(h)))
    return Server(h, keep=[])


def hc_server_add_layer(srv, ctx, w):
    lid = C.c_uint32()
    _check(lib().hc_server_add_layer(srv.ptr, ctx.ptr, w.ptr, C.byref(lid)))
    srv._keep.append((ctx, w))
    return int(lid.value)


def hc_server_submit(srv, layer_id, h_in, h_out=None):
    """Queue a request; h_in / h_out: host arrays (pinned CPU tensors or numpy), h_out None = keep on device.
    The caller keeps both alive until the request is done.  Returns the ticket."""
    t = C.c_uint64()
    _check(lib().hc_server_submit(srv.ptr, layer_id, _hptr(h_in), _hptr(h_out) if h_out is not None else None,
                                  C.byref(t)))
    return int(t.value)


def _info(i):
    return {"status": int(i.status), "batch_size": int(i.batch_size), "queue_ms": float(i.queue_ms),
            "latency_ms": float(i.latency_ms)}


def hc_server_wait(srv, ticket, timeout_s=-1.0):
    i = hc_request_info()
    _check(lib().hc_server_wait(srv.ptr, ticket, timeout_s, C.byref(i)))
    return _info(i)


def hc_server_poll(srv, ticket):
    """None while running, else the request's info dict."""
    d, i = C.c_int(), hc_request_info()
    _check(lib().hc_server_poll(srv.ptr, ticket, C.byref(d), C.byref(i)))
    return _info(i) if d.value else None


def hc_server_result(srv, ticket):
    """Device address of a done request's pool-resident result."""
    p = C.c_void_p()
    _check(lib().hc_server_result(srv.ptr, ticket, C.byref(p)))
    return int(p.value)


def hc_server_fetch(srv, ticket, h_out):
    _check(lib().hc_server_fetch(srv.ptr, ticket, _hptr(h_out)))


def hc_server_release(srv, ticket):
    _check(lib().hc_server_release(srv.ptr, ticket))


def hc_server_stats_get(srv):
    st = hc_server_stats()
    _check(lib().hc_server_stats_get(srv.ptr, C.byref(st)))
    return {n: int(getattr(st, n)) for n, _ in hc_server_stats._fields_}


def hc_server_shutdown(srv):
    _check(lib().hc_server_shutdown(srv.ptr))


def hc_profile_enable(on=True):
    lib().hc_profile_enable(1 if on else 0)


def hc_profile_collect():
    """{kernel name: (launches, total device ms)} since the last collect."""
    cap = 64
    arr = (hc_kernel_time * cap)()
    n = C.c_size_t()
    _check(lib().hc_profile_collect(C.cast(arr, C.c_void_p), cap, C.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n.value, cap))}


def hc_free(handle):
    if isinstance(handle, _Handle):
        handle.close()
    elif handle:
        lib().hc_free(handle)


def hc_status_str(status):
    return lib().hc_status_str(status).decode()


def hc_last_error():
    return lib().hc_last_error().decode(errors="replace")


def hc_version():
    return lib().hc_version().decode()
