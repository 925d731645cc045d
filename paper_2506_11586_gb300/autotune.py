"""Launch-shape autotuner.

For a context (ring degree N, L limbs) it times every launch variant of each
kernel family on a representative batch through the C ABI (CUDA events on
the launching stream, L2 flushed between repetitions), keeps the fastest and
records the choice in the context with hc_ctx_set_variant.  Every variant
computes the same bits (tests/test_gpu_variants.py), so tuning only changes
speed.  Results are cached in a JSON file keyed by GPU name, SM count, N and
L; a cached entry is applied without timing.
"""
import json
import os

import numpy as np

from . import _lib as L
from .build import BUILD
from .inputs import Stream, uniform_residues

DEFAULT_CACHE = os.path.join(BUILD, "autotune.json")

KINDS = {
    "ntt_fwd": L.KIND_NTT_FWD,
    "ntt_inv": L.KIND_NTT_INV,
    "mac_intt": L.KIND_MAC_INTT,
    "product": L.KIND_PRODUCT,
    "ntt_fwd_ct": L.KIND_NTT_FWD_CT,
    "ntt_inv_ct": L.KIND_NTT_INV_CT,
}


def _key(ctx):
    import torch
    dev = torch.cuda.current_device()
    p = torch.cuda.get_device_properties(dev)
    return "%s|sm%d|N%d|L%d" % (p.name, p.multi_processor_count, ctx.N, ctx.L)


def _time(fn, reps=5):
    import torch
    flush = torch.empty(32 << 20, dtype=torch.int64, device="cuda")
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def _workloads(ctx):
    """name -> callable running one representative launch of that family."""
    import torch
    N, moduli = ctx.N, ctx.moduli
    n_ct = max(32, (1 << 21) // (N * ctx.L))            # ~16 MB of ciphertexts
    s = Stream(0xA7, N)
    ct = torch.from_numpy(uniform_residues(s, moduli, (n_ct, 2), N).view(np.int64)).cuda()
    pt = torch.from_numpy(uniform_residues(s, moduli, (n_ct,), N).view(np.int64)).cuda()
    buf = torch.empty_like(ct)
    out = torch.empty_like(ct)
    slots_single = np.arange(n_ct, dtype=np.uint32)
    slots_group = (np.arange(n_ct) // 8).astype(np.uint32)
    out_group = torch.empty(((n_ct + 7) // 8) * 2 * ctx.L * N, dtype=torch.int64, device="cuda")
    return {
        "ntt_fwd": lambda: L.hc_ntt_fwd(ctx, buf.copy_(ct)),
        "ntt_inv": lambda: L.hc_ntt_inv(ctx, buf.copy_(ct)),
        "ntt_fwd_ct": lambda: L.hc_ctpt_mac(ctx, ct, pt, slots_group, out_group),
        "mac_intt": lambda: L.hc_ctpt_mac(ctx, ct, pt, slots_group, out_group),
        "product": lambda: L.hc_ctpt_mac(ctx, ct, pt, slots_single, out),
        "ntt_inv_ct": lambda: L.hc_ntt_inv(ctx, buf.copy_(ct)),
    }


def _time_kind_via_trace(ctx, kind, fn, kernel_prefix):
    """Device time of the kernel family alone, from the library's own trace."""
    L.hc_profile_collect()
    L.hc_profile_enable(True)
    try:
        for _ in range(3):
            fn()
        import torch
        torch.cuda.synchronize()
    finally:
        L.hc_profile_enable(False)
    prof = L.hc_profile_collect()
    ms = [v[1] / v[0] for k, v in prof.items() if k.startswith(kernel_prefix)]
    return min(ms) if ms else None


def autotune(ctx, cache_path=DEFAULT_CACHE, kinds=None, verbose=False):
    """Pick the fastest launch variant of each kernel family for ctx; returns {name: variant}."""
    key = _key(ctx)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    names = list(kinds or KINDS)
    if key in cache and all(n in cache[key] for n in names):
        for n in names:
            L.hc_ctx_set_variant(ctx, KINDS[n], int(cache[key][n]))
        return {n: int(cache[key][n]) for n in names}
    work = _workloads(ctx)
    prefix = {"ntt_fwd": "k_ntt_fwd", "ntt_inv": "k_ntt_inv", "ntt_fwd_ct": "k_ntt_fwd",
              "mac_intt": "k_mac_intt", "product": "k_product", "ntt_inv_ct": "k_ntt_inv"}
    chosen = {}
    for n in names:
        kind = KINDS[n]
        best, best_ms = None, None
        for v in range(L.N_VARIANTS):
            L.hc_ctx_set_variant(ctx, kind, v)
            if n == "ntt_inv_ct":
                ms = _time_invct(ctx, v)
            else:
                ms = _time_kind_via_trace(ctx, kind, work[n], prefix[n])
            if verbose:
                print("autotune %s N=%d L=%d variant %d: %.4f ms" % (n, ctx.N, ctx.L, v, ms), flush=True)
            if ms is not None and (best_ms is None or ms < best_ms):
                best, best_ms = v, ms
        L.hc_ctx_set_variant(ctx, kind, best)
        chosen[n] = best
    cache.setdefault(key, {}).update(chosen)
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return chosen


def _time_invct(ctx, variant):
    """Inverse NTT of whole ciphertexts, as the convolution's last phase runs it."""
    import torch
    N = ctx.N
    K = np.zeros((64, 32, 1, 1), dtype=np.int8)
    w = L.hc_weights_preprocess(ctx, L.make_desc(32, 16, 16, 64, 1, 1), K)
    d_in = torch.zeros(w.I * 2 * ctx.L * N, dtype=torch.int64, device="cuda")
    d_out = torch.empty(w.O * 2 * ctx.L * N, dtype=torch.int64, device="cuda")
    return _time_kind_via_trace(ctx, L.KIND_NTT_INV_CT, lambda: L.hc_conv_ct_pt(ctx, w, d_in, d_out),
                                "k_ntt_inv")
