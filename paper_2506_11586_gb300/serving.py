"""Serving workload driver: Poisson arrivals of conv-layer requests into the
library's request loop (hc_server_*), as a server answering many clients'
linear layers would see them (Sec. 6.2 server role; Sec. 8 networks).

Layers: the 25 stride-1 SqueezeNet-1.1 convolutions at N = 8192 with three
50-bit primes and the 46 stride-1 ResNet-50 convolution instances at
N = 16384 with four, every one with its own seeded int8 weights,
preprocessed once and resident.  Each layer has one seeded input
ciphertext set in pinned host memory, which every request of that layer
sends (the values do not change the work).  Requests keep their results in
the server's pool; a consumer thread retires them in arrival order and
releases them.

All computation happens in the library; this module only builds the
workload, paces the submissions and summarises the latencies the library
measured (submission -> result ready)."""
import threading
import time

import numpy as np

from . import _lib as L
from .inputs import (CANONICAL_PRIMES, SQUEEZENET_1_1, T_PLAIN, Stream, resnet50_instances, serving_trace,
                     uniform_residues)

FAMILIES = ((8192, 3), (16384, 4))


class ServingLayers:
    """Contexts, resident weights and pinned inputs of every servable layer."""

    def __init__(self, seed=5, pin=True, conv_form=None):
        import torch
        self.ctx = [L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN) for N, nl in FAMILIES]
        if conv_form is not None:           # launch form of every request's layer (kernel family 7)
            for c in self.ctx:
                L.hc_ctx_set_variant(c, L.KIND_CONV_FORM, conv_form)
        self.layers = [[], []]          # per family: dicts(name, w, h_in, nl, N)
        shapes = [[(sh, 0) for sh in SQUEEZENET_1_1], resnet50_instances()]
        t0 = time.perf_counter()
        for fam, lst in enumerate(shapes):
            N, nl = FAMILIES[fam]
            for idx, (sh, occ) in enumerate(lst):
                s = Stream(seed, 1000 * fam + idx)
                K = s.int8(sh.M * sh.C * sh.kh * sh.kw).reshape(sh.M, sh.C, sh.kh, sh.kw)
                w = L.hc_weights_preprocess(self.ctx[fam], L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw,
                                                                      pad=sh.pad), K)
                ct = uniform_residues(s, CANONICAL_PRIMES[:nl], (w.I, 2), N)
                h_in = torch.from_numpy(ct.view(np.int64).reshape(-1))
                if pin:
                    h_in = h_in.pin_memory()
                name = sh.name if fam == 0 else "%s#%d" % (sh.name, occ)
                self.layers[fam].append(dict(name=name, w=w, h_in=h_in, ct=ct, nl=nl, N=N,
                                             products=w.desc.M * w.I))
        torch.cuda.synchronize()
        self.setup_s = time.perf_counter() - t0
        self.weight_bytes = sum(L.hc_weights_data(d["w"])[1] * d["nl"] * d["N"] * 8
                                for fam in self.layers for d in fam)


def run(layers: ServingLayers, n_requests=6000, rate=200.0, seed=5, budget_bytes=32 << 30, max_batch=64,
        max_inflight=0, flags=0, check_every=100):
    """Replay a Poisson trace through a fresh server; returns a summary dict.
    Every `check_every`-th request keeps its result in the pool until the trace has
    ended; it is then fetched and compared bit for bit with the same layer run alone
    on the same input (computed before the trace starts), so that checking adds no
    copies or host work to the timed trace.  max_inflight 0 and flags 0:
    the library's defaults (four stream slots, smaller ring degrees at higher stream
    priority)."""
    trace = serving_trace(n_requests, rate, seed, (len(layers.layers[0]), len(layers.layers[1])))
    check_idx = set(range(0, n_requests, check_every)) if check_every else set()
    alone = {}
    for j in sorted(check_idx):
        key = (int(trace.family[j]), int(trace.layer[j]))
        if key not in alone:
            d = layers.layers[key[0]][key[1]]
            out = np.zeros((d["w"].O, 2, d["nl"], d["N"]), dtype=np.uint64)
            L.hc_conv_ct_pt_host(layers.ctx[key[0]], d["w"], d["ct"], out)
            alone[key] = out
    srv = L.hc_server_create(budget_bytes=budget_bytes, max_batch=max_batch, max_inflight=max_inflight,
                             flags=flags)
    ids = [[L.hc_server_add_layer(srv, layers.ctx[f], d["w"]) for d in layers.layers[f]] for f in range(2)]
    tickets = [None] * n_requests
    submitted = threading.Semaphore(0)
    matches = {}
    infos = [None] * n_requests

    def consumer():
        for j in range(n_requests):
            submitted.acquire()
            infos[j] = L.hc_server_wait(srv, tickets[j])
            if j not in check_idx:
                L.hc_server_release(srv, tickets[j])

    th = threading.Thread(target=consumer)
    th.start()
    t0 = time.perf_counter()
    lag = []
    for j in range(n_requests):
        target = t0 + float(trace.t[j])
        while True:
            now = time.perf_counter()
            if now >= target:
                break
            time.sleep(min(target - now, 0.0005) if target - now > 0.0002 else 0)
        lag.append(now - target)
        d = layers.layers[int(trace.family[j])][int(trace.layer[j])]
        tickets[j] = L.hc_server_submit(srv, ids[int(trace.family[j])][int(trace.layer[j])], d["h_in"])
        submitted.release()
    th.join()
    wall = time.perf_counter() - t0
    st = L.hc_server_stats_get(srv)
    for j in sorted(check_idx):
        key = (int(trace.family[j]), int(trace.layer[j]))
        out = np.empty_like(alone[key])
        L.hc_server_fetch(srv, tickets[j], out)
        L.hc_server_release(srv, tickets[j])
        matches[j] = bool(np.array_equal(out, alone[key]))
    L.hc_free(srv)

    bit_exact = all(matches.values())
    lat = np.array([i["latency_ms"] for i in infos])
    qms = np.array([i["queue_ms"] for i in infos])
    bsz = np.array([i["batch_size"] for i in infos])
    ok = all(i["status"] == L.HC_OK for i in infos)
    by_fam = {}
    for f, nm in enumerate(("squeezenet_N8192_L3", "resnet50_N16384_L4")):
        sel = trace.family == f
        if sel.any():
            by_fam[nm] = {"requests": int(sel.sum()), "p50_ms": float(np.percentile(lat[sel], 50)),
                          "p99_ms": float(np.percentile(lat[sel], 99))}
    return {
        "requests": n_requests, "rate_per_s": rate, "seed": seed, "all_ok": ok,
        "p50_ms": float(np.percentile(lat, 50)), "p90_ms": float(np.percentile(lat, 90)),
        "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
        "queue_p99_ms": float(np.percentile(qms, 99)),
        "products": int(st["products"]), "wall_s": wall, "products_per_s": st["products"] / wall,
        "batches": int(st["batches"]), "mean_batch": float(bsz.mean()), "max_batch": int(st["max_batch_seen"]),
        "pool_bytes": int(st["pool_bytes"]), "peak_pool_bytes": int(st["peak_bytes_in_use"]),
        "submit_lag_p99_ms": float(np.percentile(np.array(lag), 99) * 1e3),
        "bit_exact_vs_alone": bit_exact, "checked_requests": len(matches), "by_family": by_fam,
        "max_inflight": max_inflight or 4, "equal_priority": bool(flags & L.HC_SERVER_EQUAL_PRIORITY),
    }
