#!/usr/bin/env python
"""Benchmark of the homomorphic-convolution hot path (SecONNds, arXiv 2506.11586, Sec. 6.2).

One step = one online HE convolution layer through the C ABI: forward NTT of
every input ciphertext, NTT-domain multiply-accumulate against the resident
NTT-preprocessed weights, inverse NTT of the outputs -- by default one
hc_conv_ct_pt call, with --step-api plan the layer as a one-item plan
(hc_plan_run) replayed from the CUDA graph the plan captures; the line carries
the other entry point's time too.  Workload:
56x56x64 activations -> 64 output channels, 3x3, stride 1, pad 1, packed into
N = 8192 polynomials over three 50-bit primes (I = 32 input ciphertexts,
P = 512 weight plaintexts, O = 256 output ciphertexts, 2048 ct x pt products).
Inputs are seeded synthetic residues uniform in [0, q_i) (the cost does not
depend on the values); weights are seeded uniform int8.

The same line also carries, measured in the same run:
  batched  -- every stride-1 SqueezeNet-1.1 convolution (25 layers, 23,568
              products, N = 8192, L = 3) as one plan replayed from a CUDA
              graph, against the 25 single-layer calls and the plain
              one-launch-per-product form; and 2000 standalone products of
              uneven ring degree (40/40/20 over N = 4096/8192/16384 with
              2/3/4 limbs) in one persistent launch, against one launch per
              degree and one launch per product;
  serving  -- Poisson arrivals (200 requests/s, seed 5) of single-layer
              requests drawn half from the SqueezeNet-1.1 layers and half
              from the 46 stride-1 ResNet-50 convolution instances
              (N = 16384, L = 4), weights resident, continuous batching under
              a 32 GiB device budget: p50/p99 latency and products/s; the
              same at 800 requests/s (batches form), and at 200 requests/s
              with every batch at one stream priority (the comparison);
  products16 -- 16 ct x pt products at N = 4096, L = 2: independent, the
              same accumulated into one slot, and one call per product;
  int_probe -- the integer multiply pipe's measured rate (lazy Shoup
              products, 32-bit and wide multiply-adds) against the peak;
  networks -- every linear layer of SqueezeNet-1.1 and of ResNet-50, each
              network one plan;
  server_step, preprocessing_modes, e2e, plain, cpu_baseline -- the server's
              whole step, the online / no-NTT weight modes, the host-buffer
              entry point, the one-launch-per-product form and the oracle's
              rate, all on the same layer;
  zp       -- SecONNds-P's Z_P operations (rotations, the multiply-
              accumulate-rotate iteration, SIMD encoding, a matrix-vector
              layer) at N = 8192, L = 3.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle (plain
schoolbook convolution) on a bounded sample of the same workload instead.
"""
import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HE conv ct x pt products/s (bit-exact)"
UNIT = "products/s"
WORKLOAD = "conv3x3_56x56x64_to64_N8192_L3"
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
TUNE_CACHE = os.path.join(ROOT, "paper_2506_11586_gb300", "_build", "autotune.txt")


KIND_NAMES = {"ntt_fwd_ct": 4, "mac_conv": 6, "ntt_inv_ct": 5, "conv_form": 7}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--conv-form", type=int, default=None, choices=[0, 1, 2],
                    help="force the layer's launch form instead of the autotuned one")
    ap.add_argument("--mac-variant", type=int, default=None, choices=[0, 1, 2, 3],
                    help="force the blocked MAC's variant (3: the tensor-core MAC) instead of the autotuned one")
    ap.add_argument("--no-mac-variants", action="store_true", help="skip the integer / tensor-core MAC section")
    ap.add_argument("--batched-reps", type=int, default=20)
    ap.add_argument("--step-api", default="direct", choices=["direct", "plan"],
                    help="timed step: a one-layer plan replayed from a CUDA graph, or one hc_conv_ct_pt call")
    ap.add_argument("--no-zp", action="store_true", help="skip the Z_P rotation section")
    ap.add_argument("--no-networks", action="store_true",
                    help="skip the whole-network plans (SqueezeNet-1.1 and ResNet-50, every linear layer)")
    ap.add_argument("--no-batched-plain", action="store_true", help="skip the one-launch-per-product comparisons")
    ap.add_argument("--serving-requests", type=int, default=6000)
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--serving-rate-high", type=float, default=800.0)
    ap.add_argument("--profile-case", default=None, choices=["ntt_inv"],
                    help="run one small case for a profiler and exit: ntt_inv = the inverse NTT of 1536 "
                         "polynomial limbs (N = 8192, L = 3) in its persistent and one-CTA shapes, then the "
                         "integer-pipe probe (lazy Shoup products)")
    return ap.parse_args()


def workload_shape():
    from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, CONV_56x56x64
    return CONV_56x56x64, 8192, CANONICAL_PRIMES[:3]


def geometry():
    """The layer's partition and counts through the library (the product's own geometry)."""
    from paper_2506_11586_gb300 import _lib as L
    sh, N, moduli = workload_shape()
    res, I, P, O = L.hc_conv_partition(L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad), N)
    G = (sh.C + res.Cw - 1) // res.Cw
    B = I // G
    return dict(I=I, P=P, O=O, G=G, B=B, products=sh.M * G * B, Cw=res.Cw, Hw=res.Hw, Ww=res.Ww)


def oracle_geometry():
    """The same layer's partition from the oracle alone (the reference arm never loads the library)."""
    from oracle import conv
    sh, N, moduli = workload_shape()
    p = conv.canonical_partition(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, sh.pad, N)
    return dict(I=p.I, P=p.P, O=p.O, G=p.G, B=p.B, products=p.products, Cw=p.Cw, Hw=p.Hw, Ww=p.Ww)


def run_config(geo, N, nl, world):
    """The workload description both arms print (identical keys and values)."""
    return {"workload": WORKLOAD, "N": N, "L": nl, "I": geo["I"], "P": geo["P"], "O": geo["O"],
            "products_per_layer": geo["products"], "partition": [geo["Cw"], geo["Hw"], geo["Ww"]],
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "GPU arm: 512 MB buffer written between timed steps (flushes the 129 MB L2)"}


def alg_bytes(geo, N, L):
    """Algorithmic HBM bytes of one layer: read 2I input polys, P weights, write 2O outputs."""
    return 8 * N * L * (2 * geo["I"] + geo["P"] + 2 * geo["O"])


# Integer-pipe cost model (measured on GB300 with ncu counters): the fmaheavy
# pipe runs 64 32-bit multiply-adds per clock per SM; a 32x32->64 multiply
# (mad.wide.u32) occupies it twice as long.  In these units a lazy Shoup
# multiplication (5 wide + 4 narrow) costs 14, a MAC term (4 wide) 8 and the
# final reduction of a MAC sum (one Shoup + one w=1 reduction) 19.
IMAD_EQ_BUTTERFLY, IMAD_EQ_MAC_TERM, IMAD_EQ_REDUCE = 14, 8, 19


def device_sms():
    """Streaming multiprocessors of the current device (152 on GB300); None without a GPU."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    except Exception:
        pass
    return None


def peak_sm_mhz():
    mhz = 2070.0
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return mhz


def alu_peak_imad_eq(sms=None):
    """T IMAD-equivalents/s: 64 per clock per SM x the device's SMs x the maximum SM clock."""
    sms = sms or device_sms() or 152
    return 64 * sms * peak_sm_mhz() * 1e6 / 1e12


def int_probe(L, ctx, stream, iters=4096):
    """The library's integer-pipe probe: lazy Shoup multiplications, narrow and wide
    multiply-adds, each as operations/s and as a fraction of the derived peak."""
    out = {"sms": device_sms(), "peak_t_imad_eq_s": alu_peak_imad_eq(), "peak_sm_mhz": peak_sm_mhz()}
    for name, form in (("shoup_lazy", 0), ("mad_lo_u32", 1), ("mad_wide_u32", 2)):
        rate, ms, eq = L.hc_probe_int_rate(ctx, form, iters if form == 0 else iters * 8, stream)
        out[name] = {"ops_per_s": rate, "imad_eq_per_op": eq, "t_imad_eq_per_s": rate * eq / 1e12,
                     "frac_of_peak": rate * eq / 1e12 / out["peak_t_imad_eq_s"], "ms": ms}
    return out


def kernel_work(name, geo, N, L):
    """Algorithmic bytes and IMAD-equivalents of one launch of a kernel of the layer."""
    logn = N.bit_length() - 1
    bfly = (N // 2) * logn
    poly = 8 * N * L
    I, P, O, prods = geo["I"], geo["P"], geo["O"], geo["products"]
    mac = prods * 2 * L * N * IMAD_EQ_MAC_TERM + O * 2 * L * N * IMAD_EQ_REDUCE
    if name.startswith("k_ntt_fwd"):
        return {"bytes": 2 * poly * 2 * I, "imad_eq": 2 * I * L * bfly * IMAD_EQ_BUTTERFLY}
    if name.startswith("k_ntt_inv"):
        return {"bytes": 2 * poly * 2 * O, "imad_eq": 2 * O * L * bfly * IMAD_EQ_BUTTERFLY}
    if name.startswith("k_mac_conv") or name.startswith("k_mac_tc"):
        return {"bytes": poly * (2 * I + P + 2 * O), "imad_eq": mac}
    # fused MAC + inverse NTT
    return {"bytes": poly * (2 * I + P + 2 * O), "imad_eq": mac + 2 * O * L * bfly * IMAD_EQ_BUTTERFLY}


def conv_imad_eq(I, O, products, N, L):
    """IMAD-equivalents of one conv layer: forward NTT of 2I, MAC, inverse NTT of 2O polynomial limbs."""
    bfly = (N // 2) * (N.bit_length() - 1)
    return (2 * I * L * bfly * IMAD_EQ_BUTTERFLY + products * 2 * L * N * IMAD_EQ_MAC_TERM
            + O * 2 * L * N * IMAD_EQ_REDUCE + 2 * O * L * bfly * IMAD_EQ_BUTTERFLY)


def product_imad_eq(N, L):
    """IMAD-equivalents of one standalone ct x pt product: NTT, pointwise product, INTT of 2L limbs."""
    bfly = (N // 2) * (N.bit_length() - 1)
    return 2 * L * (2 * bfly * IMAD_EQ_BUTTERFLY + N * IMAD_EQ_BUTTERFLY)


def roofline_fracs(nbytes, imad_eq, ms):
    """Fractions of the measured HBM peak and of the integer-pipe peak, and the larger (the bound)."""
    peak, src = measured_peaks()
    hbm = nbytes / (ms / 1e3) / 1e9 / peak
    alu = imad_eq / (ms / 1e3) / 1e12 / alu_peak_imad_eq()
    return {"hbm_frac": hbm, "alu_frac": alu, "bound": "alu" if alu >= hbm else "hbm",
            "imad_eq": imad_eq, "hbm_peak_source": src}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


DEVICE_SOURCES = ("*.cuh", "hc_internal.h", "hc_launch.cu", "hc_kernels_n*.cu", "hc_mixed.cu", "hc_fused.cu")


def source_hash():
    """Hash of the files that define the kernels (not the host-only runtime)."""
    h = hashlib.sha256()
    files = set()
    for pat in DEVICE_SOURCES:
        files.update(glob.glob(os.path.join(ROOT, "paper_2506_11586_gb300", "csrc", pat)))
    for f in sorted(files):
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode() + fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel_key):
    """DRAM bytes per launch of a kernel from the committed ncu summary, or None
    if absent or taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_hash") != source_hash():
        return None
    v = vals.get(kernel_key)
    return float(v) if v else None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


class OracleLayer:
    """The metric layer set up once for the oracle: packed weights, one seeded input
    batch, and a seeded order of output ciphertexts; run(k) computes the next k
    output ciphertexts by the oracle's sparse schoolbook products."""

    def __init__(self, seed=2):
        import numpy as np
        from oracle import conv
        from paper_2506_11586_gb300.inputs import Stream, conv_tensors, uniform_residues
        sh, N, self.moduli = workload_shape()
        _, K = conv_tensors(sh, seed=seed)
        self.p = conv.canonical_partition(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, sh.pad, N)
        self.ct = uniform_residues(Stream(seed, 5), self.moduli, (self.p.I, 2), N)
        self.Kp = conv.pack_weights(K.astype(np.int64), self.p)
        self.order = [int(o) for o in Stream(seed, 6).u64(self.p.O).argsort()]
        self.next = 0
        self.conv = conv

    def run(self, k):
        """k output ciphertexts (cycling through the layer); returns the products computed."""
        for _ in range(k):
            o = self.order[self.next % self.p.O]
            self.next += 1
            self.conv.conv_ct_pt(self.ct, self.Kp, self.p, self.moduli, outputs=[o])
        return k * self.p.G


def oracle_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def cpu_oracle_rate(seconds, layer=None):
    """Oracle convolution (plain schoolbook) of as many output ciphertexts as fit in
    ~`seconds`, set-up excluded; returns (products/s, outputs done, products done,
    elapsed, threads)."""
    layer = layer or OracleLayer()
    layer.run(1)                                   # warm-up (first-call costs of the C core)
    done = prods = 0
    t0 = time.perf_counter()
    while done < layer.p.O:
        prods += layer.run(1)
        done += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return prods / el, done, prods, el, oracle_threads()


# output ciphertexts per step of the reference arm: 16 of the layer's 256 (128 products)
REFERENCE_OUTPUTS_PER_STEP = 16


def run_reference(args):
    """The oracle on the host cores, on a bounded sample of the same layer per step.
    Loads only the oracle's C core: the partition comes from oracle.conv."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import build_oracle
    build_oracle()
    geo = oracle_geometry()
    sh, N, moduli = workload_shape()
    layer = OracleLayer()
    for _ in range(args.warmup):
        layer.run(REFERENCE_OUTPUTS_PER_STEP)
    times = []
    products = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        products += layer.run(REFERENCE_OUTPUTS_PER_STEP)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = products / total
    sample = ("%d of %d output ciphertexts per step (%d products), sparse schoolbook oracle, set-up untimed"
              % (REFERENCE_OUTPUTS_PER_STEP, geo["O"], REFERENCE_OUTPUTS_PER_STEP * geo["G"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": run_config(geo, N, len(moduli), 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _events_ms(fn, reps, stream, flush=None):
    """Device time (ms) of each of reps calls of fn, CUDA events on stream."""
    import torch
    out = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b))
    return out


def _kernel_trace(L, fn, nvtx_name):
    """Per-kernel device times of one call of fn (library trace), inside an NVTX range."""
    import torch
    L.hc_profile_collect()
    L.hc_profile_enable(True)
    torch.cuda.nvtx.range_push(nvtx_name)
    fn()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    L.hc_profile_enable(False)
    return {k: {"launches": v[0], "ms": v[1]} for k, v in L.hc_profile_collect().items()}


def batched_squeezenet(L, stream, reps=20, with_plain=True):
    """All 25 stride-1 SqueezeNet-1.1 layers as one plan (CUDA graph) vs per-layer calls vs plain."""
    import numpy as np
    import torch
    from paper_2506_11586_gb300.inputs import (CANONICAL_PRIMES, SQUEEZENET_1_1, T_PLAIN, Stream, conv_tensors,
                                               uniform_residues)
    ctx = L.hc_ctx_create(8192, CANONICAL_PRIMES[:3], T_PLAIN)
    items = []
    kernels = [conv_tensors(sh, seed=3)[1] for sh in SQUEEZENET_1_1]
    torch.cuda.synchronize()
    t_pre = time.perf_counter()
    ws = [L.hc_weights_preprocess(ctx, L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad), K)
          for sh, K in zip(SQUEEZENET_1_1, kernels)]
    torch.cuda.synchronize()
    offline_s = time.perf_counter() - t_pre
    for i, (sh, w) in enumerate(zip(SQUEEZENET_1_1, ws)):
        ct = uniform_residues(Stream(3, 100 + i), CANONICAL_PRIMES[:3], (w.I, 2), 8192)
        items.append((w, torch.from_numpy(ct.view(np.int64)).cuda(),
                      torch.empty(w.O * 2 * 3 * 8192, dtype=torch.int64, device="cuda")))
    plan = L.hc_plan_create([L.work_conv(ctx, w, a, b) for w, a, b in items])
    products, nbytes, launches = L.hc_plan_info(plan)
    L.hc_plan_autotune(plan, TUNE_CACHE, stream)
    for _ in range(3):
        L.hc_plan_run(plan, stream)
    g = _events_ms(lambda: L.hc_plan_run(plan, stream), reps, stream)
    batched = [b.clone() for _, _, b in items]

    def per_layer():
        for w, a, b in items:
            L.hc_conv_ct_pt(ctx, w, a, b, stream)
    per_layer()
    pl = _events_ms(per_layer, max(3, reps // 2), stream)
    exact_layers = all(bool(torch.equal(x, b)) for x, (_, _, b) in zip(batched, items))
    pp, exact_plain = [None], None
    if with_plain:
        pp = _events_ms(lambda: L.hc_plan_run_plain(plan, stream), 1, stream)
        exact_plain = all(bool(torch.equal(x, b)) for x, (_, _, b) in zip(batched, items))
    kern = _kernel_trace(L, lambda: L.hc_plan_run(plan, stream), "squeezenet_plan")
    ms = statistics.median(g)
    out = {"workload": "squeezenet1.1_stride1_25layers_N8192_L3", "products": products, "alg_bytes": nbytes,
           "launches_per_pass": launches, "batched_ms": ms, "batched_p99_ms": max(g),
           "value": products / (ms / 1e3), "unit": UNIT, "alg_gbs": nbytes / (ms / 1e3) / 1e9,
           "per_layer_ms": statistics.median(pl), "per_layer_launches": 3 * len(items),
           "plain_ms": pp[0], "plain_launches": products,
           "speedup_vs_per_layer": statistics.median(pl) / ms,
           "speedup_vs_plain": pp[0] / ms if pp[0] is not None else None,
           "bit_exact_vs_per_layer": exact_layers, "bit_exact_vs_plain": exact_plain, "kernels": kern,
           "offline_weight_ntt_s": offline_s,
           "variants": {name: L.hc_ctx_get_variant(ctx, k) for name, k in KIND_NAMES.items()},
           "roofline": roofline_fracs(nbytes, sum(conv_imad_eq(w.I, w.O, w.products, 8192, 3) for w in ws), ms)}
    plan.close()
    return out


def whole_networks(L, stream, reps=10):
    """Every linear layer of SqueezeNet-1.1 (26: conv1 stride 2 and the 25 stride-1
    layers; N = 8192, L = 3) and of ResNet-50 (54: 46 stride-1 and 7 strided
    convolutions and the fully connected classifier; N = 16384, L = 4), each
    network one plan replayed from a CUDA graph, vs one call per layer."""
    import numpy as np
    import torch
    from paper_2506_11586_gb300.inputs import (CANONICAL_PRIMES, RESNET50_FC, RESNET50_STRIDED, SQUEEZENET_1_1,
                                               SQUEEZENET_CONV1, T_PLAIN, Stream, conv_tensors, resnet50_instances,
                                               uniform_residues)
    nets = {
        "squeezenet1.1_all26_N8192_L3": ([SQUEEZENET_CONV1] + list(SQUEEZENET_1_1), 8192, 3),
        "resnet50_all54_N16384_L4": ([sh for sh, _ in resnet50_instances()] + list(RESNET50_STRIDED)
                                     + [RESNET50_FC], 16384, 4),
    }
    out = {}
    for seed, (name, (shapes, N, nl)) in enumerate(nets.items()):
        ctx = L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN)
        torch.cuda.synchronize()
        t_pre = time.perf_counter()
        ws, kinds = [], {"stride1": 0, "strided": 0, "fc": 0}
        for i, sh in enumerate(shapes):
            if isinstance(sh, tuple):                         # fully connected (C, M)
                Wm = Stream(4 + seed, 300 + i).int8(sh[0] * sh[1]).reshape(sh[1], sh[0])
                w = L.hc_weights_preprocess_fc(ctx, L.make_fc_desc(sh[0], sh[1]), Wm)
                kinds["fc"] += w.products
            else:
                K = conv_tensors(sh, seed=4 + seed + 1000 * i)[1]
                st = getattr(sh, "stride", 1)
                w = L.hc_weights_preprocess(ctx, L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad,
                                                             stride=st), K)
                kinds["strided" if st > 1 else "stride1"] += w.products
            ws.append(w)
        torch.cuda.synchronize()
        offline_s = time.perf_counter() - t_pre
        items = []
        for i, w in enumerate(ws):
            ct = uniform_residues(Stream(4 + seed, 100 + i), CANONICAL_PRIMES[:nl], (w.I, 2), N)
            items.append((w, torch.from_numpy(ct.view(np.int64)).cuda(),
                          torch.empty(w.O * 2 * nl * N, dtype=torch.int64, device="cuda")))
        plan = L.hc_plan_create([L.work_conv(ctx, w, a, b) for w, a, b in items])
        products, nbytes, launches = L.hc_plan_info(plan)
        L.hc_plan_autotune(plan, TUNE_CACHE, stream)
        for _ in range(3):
            L.hc_plan_run(plan, stream)
        g = _events_ms(lambda: L.hc_plan_run(plan, stream), reps, stream)
        batched = [b.clone() for _, _, b in items]

        def per_layer():
            for w, a, b in items:
                L.hc_conv_ct_pt(ctx, w, a, b, stream)
        per_layer()
        pl = _events_ms(per_layer, max(3, reps // 2), stream)
        exact = all(bool(torch.equal(x, b)) for x, (_, _, b) in zip(batched, items))
        kern = _kernel_trace(L, lambda: L.hc_plan_run(plan, stream), name)
        ms = statistics.median(g)
        out[name] = {"layers": len(shapes), "products": products, "products_by_kind": kinds, "alg_bytes": nbytes,
                     "resident_weight_bytes": sum(L.hc_weights_data(w)[1] * nl * N * 8 for w in ws),
                     "launches_per_pass": launches, "batched_ms": ms, "batched_p99_ms": max(g),
                     "value": products / (ms / 1e3), "unit": UNIT, "alg_gbs": nbytes / (ms / 1e3) / 1e9,
                     "per_layer_ms": statistics.median(pl), "speedup_vs_per_layer": statistics.median(pl) / ms,
                     "bit_exact_vs_per_layer": exact, "offline_weight_ntt_s": offline_s, "kernels": kern,
                     "variants": {k: L.hc_ctx_get_variant(ctx, v) for k, v in KIND_NAMES.items()},
                     "roofline": roofline_fracs(nbytes, sum(conv_imad_eq(w.I, w.O, w.products, N, nl)
                                                            for w in ws), ms)}
        plan.close()
        del items, batched
        for w in ws:
            w.close()
        ctx.close()
        torch.cuda.empty_cache()
    return out


def batched_uneven(L, stream, reps=20, with_plain=True):
    """2000 standalone products of mixed degree in one persistent launch vs per-degree vs plain."""
    import numpy as np
    import torch
    from paper_2506_11586_gb300.inputs import (CANONICAL_PRIMES, T_PLAIN, UNEVEN_CLASSES, Stream, uneven_mix,
                                               uniform_residues)
    labels = uneven_mix(2000, seed=4)
    items, ctxs = [], []
    for cls, (N, nl, _) in enumerate(UNEVEN_CLASSES):
        n = int((labels == cls).sum())
        ctx = L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN)
        s = Stream(4, 10 + cls)
        ct = torch.from_numpy(uniform_residues(s, CANONICAL_PRIMES[:nl], (n, 2), N).view(np.int64)).cuda()
        pt = torch.from_numpy(uniform_residues(s, CANONICAL_PRIMES[:nl], (n,), N).view(np.int64)).cuda()
        L.hc_ntt_fwd(ctx, pt, stream)
        items.append((ctx, ct, pt, torch.empty_like(ct), n))
        ctxs.append(ctx)
    plan = L.hc_plan_create([L.work_products(c, a, p, o) for c, a, p, o, _ in items])
    products, nbytes, launches = L.hc_plan_info(plan)
    for _ in range(3):
        L.hc_plan_run(plan, stream)
    g = _events_ms(lambda: L.hc_plan_run(plan, stream), reps, stream)
    batched = [o.clone() for _, _, _, o, _ in items]

    def per_degree():
        for c, a, p, o, n in items:
            L.hc_ctpt_mac(c, a, p, np.arange(n), o, stream)
    per_degree()
    pd = _events_ms(per_degree, reps, stream)
    exact_deg = all(bool(torch.equal(x, it[3])) for x, it in zip(batched, items))
    pp, exact_plain = [None], None
    if with_plain:
        pp = _events_ms(lambda: L.hc_plan_run_plain(plan, stream), 2, stream)
        exact_plain = all(bool(torch.equal(x, it[3])) for x, it in zip(batched, items))
    kern = _kernel_trace(L, lambda: L.hc_plan_run(plan, stream), "uneven_plan")
    ms = statistics.median(g)
    out = {"workload": "uneven_2000_products_40_40_20_N4096L2_N8192L3_N16384L4", "products": products,
           "alg_bytes": nbytes, "launches_per_pass": launches, "batched_ms": ms, "batched_p99_ms": max(g),
           "value": products / (ms / 1e3), "unit": UNIT, "alg_gbs": nbytes / (ms / 1e3) / 1e9,
           "per_degree_ms": statistics.median(pd),
           "plain_ms": statistics.median(pp) if pp[0] is not None else None, "plain_launches": products,
           "speedup_vs_per_degree": statistics.median(pd) / ms,
           "speedup_vs_plain": statistics.median(pp) / ms if pp[0] is not None else None,
           "bit_exact_vs_per_degree": exact_deg, "bit_exact_vs_plain": exact_plain, "kernels": kern,
           "roofline": roofline_fracs(nbytes, sum(n * product_imad_eq(c.N, c.L) for c, _, _, _, n in items), ms)}
    plan.close()
    return out


def mac_variants_section(L, ctx, w, d_in, d_out, stream, flush, reps=50):
    """The layer with the integer MAC (stages of 16 weight rows) and with the
    tensor-core MAC, launch form 0: MAC kernel time per launch, layer time, and
    every output residue of the tensor-core MAC against the integer MAC's."""
    import torch
    kinds = (L.KIND_MAC_CONV, L.KIND_CONV_FORM)
    saved = [L.hc_ctx_get_variant(ctx, k) for k in kinds]
    out, ref = {}, None
    L.hc_ctx_set_variant(ctx, L.KIND_CONV_FORM, 0)
    for name, v, kern in (("integer", 1, "k_mac_conv"), ("tensor_core", 3, "k_mac_tc")):
        L.hc_ctx_set_variant(ctx, L.KIND_MAC_CONV, v)
        fn = lambda: L.hc_conv_ct_pt(ctx, w, d_in, d_out, stream)
        fn()
        layer = statistics.median(_events_ms(fn, reps, stream, flush))
        L.hc_profile_collect()
        L.hc_profile_enable(True)
        for _ in range(reps):
            flush.zero_()
            fn()
        torch.cuda.synchronize()
        L.hc_profile_enable(False)
        prof = L.hc_profile_collect()
        n, ms = prof.get(kern, (0, 0.0))
        out[name] = {"kernel": kern, "mac_us": 1000 * ms / n if n else None, "layer_form0_ms": layer}
        if ref is None:
            ref = d_out.clone()
        else:
            out[name]["bit_exact_vs_integer"] = bool(torch.equal(ref, d_out))
    for k, v in zip(kinds, saved):
        L.hc_ctx_set_variant(ctx, k, v)
    return out


def products16(L, stream, flush, reps=50):
    """The plain ct x pt batch (seed 1): N = 4096, two 50-bit primes, 16 products of
    uniform residues.  The 16 independent products (one output slot each) in one
    hc_ctpt_mac call, the same 16 accumulated into one slot in one call, and the
    plain form (one call, i.e. one fused NTT -> product -> INTT launch, per product);
    L2 flushed before every timed call.  The batch is 5.2 MB, so it is bound by
    launch latency and the transforms' dependency chains, not by HBM."""
    import numpy as np
    import torch
    from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream, uniform_residues
    N, nl, n = 4096, 2, 16
    ctx = L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    s = Stream(1, 0)
    # flat device tensors, so that slices select products
    ct = torch.from_numpy(uniform_residues(s, CANONICAL_PRIMES[:nl], (n, 2), N).view(np.int64).reshape(-1)).cuda()
    pt = torch.from_numpy(uniform_residues(s, CANONICAL_PRIMES[:nl], (n,), N).view(np.int64).reshape(-1)).cuda()
    L.hc_ntt_fwd(ctx, pt, stream)
    out = torch.empty_like(ct)
    acc = torch.empty(2 * nl * N, dtype=torch.int64, device="cuda")
    plain_out = torch.empty_like(ct)
    poly = N * nl
    per = 2 * poly

    def plain():
        for j in range(n):
            L.hc_ctpt_mac(ctx, ct[j * per:(j + 1) * per], pt[j * poly:(j + 1) * poly], np.zeros(1),
                          plain_out[j * per:(j + 1) * per], stream)
    fi = lambda: L.hc_ctpt_mac(ctx, ct, pt, np.arange(n), out, stream)
    fa = lambda: L.hc_ctpt_mac(ctx, ct, pt, np.zeros(n), acc, stream)
    for f in (fi, fa, plain):
        for _ in range(3):
            f()
    ti, ta = _events_ms(fi, reps, stream, flush), _events_ms(fa, reps, stream, flush)
    tp = _events_ms(plain, max(5, reps // 5), stream, flush)
    exact = bool(torch.equal(out, plain_out))
    bfly = (N // 2) * (N.bit_length() - 1)
    ind_bytes = n * 8 * N * nl * 5
    acc_bytes = n * 8 * N * nl * 3 + 8 * N * nl * 2
    acc_imad = (n * 2 * nl * bfly * IMAD_EQ_BUTTERFLY + n * 2 * nl * N * IMAD_EQ_MAC_TERM
                + 2 * nl * N * IMAD_EQ_REDUCE + 2 * nl * bfly * IMAD_EQ_BUTTERFLY)
    mi, ma, mp = statistics.median(ti), statistics.median(ta), statistics.median(tp)
    res = {"workload": "ctpt_16_products_N4096_L2", "products": n,
           "independent": {"ms": mi, "p99_ms": sorted(ti)[int(0.99 * (len(ti) - 1))], "value": n / (mi / 1e3),
                           "unit": UNIT, "alg_bytes": ind_bytes,
                           "roofline": roofline_fracs(ind_bytes, n * product_imad_eq(N, nl), mi),
                           "kernels": _kernel_trace(L, fi, "products16_independent")},
           "accumulated": {"ms": ma, "p99_ms": sorted(ta)[int(0.99 * (len(ta) - 1))], "value": n / (ma / 1e3),
                           "unit": UNIT, "alg_bytes": acc_bytes, "roofline": roofline_fracs(acc_bytes, acc_imad, ma),
                           "kernels": _kernel_trace(L, fa, "products16_accumulated")},
           "plain": {"ms": mp, "value": n / (mp / 1e3), "unit": UNIT, "launches": n,
                     "bit_exact_vs_batched": exact},
           "speedup_vs_plain": mp / mi}
    ctx.close()
    return res


def zp_rotations(L, stream, reps=20):
    """SecONNds-P's Z_P layer operations (Sec. 6.1, Sec. 2.1): key-switched slot
    rotations of a batch of ciphertexts, one multiply-accumulate-rotate pass, SIMD
    encoding and a 64 x 64 matrix-vector layer, N = 8192, three limbs plus one
    special prime, a 37-bit P. Key, ciphertexts and weights are uniform residues:
    the cost does not depend on the values."""
    import numpy as np
    import torch
    from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream, uniform_residues
    N, nl, n_ct, n_w = 8192, 3, 64, 16
    moduli, special = CANONICAL_PRIMES[:nl], CANONICAL_PRIMES[nl]
    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    s = Stream(5, 77)
    key_h = uniform_residues(s, moduli + (special,), (nl, 2), N)        # [L][2][L+1][N]
    key = L.hc_galois_key_create(ctx, special, 5, key_h, stream)
    cts = torch.from_numpy(uniform_residues(s, moduli, (n_ct, 2), N).view(np.int64)).cuda()
    rot = torch.empty_like(cts)
    w = torch.from_numpy(uniform_residues(s, moduli, (n_w,), N).view(np.int64)).cuda()
    acc = torch.empty(2 * nl * N, dtype=torch.int64, device="cuda")
    fr = lambda: L.hc_ct_rotate(ctx, key, cts, rot, stream)
    fm = lambda: L.hc_mac_rotate(ctx, key, cts[:2 * nl * N], w, acc, stream)
    for _ in range(3):
        fr()
        fm()
    tr, tm = _events_ms(fr, reps, stream), _events_ms(fm, reps, stream)
    out = {"workload": "zp_rotations_N8192_L3_special1_batch64_mac16", "rotations_per_call": n_ct,
           "rotate_ms": statistics.median(tr), "rotations_per_s": n_ct / (statistics.median(tr) / 1e3),
           "mac_rotate_terms": n_w, "mac_rotate_ms": statistics.median(tm),
           "mac_rotate_p99_ms": max(tm),
           "kernels_rotate": _kernel_trace(L, fr, "zp_rotate"), "kernels_mac_rotate": _kernel_trace(L, fm, "zp_mac")}
    # SIMD encoding of 256 slot vectors, and a 64 x 64 matrix-vector layer (diagonal method:
    # weights preprocessed once, then 64 products and 63 rotations per input ciphertext)
    P = zp_plain_prime(N)
    ctx_p = L.hc_ctx_create(N, [P], P)
    n_enc = 256
    slots = torch.from_numpy(s.below(P, n_enc * N).view(np.int64)).cuda()
    poly = torch.empty_like(slots)
    fe = lambda: L.hc_zp_encode(ctx_p, slots, poly, stream)
    fe()
    te = _events_ms(fe, reps, stream)
    Wm = s.below(P, 64 * 64).reshape(64, 64)
    wv = torch.empty(64 * nl * N, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_terms = L.hc_zp_matvec_preprocess(ctx, ctx_p, Wm, wv, stream)
    pre_s = time.perf_counter() - t0
    fv = lambda: L.hc_mac_rotate(ctx, key, cts[:2 * nl * N], wv, acc, stream)
    fv()
    tv = _events_ms(fv, max(3, reps // 4), stream)
    # the same layer for all 64 ciphertexts at once (hc_mac_rotate_many: one rotation chain)
    outs = torch.empty_like(cts)
    fb = lambda: L.hc_mac_rotate_many(ctx, key, cts, wv, outs, stream)
    fb()
    tb = _events_ms(fb, max(3, reps // 4), stream)
    out.update({"encode_vectors_per_call": n_enc, "encode_ms": statistics.median(te),
                "encodes_per_s": n_enc / (statistics.median(te) / 1e3),
                "matvec": {"n": n_terms, "preprocess_s": pre_s, "ms": statistics.median(tv),
                           "rotations": n_terms - 1, "products": n_terms,
                           "batch": n_ct, "batch_ms": statistics.median(tb),
                           "batch_vectors_per_s": n_ct / (statistics.median(tb) / 1e3)}})
    out["conv"] = zp_conv_section(L, stream, ctx, ctx_p, key, s, moduli, special, reps)
    ctx_p.close()
    key.close()
    ctx.close()
    return out


def zp_rotation_imad_eq(N, nl):
    """IMAD-equivalents of one key-switched rotation of one ciphertext: forward NTT of the
    L digits over L+1 moduli, the digit-key MAC, inverse NTT of 2(L+1) limbs, mod-down."""
    bfly = (N // 2) * (N.bit_length() - 1)
    return ((nl * (nl + 1) + 2 * (nl + 1)) * bfly * IMAD_EQ_BUTTERFLY
            + nl * 2 * (nl + 1) * N * IMAD_EQ_MAC_TERM + 2 * (nl + 1) * N * IMAD_EQ_REDUCE
            + 2 * nl * N * IMAD_EQ_BUTTERFLY)


def zp_conv_section(L, stream, ctx, ctx_p, key_1, s, moduli, special, reps):
    """SecONNds-P's convolution over Z_P (Sec. 6.1): SqueezeNet-1.1's fire2 expand 3x3
    layer (16 -> 64 channels, 55 x 55, pad 1) as the multiply-accumulate-rotate
    iteration at N = 8192, L = 3: 16 input ciphertexts, 32 output ciphertexts, 4608
    ct x pt products, 256 rotations.  Uniform residues stand in for the ciphertexts and
    the second Galois key; int8 weights mod P."""
    import numpy as np
    import torch
    from paper_2506_11586_gb300.inputs import uniform_residues
    N, nl = ctx.N, ctx.L
    C_, H, W, M, k, pad = 16, 55, 55, 64, 3, 1
    Wp = W + 2 * pad
    g_row = pow(5, Wp - k + 1, 2 * N)
    key_row = L.hc_galois_key_create(ctx, special, g_row,
                                     uniform_residues(s, moduli + (special,), (nl, 2), N), stream)
    desc = L.make_desc(C_, H, W, M, k, k, pad=pad)
    P = ctx_p.moduli[0]
    K = np.mod(s.int8(M * C_ * k * k).astype(np.int64).reshape(M, C_, k, k), P).astype(np.uint64)
    Y, kk = (M + 1) // 2, k * k
    n_plain = Y * kk * C_
    w = torch.empty(n_plain * nl * N, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.hc_zp_conv_preprocess(ctx, ctx_p, desc, K, w, stream)
    pre_s = time.perf_counter() - t0
    cts = torch.from_numpy(uniform_residues(s, moduli, (C_, 2), N).view(np.int64)).cuda()
    out = torch.empty(Y * 2 * nl * N, dtype=torch.int64, device="cuda")
    f = lambda: L.hc_zp_conv(ctx, desc, key_1, key_row, w, cts, out, stream)
    for _ in range(3):
        f()
    t = _events_ms(f, max(5, reps // 2), stream)
    ms = statistics.median(t)
    bfly = (N // 2) * (N.bit_length() - 1)
    poly = 8 * N * nl
    rot = Y * (kk - 1)
    nbytes = (poly * (2 * C_ + n_plain + 2 * Y) + (kk - 1) * (poly * 2 * Y * 3 + 8 * N * nl * 2 * (nl + 1)))
    imad = (2 * C_ * nl * bfly * IMAD_EQ_BUTTERFLY + n_plain * 2 * nl * N * IMAD_EQ_MAC_TERM
            + kk * Y * 2 * nl * N * IMAD_EQ_REDUCE + kk * Y * 2 * nl * bfly * IMAD_EQ_BUTTERFLY
            + rot * zp_rotation_imad_eq(N, nl))
    res = {"workload": "zp_conv_fire2_expand3x3_16to64_55x55_N8192_L3", "products": n_plain, "rotations": rot,
           "input_cts": C_, "output_cts": Y, "ms": ms, "p99_ms": max(t), "value": n_plain / (ms / 1e3),
           "unit": UNIT, "rotations_per_s": rot / (ms / 1e3), "preprocess_s": pre_s,
           "resident_weight_bytes": n_plain * poly, "alg_bytes": nbytes,
           "roofline": roofline_fracs(nbytes, imad, ms), "kernels": _kernel_trace(L, f, "zp_conv")}
    key_row.close()
    return res


def zp_plain_prime(N, bits=37):
    """The largest prime below 2^bits that is 1 mod 2N (SecONNds-P's 37-bit plaintext modulus)."""
    def is_prime(n):                       # deterministic Miller-Rabin for n < 3.3e24
        if n < 2:
            return False
        bases = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41)
        for b in bases:
            if n % b == 0:
                return n == b
        d, r = n - 1, 0
        while d % 2 == 0:
            d, r = d // 2, r + 1
        for b in bases:
            x = pow(b, d, n)
            if x in (1, n - 1):
                continue
            for _ in range(r - 1):
                x = x * x % n
                if x == n - 1:
                    break
            else:
                return False
        return True
    p = ((1 << bits) - 1) // (2 * N) * (2 * N) + 1
    while p >= (1 << bits) or not is_prime(p):
        p -= 2 * N
    return p


def run_gb300(args):
    import numpy as np
    import torch
    from paper_2506_11586_gb300 import replicas
    from paper_2506_11586_gb300.build import build
    build()
    from paper_2506_11586_gb300 import _lib as L
    from paper_2506_11586_gb300.inputs import T_PLAIN, Stream, conv_tensors, uniform_residues

    rank, world, local = replicas.init()
    torch.cuda.set_device(local)
    sh, N, moduli = workload_shape()
    nl = len(moduli)
    geo = geometry()
    _, K = conv_tensors(sh, seed=2)

    ctx = L.hc_ctx_create(N, moduli, T_PLAIN)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    w = L.hc_weights_preprocess(ctx, L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad), K)
    offline_s = time.perf_counter() - t0

    ct_host = uniform_residues(Stream(2, 5 + rank), moduli, (geo["I"], 2), N)
    d_in = torch.from_numpy(ct_host.view(np.int64)).cuda()
    d_out = torch.empty(geo["O"] * 2 * nl * N, dtype=torch.int64, device="cuda")
    tuned = None
    if not args.no_autotune:                # the library's autotuner, timed on this layer as a plan
        plan = L.hc_plan_create([L.work_conv(ctx, w, d_in, d_out)])
        L.hc_plan_autotune(plan, TUNE_CACHE)
        plan.close()
        tuned = {name: L.hc_ctx_get_variant(ctx, k) for name, k in KIND_NAMES.items()}
    if args.conv_form is not None:
        L.hc_ctx_set_variant(ctx, L.KIND_CONV_FORM, args.conv_form)
    if args.mac_variant is not None:
        L.hc_ctx_set_variant(ctx, L.KIND_MAC_CONV, args.mac_variant)
    flush = torch.empty(L2_FLUSH_BYTES // 8, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    def direct_step():
        L.hc_conv_ct_pt(ctx, w, d_in, d_out, stream)

    # the timed step: the layer as a one-item plan, replayed from the CUDA graph the
    # plan captures on its second run (--step-api direct: one hc_conv_ct_pt call)
    plan_step = None
    if args.step_api == "plan":
        plan_step = L.hc_plan_create([L.work_conv(ctx, w, d_in, d_out)])

        def step():
            L.hc_plan_run(plan_step, stream)
    else:
        step = direct_step

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    # the library's kernels per step, counted by its trace on one untimed step (the trace
    # records CUDA events around every launch, so it stays off in the timed region)
    L.hc_profile_collect()
    L.hc_profile_enable(True)
    direct_step()
    torch.cuda.synchronize()
    L.hc_profile_enable(False)
    launches_per_step = sum(v[0] for v in L.hc_profile_collect().values())
    if plan_step is not None:
        launches_per_step = L.hc_plan_info(plan_step)[2]

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    replicas.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)                        # let the sampler attach before the timed region
    torch.cuda.nvtx.range_push("timed_steps")  # profilers can select the timed launches by this range
    for k in range(args.steps):
        flush.zero_()                      # L2 flush between steps, outside the timed events
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    replicas.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    max_total_ms = replicas.reduce_max(total_ms)
    value = replicas.whole_job_throughput(geo["products"] * args.steps, world, max_total_ms / 1000.0)

    # roofline of the dominant kernel (largest share of device time in the trace).  The
    # per-kernel figures come from a second, traced pass of the same layer (same stream,
    # same L2 flush) in the form of one launch per phase: the timed region is not traced,
    # and the tuned form runs each limb's chain on its own stream, where kernels overlap
    # and a launch's duration no longer isolates its own work; the line says so.
    launches = launches_per_step * args.steps
    form = L.hc_ctx_get_variant(ctx, L.KIND_CONV_FORM)
    L.hc_ctx_set_variant(ctx, L.KIND_CONV_FORM, 0)
    rsteps = min(args.steps, 300)
    direct_step()
    torch.cuda.synchronize()
    L.hc_profile_collect()
    L.hc_profile_enable(True)
    rms = _events_ms(direct_step, rsteps, stream, flush)
    L.hc_profile_enable(False)
    rprof = L.hc_profile_collect()
    L.hc_ctx_set_variant(ctx, L.KIND_CONV_FORM, form)
    measured_with = ("a traced pass of %d direct calls with one launch per phase (%.4f ms per layer); "
                     "the timed region ran %s with launch form %d, untraced"
                     % (rsteps, statistics.median(rms),
                        "graph replays of a one-layer plan" if plan_step is not None else "direct calls", form))
    kname = max(rprof, key=lambda k: rprof[k][1])
    kl, kms = rprof[kname]
    k_avg_ms = kms / kl
    work = kernel_work(kname, geo, N, nl)
    bytes_layer = alg_bytes(geo, N, nl)
    hbm_peak, peak_kind = measured_peaks()
    alu_peak = alu_peak_imad_eq()
    hbm_achieved = work["bytes"] / (k_avg_ms / 1000.0) / 1e9
    alu_achieved = work["imad_eq"] / (k_avg_ms / 1000.0) / 1e12
    hbm_frac, alu_frac = hbm_achieved / hbm_peak, alu_achieved / alu_peak
    traffic = committed_traffic(kname)
    if alu_frac >= hbm_frac:
        roofline = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "T IMAD-eq/s",
                    "frac": alu_frac}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_frac}
    rtotal = sum(v[1] for v in rprof.values())
    roofline.update({"sms": device_sms(), "peak_sm_mhz": peak_sm_mhz(),
                     "sm_mhz_under_load": clocks["sm_mhz"] if clocks else None,
                     "peak_rule": "alu: 64 IMAD-eq per clock per SM x sms x peak_sm_mhz; hbm: measured copy",
                     "kernel": kname, "traffic": traffic, "hbm_gbs": hbm_achieved, "hbm_peak_gbs": hbm_peak,
                     "hbm_frac": hbm_frac, "hbm_peak_source": peak_kind, "alu_frac": alu_frac,
                     "alg_bytes_per_launch": work["bytes"], "alg_imad_eq_per_launch": work["imad_eq"],
                     "kernel_ms": k_avg_ms, "kernel_share": kms / rtotal if rtotal else None,
                     "measured_with": measured_with})
    layer_gbs = bytes_layer * args.steps / (total_ms / 1000.0) / 1e9

    # the other entry point on the same layer (same stream, same L2 flush): direct
    # hc_conv_ct_pt calls when the timed region replayed the plan, and vice versa
    alt = None
    if args.plain_steps > 0:
        if plan_step is not None:
            for _ in range(3):
                direct_step()
            gms = _events_ms(direct_step, 200, stream, flush)
            alt = {"api": "hc_conv_ct_pt (direct call)"}
        else:
            plan1 = L.hc_plan_create([L.work_conv(ctx, w, d_in, d_out)])
            for _ in range(3):
                L.hc_plan_run(plan1, stream)
            gms = _events_ms(lambda: L.hc_plan_run(plan1, stream), 200, stream, flush)
            plan1.close()
            alt = {"api": "hc_plan_run (one-layer plan, graph replay)"}
        alt.update({"ms_per_step": statistics.median(gms), "p99_ms": sorted(gms)[int(0.99 * (len(gms) - 1))],
                    "value": geo["products"] / (statistics.median(gms) / 1e3), "unit": UNIT})

    # plain one-launch-per-product path on the same inputs (comparison)
    plain = None
    if args.plain_steps > 0:
        d_plain = torch.empty_like(d_out)
        L.hc_conv_ct_pt_plain(ctx, w, d_in, d_plain, stream)
        torch.cuda.synchronize()
        bit_exact = bool(torch.equal(d_plain, d_out))
        pms = []
        for _ in range(args.plain_steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            L.hc_conv_ct_pt_plain(ctx, w, d_in, d_plain, stream)
            b.record(stream)
            torch.cuda.synchronize()
            pms.append(a.elapsed_time(b))
        plain = {"value": geo["products"] / (statistics.mean(pms) / 1000.0), "unit": UNIT,
                 "ms_per_step": statistics.mean(pms), "launches_per_step": geo["products"],
                 "bit_exact_vs_batched": bit_exact}

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if args.e2e_steps > 0:
        h_in = torch.from_numpy(ct_host.view(np.int64)).pin_memory()
        h_out = torch.empty(geo["O"] * 2 * nl * N, dtype=torch.int64).pin_memory()
        L.hc_conv_ct_pt_host(ctx, w, h_in, h_out, stream)
        ts = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            L.hc_conv_ct_pt_host(ctx, w, h_in, h_out, stream)   # H2D, layer, D2H, synchronise
            ts.append(time.perf_counter() - t0)
        e2e_s = replicas.reduce_max(sum(ts))
        e2e_exact = bool(torch.equal(h_out, d_out.cpu()))
        # the copies alone, for the bound: pinned host <-> device, same byte counts
        d_tmp = torch.empty_like(d_out)

        def copy_gbs(dst, src, nbytes):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(5):
                dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            return 5 * nbytes / (time.perf_counter() - t0) / 1e9
        h2d_gbs = copy_gbs(d_in.new_empty(d_in.shape), h_in, ct_host.nbytes)
        d2h_gbs = copy_gbs(h_out, d_tmp, h_out.numel() * 8)
        e2e = {"value": replicas.whole_job_throughput(geo["products"] * args.e2e_steps, world, e2e_s),
               "copy_h2d_gbs": h2d_gbs, "copy_d2h_gbs": d2h_gbs,
               "unit": UNIT, "h2d_bytes_per_step": int(ct_host.nbytes),
               "d2h_bytes_per_step": int(h_out.numel() * 8), "ms_per_step": 1000 * statistics.mean(ts),
               "bit_exact_vs_device": e2e_exact}

    # the server's whole step on the same layer: share add, convolution, output mask, slot extraction
    step_full = None
    if args.plain_steps > 0:
        s_share = torch.from_numpy(Stream(2, 90).below(T_PLAIN, sh.C * sh.H * sh.W).view(np.int64)).cuda()
        ho, wo = sh.H + 2 * sh.pad - sh.kh + 1, sh.W + 2 * sh.pad - sh.kw + 1
        s_mask = torch.from_numpy(Stream(2, 91).below(T_PLAIN, sh.M * ho * wo).view(np.int64)).cuda()
        n_slots = L.slot_count(w)
        d_slots = torch.empty(geo["O"] * nl * n_slots, dtype=torch.int64, device="cuda")
        d_full = torch.empty_like(d_out)
        fn = lambda: L.hc_conv_server_step(ctx, w, d_in, s_share, s_mask, d_full, d_slots, stream)
        for _ in range(3):
            fn()
        sms = _events_ms(fn, 50, stream, flush)
        step_full = {"ms_per_layer": statistics.median(sms), "value": geo["products"] / (statistics.median(sms) / 1e3),
                     "unit": UNIT, "slots_per_output": n_slots,
                     "returned_bytes": int(d_slots.numel() * 8 + geo["O"] * nl * N * 8)}
        # the same step with the extraction fused into the inverse NTT: c0 is never stored in full
        d_c1 = torch.empty(geo["O"] * nl * N, dtype=torch.int64, device="cuda")
        d_slots2 = torch.empty_like(d_slots)
        fs = lambda: L.hc_conv_server_step_sparse(ctx, w, d_in, s_share, s_mask, d_c1, d_slots2, stream)
        for _ in range(3):
            fs()
        sps = _events_ms(fs, 50, stream, flush)
        step_full["sparse"] = {
            "ms_per_layer": statistics.median(sps), "value": geo["products"] / (statistics.median(sps) / 1e3),
            "unit": UNIT, "bit_exact_vs_full_step": bool(torch.equal(d_slots2, d_slots)) and bool(
                torch.equal(d_c1.view(geo["O"], -1), d_full.view(geo["O"], 2, -1)[:, 1])),
            "kernels": _kernel_trace(L, fs, "server_step_sparse")}

    # the same layer with online NTT preprocessing and with none (Sec. 9's preprocessing modes)
    modes = None
    if args.plain_steps > 0:
        modes = {"offline_ntt_ms": max_total_ms / args.steps}
        for name, mode in (("online_ntt_ms", L.HC_WEIGHTS_NTT_ONLINE), ("no_ntt_ms", L.HC_WEIGHTS_NO_NTT)):
            wm = L.hc_weights_preprocess_ex(ctx, L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad), K,
                                            mode)
            d_m = torch.empty_like(d_out)
            fn = lambda: L.hc_conv_ct_pt(ctx, wm, d_in, d_m, stream)
            fn()
            ms = _events_ms(fn, 5 if mode == L.HC_WEIGHTS_NO_NTT else 20, stream, flush)
            modes[name] = statistics.median(ms)
            modes[name.replace("_ms", "_bit_exact")] = bool(torch.equal(d_m, d_out))
            wm.close()

    small = products16(L, stream, flush) if rank == 0 and not args.no_batched else None
    probe = int_probe(L, ctx, stream) if rank == 0 else None
    macs = mac_variants_section(L, ctx, w, d_in, d_out, stream, flush) if rank == 0 and not args.no_mac_variants \
        else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, outs, prods, el, threads = cpu_oracle_rate(args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d of %d output ciphertexts (%d products) of the same layer, %.1f s, set-up untimed"
                         % (outs, geo["O"], prods, el)}

    # serving first among the extra sections: replays of the Poisson trace in one process
    # drift upward run after run (host side; the GPU work per request stays constant), so
    # the trace the line reports is the first one the process replays
    serving = None
    if rank == 0 and args.serving_requests > 0:
        from paper_2506_11586_gb300 import serving as srv_mod
        layers = srv_mod.ServingLayers()
        serving = srv_mod.run(layers, n_requests=args.serving_requests, rate=args.serving_rate)
        serving.update({"workload": "poisson_squeezenet1.1_N8192L3_resnet50_N16384L4",
                        "setup_s": layers.setup_s, "resident_weight_bytes": layers.weight_bytes})
        # the same trace with every batch at the same stream priority (the comparison; it
        # replays second, so it carries one replay's drift)
        serving["equal_priority"] = srv_mod.run(layers, n_requests=max(1000, args.serving_requests // 2),
                                                rate=args.serving_rate, flags=L.HC_SERVER_EQUAL_PRIORITY)
        if args.serving_rate_high > 0:     # a rate at which requests queue and batches form
            serving["high_rate"] = srv_mod.run(layers, n_requests=max(1000, args.serving_requests * 2 // 3),
                                               rate=args.serving_rate_high)
        del layers
    batched = None
    if rank == 0 and not args.no_batched:
        wp = not args.no_batched_plain
        batched = {"squeezenet": batched_squeezenet(L, stream, args.batched_reps, wp),
                   "uneven": batched_uneven(L, stream, args.batched_reps, wp)}
    zp = None
    if rank == 0 and not args.no_zp:
        zp = zp_rotations(L, stream, max(5, args.batched_reps))
    networks = None
    if rank == 0 and not args.no_networks:
        networks = whole_networks(L, stream, max(5, args.batched_reps // 2))

    srt = sorted(step_ms)
    p99 = srt[min(len(srt) - 1, int(round(0.99 * (len(srt) - 1))))]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": max_total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": run_config(geo, N, nl, world),
        "step_api": ("hc_plan_run: one-layer plan replayed from a CUDA graph" if plan_step is not None
                     else "hc_conv_ct_pt: direct call"),
        "p50_ms": statistics.median(step_ms), "p99_ms": p99, "layer_gbs": layer_gbs,
        "roofline": roofline, "other_entry_point": alt, "plain": plain, "e2e": e2e, "cpu_baseline": cpu,
        "server_step": step_full, "preprocessing_modes": modes, "products16": small, "int_probe": probe,
        "mac_variants": macs,
        "batched": batched, "networks": networks, "zp": zp,
        "serving": serving, "gpu_launches": launches,
        "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in rprof.items()},
        "kernels_from": measured_with.split(";")[0],
        "launch_form": form,
        "offline_weights_s": offline_s, "launch_variants": tuned, "clocks": clocks, "device": torch.cuda.get_device_name(local),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if plan_step is not None:
        plan_step.close()
    w.close()
    ctx.close()
    replicas.shutdown()
    return 0


def profile_case(args):
    """A small, fixed case for ncu captures (a few launches, ~150 MB on the device)."""
    import numpy as np
    import torch
    from paper_2506_11586_gb300.build import build
    build()
    from paper_2506_11586_gb300 import _lib as L
    from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, T_PLAIN, Stream, uniform_residues
    N, nl = 8192, 3
    ctx = L.hc_ctx_create(N, CANONICAL_PRIMES[:nl], T_PLAIN)
    a = uniform_residues(Stream(9, 1), CANONICAL_PRIMES[:nl], (512,), N)
    d = torch.from_numpy(a.view(np.int64).reshape(-1)).cuda()
    s = torch.cuda.current_stream()
    for v in (2, 1):                        # persistent prefetching shape, then the one-CTA shape
        L.hc_ctx_set_variant(ctx, L.KIND_NTT_INV, v)
        L.hc_ntt_inv(ctx, d, s)
        L.hc_ntt_fwd(ctx, d, s)
    torch.cuda.synchronize()
    ok = bool(np.array_equal(d.cpu().numpy().view(np.uint64).reshape(a.shape), a))
    rate, ms, eq = L.hc_probe_int_rate(ctx, 0, 64, s)
    print(json.dumps({"profile_case": args.profile_case, "limbs": 512 * nl, "round_trip_exact": ok,
                      "shoup_ops_per_s": rate}), flush=True)
    return 0 if ok else 1


def main():
    args = parse()
    if args.profile_case:
        return profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
