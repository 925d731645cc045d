#!/usr/bin/env python
"""Benchmark of the homomorphic-convolution hot path (SecONNds, arXiv 2506.11586, Sec. 6.2).

One step = one online HE convolution layer through the C ABI (hc_conv_ct_pt):
forward NTT of every input ciphertext, NTT-domain multiply-accumulate against
the resident NTT-preprocessed weights, inverse NTT of the outputs.  Workload:
56x56x64 activations -> 64 output channels, 3x3, stride 1, pad 1, packed into
N = 8192 polynomials over three 50-bit primes (I = 32 input ciphertexts,
P = 512 weight plaintexts, O = 256 output ciphertexts, 2048 ct x pt products).
Inputs are seeded synthetic residues uniform in [0, q_i) (the cost does not
depend on the values); weights are seeded uniform int8.

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
    return ap.parse_args()


def workload_shape():
    from paper_2506_11586_gb300.inputs import CANONICAL_PRIMES, CONV_56x56x64
    return CONV_56x56x64, 8192, CANONICAL_PRIMES[:3]


def geometry():
    from paper_2506_11586_gb300 import _lib as L
    sh, N, moduli = workload_shape()
    res, I, P, O = L.hc_conv_partition(L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad), N)
    G = (sh.C + res.Cw - 1) // res.Cw
    B = I // G
    return dict(I=I, P=P, O=O, G=G, B=B, products=sh.M * G * B, Cw=res.Cw, Hw=res.Hw, Ww=res.Ww)


def alg_bytes(geo, N, L):
    """Algorithmic HBM bytes of one layer: read 2I input polys, P weights, write 2O outputs."""
    return 8 * N * L * (2 * geo["I"] + geo["P"] + 2 * geo["O"])


# Integer-pipe cost model (measured on GB300 with ncu counters): the fmaheavy
# pipe runs 64 32-bit multiply-adds per clock per SM; a 32x32->64 multiply
# (mad.wide.u32) occupies it twice as long.  In these units a lazy Shoup
# multiplication (5 wide + 4 narrow) costs 14, a MAC term (4 wide) 8 and the
# final reduction of a MAC sum (one Shoup + one w=1 reduction) 19.
IMAD_EQ_BUTTERFLY, IMAD_EQ_MAC_TERM, IMAD_EQ_REDUCE = 14, 8, 19


def alu_peak_imad_eq():
    """T IMAD-equivalents/s: 64 per clock per SM at the maximum SM clock."""
    mhz, sms = 2070.0, 152
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return 64 * sms * mhz * 1e6 / 1e12


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
    if name.startswith("k_mac_conv"):
        return {"bytes": poly * (2 * I + P + 2 * O), "imad_eq": mac}
    # fused MAC + inverse NTT
    return {"bytes": poly * (2 * I + P + 2 * O), "imad_eq": mac + 2 * O * L * bfly * IMAD_EQ_BUTTERFLY}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_hash():
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2506_11586_gb300", "csrc", "*"))):
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


def cpu_oracle_rate(seconds, seed=2, max_outputs=None):
    """Oracle convolution (plain schoolbook) of as many output ciphertexts as fit in
    ~`seconds`; returns (products/s, outputs done, products done, elapsed, threads)."""
    import numpy as np
    from oracle import conv
    from paper_2506_11586_gb300.inputs import Stream, conv_tensors, uniform_residues
    sh, N, moduli = workload_shape()
    _, K = conv_tensors(sh, seed=seed)
    p = conv.canonical_partition(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, sh.pad, N)
    ct = uniform_residues(Stream(seed, 5), moduli, (p.I, 2), N)
    Kp = conv.pack_weights(K.astype(np.int64), p)
    order = Stream(seed, 6).u64(p.O).argsort()
    done, t0 = 0, time.perf_counter()
    while done < p.O and (max_outputs is None or done < max_outputs):
        conv.conv_ct_pt(ct, Kp, p, moduli, outputs=[int(order[done])])
        done += 1
        if max_outputs is None and time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return done * p.G / el, done, done * p.G, el, threads


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    geo = geometry()
    from oracle import build_oracle
    build_oracle()
    per_step_outputs = 2
    for _ in range(args.warmup):
        cpu_oracle_rate(0, max_outputs=per_step_outputs)
    times = []
    products = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, _, prods, _, threads = cpu_oracle_rate(0, max_outputs=per_step_outputs)
        times.append(time.perf_counter() - t0)
        products += prods
    total = sum(times)
    value = products / total
    sample = ("%d of %d output ciphertexts per step (%d products), schoolbook oracle"
              % (per_step_outputs, geo["O"], per_step_outputs * geo["G"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "products_per_layer": geo["products"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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
    tuned = None
    if not args.no_autotune:
        from paper_2506_11586_gb300.autotune import autotune
        tuned = autotune(ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    w = L.hc_weights_preprocess(ctx, L.make_desc(sh.C, sh.H, sh.W, sh.M, sh.kh, sh.kw, pad=sh.pad), K)
    offline_s = time.perf_counter() - t0

    ct_host = uniform_residues(Stream(2, 5 + rank), moduli, (geo["I"], 2), N)
    d_in = torch.from_numpy(ct_host.view(np.int64)).cuda()
    d_out = torch.empty(geo["O"] * 2 * nl * N, dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 8, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        L.hc_conv_ct_pt(ctx, w, d_in, d_out, stream)

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    replicas.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)                        # let the sampler attach before the timed region
    L.hc_profile_collect()
    L.hc_profile_enable(True)
    for k in range(args.steps):
        flush.zero_()                      # L2 flush between steps, outside the timed events
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    L.hc_profile_enable(False)
    replicas.barrier()
    clocks = sampler.stop()
    prof = L.hc_profile_collect()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    max_total_ms = replicas.reduce_max(total_ms)
    value = replicas.whole_job_throughput(geo["products"] * args.steps, world, max_total_ms / 1000.0)

    # roofline of the dominant kernel (largest share of device time in the trace)
    launches = sum(v[0] for v in prof.values())
    kname = max(prof, key=lambda k: prof[k][1])
    kl, kms = prof[kname]
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
    roofline.update({"kernel": kname, "traffic": traffic, "hbm_gbs": hbm_achieved, "hbm_peak_gbs": hbm_peak,
                     "hbm_frac": hbm_frac, "hbm_peak_source": peak_kind, "alu_frac": alu_frac,
                     "alg_bytes_per_launch": work["bytes"], "alg_imad_eq_per_launch": work["imad_eq"],
                     "kernel_ms": k_avg_ms, "kernel_share": kms / total_ms if total_ms else None})
    layer_gbs = bytes_layer * args.steps / (total_ms / 1000.0) / 1e9

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
        e2e = {"value": replicas.whole_job_throughput(geo["products"] * args.e2e_steps, world, e2e_s),
               "unit": UNIT, "h2d_bytes_per_step": int(ct_host.nbytes),
               "d2h_bytes_per_step": int(h_out.numel() * 8), "ms_per_step": 1000 * statistics.mean(ts),
               "bit_exact_vs_device": bool(torch.equal(h_out, d_out.cpu()))}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, outs, prods, el, threads = cpu_oracle_rate(args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d of %d output ciphertexts (%d products) of the same layer, %.1f s"
                         % (outs, geo["O"], prods, el)}

    srt = sorted(step_ms)
    p99 = srt[min(len(srt) - 1, int(round(0.99 * (len(srt) - 1))))]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": max_total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "L": nl, "I": geo["I"], "P": geo["P"], "O": geo["O"],
                   "products_per_layer": geo["products"], "partition": [geo["Cw"], geo["Hw"], geo["Ww"]],
                   "parallelism": "replicas" if world > 1 else "single", "l2": "flushed between steps"},
        "p50_ms": statistics.median(step_ms), "p99_ms": p99, "layer_gbs": layer_gbs,
        "roofline": roofline, "plain": plain, "e2e": e2e, "cpu_baseline": cpu,
        "gpu_launches": launches, "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()},
        "offline_weights_s": offline_s, "launch_variants": tuned, "clocks": clocks, "device": torch.cuda.get_device_name(local),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    w.close()
    ctx.close()
    replicas.shutdown()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
