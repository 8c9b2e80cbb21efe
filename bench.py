#!/usr/bin/env python
"""Benchmark: encrypted-CNN images/s at N = 2^16 (RNS-CKKS on one GB300).

One step is one encrypted inference of the three-layer CNN
conv 8x5x5 stride 2 -> x^2 -> conv 16x3x3 stride 2 -> x^2 -> FC 10
over one batch of 128x128 images packed into the column layout (w = 128
ciphertexts of h = 128 pixels; `--batch` images side by side in blocks of
128 slots, 256 fills the 32768 slots). Ring degree N = 2^16, Q = 60 + 12 x 45
bits, P = 2 x 60 bits, key-switching digits of two primes, scale 2^45.

The step covers every row of the path: hoisted rotations with hybrid key
switching, the ciphertext-scalar multiply-accumulate of the convolutions,
ciphertext-ciphertext products with relinearisation, rescales, ciphertext-
plaintext products and rotate-and-add of the dense layer, all on the NTT
engine. Inputs are synthetic (seeded), already encrypted and resident in
device memory when the timed region starts; they are larger than L2.

The default run (N = 1) also measures the other configurations of the
method, each in a process of its own after the CNN's measurement (which
releases its device memory first), and reports each
JSON line whole under "workloads": 4096 small matmuls A(4x8) B(8x4) at
N = 2^13 (plain calls, one batched call, its CUDA graph); one conv + x^2 layer
on 64x64 images at N = 2^15; 64 matmuls of uneven m, n, p at N = 2^16
(zero-rotation layout, baby-step giant-step, batched and plain revolver); a
Poisson stream of CNN requests of sides 64/128/256 served by continuous
batching against one request at a time (p50/p99). Each carries its own
clock record and oracle baseline. --no-extra skips them.

--impl reference times the CPU oracle (oracle/) on a bounded sample of the
same workload on the host cores and reports the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from inputs import synthetic  # noqa: E402

METRIC = "encrypted-CNN images/s (N=2^16, 128x128, conv5x5s2x8-x2-conv3x3s2x16-x2-fc10)"
UNIT = "images/s"
SIDE = 128
H = 128  # block stride (rows per image block)
ROT_STEPS = [1, 2, 3, 4, 8, 16, 32, 64]
CNN_PRESETS = {"cnn_n16": synthetic.CNN_N16, "cnn_n16_dnum3": synthetic.CNN_N16_DNUM3}
KS_DESC = {"cnn_n16": "P=2x60, alpha=2 (7 digits)",
           "cnn_n16_dnum3": "P=5x60, dnum=3 (alpha=5: the stated dnum with a special modulus above the digits)"}
WORKLOAD = ("encrypted CNN conv5x5s2(8)->x^2->conv3x3s2(16)->x^2->fc10 on 128x128 grayscale images in the "
            "column layout (128 ciphertexts of 128 pixels); RNS-CKKS N=2^16, Q=60+12x45, P=2x60, alpha=2 (7 digits), "
            "scale 2^45")


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def rank_seeds(rank: int) -> dict:
    """Each rank encrypts its own batch: distinct keys and images, same weights."""
    return {"ctx_seed": 1000 + rank, "image_seed": 301 + rank, "weight_seed": 302}


def max_over_ranks(x: float, world: int) -> float:
    """The slowest rank's time (gloo all-reduce on CPU; no data-path collective)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(images_per_step: int, steps: int, world: int, t_max_s: float) -> float:
    """Whole-job images/s: every rank processed images_per_step * steps images."""
    return images_per_step * steps * world / t_max_s


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "fallback": True}


def profile_read(lib):
    import ctypes
    n = ctypes.c_int()
    names = ctypes.create_string_buffer(1 << 16)
    ms = (ctypes.c_double * 256)()
    cnt = (ctypes.c_uint64 * 256)()
    by = (ctypes.c_double * 256)()
    pr = (ctypes.c_double * 256)()
    rc = lib.he_profile_read(names, len(names), ms, cnt, by, pr, 256, ctypes.byref(n))
    assert rc == 0
    nm = names.value.decode().split("\n")[: n.value]
    return {nm[i]: {"ms": ms[i], "launches": int(cnt[i]), "bytes": by[i], "products": pr[i]}
            for i in range(n.value)}


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def ncu_traffic(kernel: str, alg_bytes_per_launch: float):
    """DRAM bytes per launch from the committed ncu capture of this kernel, scaled
    from the captured launch to this launch by algorithmic bytes (None if absent)."""
    try:
        t = json.load(open(TRAFFIC_FILE)).get(kernel)
    except (OSError, ValueError):
        return None
    if not t:
        return None
    return t["dram_bytes"] / t["alg_bytes"] * alg_bytes_per_launch


MAC96_KERNELS = ("k_conv_mac96_kernel", "k_fc_mac96_kernel")


def alu_peak_for(name, modmul_peak, mac96_peak, bfly_peak=None):
    """(products/s, unit, source) of the kernel's own product: the 96-bit multiply-accumulate for the
    kernels built on it, the growing-range butterfly of the 45-bit primes for the transforms (most of
    their rows; the 60-bit rows run Harvey's slower butterfly, reported beside it), else the Shoup
    product."""
    if name.startswith(MAC96_KERNELS):
        return mac96_peak, "Gmac96/s", "measured (he_calibrate_mac96: 96-bit multiply-accumulates in registers, all SMs)"
    if bfly_peak and name.startswith("k_ntt_"):
        return bfly_peak, "Gbfly/s", ("measured (he_calibrate_butterfly, narrow primes: growing-range butterflies in "
                                      "registers, all SMs)")
    return modmul_peak, "Gmodmul/s", "measured (he_calibrate_modmul: Shoup products in registers, all SMs)"


def roofline_for(name, t, total_ms, hbm, measured, modmul_peak, log_n, mac96_peak=None, bfly_peak=None):
    """The kernel's bound is whichever takes longer at peak: its algorithmic bytes at the measured HBM
    bandwidth, or its products at the measured rate of that product (he_calibrate_modmul for Shoup
    products, he_calibrate_mac96 for 96-bit multiply-accumulates)."""
    alu_peak, alu_unit, alu_src = alu_peak_for(name, modmul_peak, mac96_peak or modmul_peak, bfly_peak)
    avg_s = t["ms"] / 1e3 / max(1, t["launches"])
    alg_per_launch = t["bytes"] / max(1, t["launches"])
    prod_per_launch = t.get("products", 0.0) / max(1, t["launches"])
    gbs = alg_per_launch / avg_s / 1e9 if avg_s > 0 else 0.0
    base = {"kernel": name, "share_of_device_time": round(t["ms"] / total_ms, 4), "launches": t["launches"],
            "avg_launch_us": round(avg_s * 1e6, 2),
            "alg_bytes_per_launch": alg_per_launch, "modmul_per_launch": prod_per_launch,
            "hbm_view": {"achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4),
                         "peak_source": "measured" if measured else "fallback"}}
    traffic = ncu_traffic(name, alg_per_launch)
    if prod_per_launch / alu_peak > alg_per_launch / (hbm * 1e9):
        ach = prod_per_launch / avg_s / 1e9
        peak = alu_peak / 1e9
        base.update({"bound": "alu", "achieved": round(ach, 1), "peak": round(peak, 1), "unit": alu_unit,
                     "frac": round(ach / peak, 4), "traffic": traffic, "peak_source": alu_src})
    else:
        base.update({"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(gbs / hbm, 4), "traffic": traffic,
                     "peak_source": "measured" if measured else "fallback"})
    return base


def cnn_step(g, x, w, pts):
    y = g.conv2d(x, 1, 1, w.conv1_w, w.conv1_b, 2)
    g.square(y)
    y = g.conv2d(y, 8, 2, w.conv2_w, w.conv2_b, 2)
    g.square(y)
    return g.fc_apply(y, pts, w.fc_b)


def run_gpu(args, rank, world, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_18646_gb300 import api, load

    lib = load()
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.Stream()
    pre = CNN_PRESETS[args.preset]
    seeds = rank_seeds(rank)
    g = api.Context.from_preset(pre, seed=seeds["ctx_seed"], stream=stream.cuda_stream)
    if getattr(args, 'no_tensor_cores', False):
        g.set_tensor_cores(False)  # the convolutions' multiply-accumulate on the CUDA cores
    g.keygen(ROT_STEPS)
    B = args.batch
    h1, h2 = synthetic.cnn_shapes(SIDE)
    w = synthetic.cnn_weights(SIDE, seed=seeds["weight_seed"])
    imgs = synthetic.images(B, SIDE, SIDE, seed=seeds["image_seed"])
    x = g.encrypt_image(imgs, H, ct_id_base=0)
    fc_limbs = pre_limbs = len(pre.q_bits) - 4
    pts = g.fc_prepare(w.fc_w, 16, h2, h2, 4, H, B, fc_limbs)
    # transform geometry tuned on a ModUp-sized batch (128 ciphertexts x 13 limbs), outside timing
    tune_rows = 128 * len(pre.q_bits)
    n1, cols, tune_us = g.ntt_autotune(tune_rows)
    g.synchronize()

    def step():
        return cnn_step(g, x, w, pts)

    for _ in range(args.warmup):
        z = step()
    g.synchronize()
    launches0 = lib.he_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        g.synchronize()
        torch.cuda.nvtx.range_push("timed_steps")
        e0.record(stream)
        for _ in range(args.steps):
            z = step()
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        e1.synchronize()
        g.synchronize()
        torch.cuda.synchronize()
    launches = lib.he_kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    t_max = max_over_ranks(ms, world)
    value = job_throughput(B, args.steps, world, t_max / 1e3)

    # the last step's logits, checked against the FP64 CNN by the CPU leg (outside timing)
    logits = g.decrypt_slots(z)[:, ::H][:, :B].T

    # measured right after the device-timed steps, before the profiling and calibration runs
    # end to end through the C ABI: host ciphertexts in (pinned), encrypted logits out
    e2e = None
    if not args.no_e2e:
        host_in = x.export()
        pin_in = torch.from_numpy(host_in).pin_memory()
        pin_arr = pin_in.numpy()
        out_words = 10 * 2 * (fc_limbs - 1) * g.N
        pin_out = [torch.empty(out_words, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
                   for _ in range(2)]
        # the context's two import staging buffers are allocated by its first overlapped imports
        for _ in range(2):
            g.import_coeffs_async(pin_arr, g.scale).free()
        g.synchronize()
        clk_e2e = ClockSampler(local_rank).__enter__()
        t0 = time.perf_counter()
        # each step's ciphertexts are uploaded while the previous step computes (he_ctset_import_async
        # copies on a stream of its own); each step's logits are exported behind it
        # (he_ctset_export_async, two host buffers in turn) and waited for once the next step is
        # queued, so the host queues step i + 1 while step i runs
        xin = g.import_coeffs_async(pin_arr, g.scale)
        prev = 0
        for i in range(args.steps):
            zz = cnn_step(g, xin, w, pts)
            xnext = g.import_coeffs_async(pin_arr, g.scale) if i + 1 < args.steps else None
            ticket = zz.export_async(pin_out[i % 2])
            del zz
            if prev:
                g.export_wait(prev)  # step i - 1's logits are on the host
            prev = ticket
            xin = xnext
        g.export_wait(prev)
        g.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, world)
        clk_e2e.__exit__()
        e2e = {"value": round(job_throughput(B, args.steps, world, t_e2e), 3), "unit": UNIT,
               "h2d_bytes_per_step": int(pin_arr.nbytes), "d2h_bytes_per_step": int(out_words * 8),
               "ms_per_step": round(1e3 * t_e2e / args.steps, 3), "clocks": clk_e2e.summary()}

    # the same step on one image per ciphertext set (same ciphertext count, same kernels)
    x1 = g.encrypt_image(imgs[:1], H, ct_id_base=0)
    cnn_step(g, x1, w, pts)
    g.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        cnn_step(g, x1, w, pts)
    e1.record(stream)
    e1.synchronize()
    plain_ms = max_over_ranks(e0.elapsed_time(e1), world)
    x1.free()

    # per-kernel device time with CUDA events on the launching stream
    lib.he_profile_enable(1)
    for _ in range(args.steps):
        step()
    g.synchronize()
    prof = profile_read(lib)
    lib.he_profile_enable(0)
    prof_total = sum(v["ms"] for v in prof.values())
    top = max(prof, key=lambda k: prof[k]["ms"])
    pk = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    import ctypes
    modmul_peak, mac96_peak = ctypes.c_double(), ctypes.c_double()
    bfly_n, bfly_w = ctypes.c_double(), ctypes.c_double()
    lib.he_calibrate_modmul(g.h, ctypes.byref(modmul_peak))
    lib.he_calibrate_mac96(g.h, ctypes.byref(mac96_peak))
    lib.he_calibrate_butterfly(g.h, 1, ctypes.byref(bfly_n))
    lib.he_calibrate_butterfly(g.h, 0, ctypes.byref(bfly_w))
    roofline = roofline_for(top, prof[top], prof_total, hbm, "fallback" not in pk, modmul_peak.value, pre.log_n,
                            mac96_peak.value, bfly_n.value)

    def entry(k, v):
        e = {"share": round(v["ms"] / prof_total, 4), "ms_per_step": round(v["ms"] / args.steps, 3),
             "launches_per_step": v["launches"] // args.steps,
             "GBps": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else 0.0,
             "hbm_frac": round(v["bytes"] / (v["ms"] / 1e3) / 1e9 / hbm, 3) if v["ms"] > 0 else 0.0,
             "alu_frac": round(v["products"] / (v["ms"] / 1e3) /
                               alu_peak_for(k, modmul_peak.value, mac96_peak.value, bfly_n.value)[0], 3)
             if v["ms"] > 0 else 0.0}
        if k.startswith("k_ntt_") and v["ms"] > 0:
            # the same products against Harvey's butterfly of the 60-bit rows (the slower class)
            e["alu_frac_wide_bfly"] = round(v["products"] / (v["ms"] / 1e3) / bfly_w.value, 3)
        return e
    breakdown = {k: entry(k, v) for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}

    clocks = clk.summary()
    return {
        "value": value, "ms_per_step": t_max / args.steps, "launches": launches // args.steps * args.steps,
        "roofline": roofline, "breakdown": breakdown, "e2e": e2e, "clocks": clocks, "logits": logits, "imgs": imgs, "weights": w,
            "ntt_geometry": {"column_stages": n1, "columns_per_block": cols, "tuned_on_limbs": tune_rows,
                             "fwd_inv_us": round(tune_us, 1)},
        "images_per_step": B, "modmul_peak": modmul_peak.value, "mac96_peak": mac96_peak.value,
        "bfly_peak": {"narrow": bfly_n.value, "wide": bfly_w.value},
        "plain_value": job_throughput(1, args.steps, world, plain_ms / 1e3),
        "plain_ms": plain_ms / args.steps,
    }


# ---------------------------------------------------------------------------
# the batched-matmul workload (--workload matmul)
# ---------------------------------------------------------------------------
MATMUL_METRIC = "HE-matmul/s (64 matmuls, m,n,p uniform over {16,32,64,128,256}, N=2^16)"


def run_matmul(args, rank, world, local_rank):
    """64 independent encrypted matmuls at the CNN parameters (top level, 13 limbs).

    Operands are encrypted (untimed) in waves that fit device memory; each wave
    is evaluated as 64-way-style batched launches (he_matmul_batched), as one
    he_matmul call per product, as one baby-step giant-step he_matmul_bsgs call per
    product, all timed with CUDA events on the context's stream, and in the
    zero-rotation layout (A encrypted with he_encrypt_matrix_a_volley, one
    he_matmul_volley per product).
    value = products / total zero-rotation time; the revolver figures are reported beside it."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_18646_gb300 import api, load
    lib = load()
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.Stream()
    pre = synthetic.CNN_N16
    g = api.Context.from_preset(pre, seed=4000 + rank, stream=stream.cuda_stream)
    if getattr(args, 'no_tensor_cores', False):
        g.set_tensor_cores(False)  # the convolutions' multiply-accumulate on the CUDA cores
    shapes = synthetic.batched_matmul_shapes(64, seed=401)
    if args.count:
        shapes = shapes[: args.count]
    t0 = time.perf_counter()
    S = (1 << pre.log_n) // 2
    bsgs_steps = set()
    for _, _, p in shapes:
        gb_ = 1
        while 4 * gb_ * gb_ <= 2 * p:
            gb_ *= 2
        gb_ = min(gb_, p)
        bsgs_steps |= {S - gb_ * i for i in range(1, -(-p // gb_))}
    g.keygen(sorted(set(range(1, max(p for _, _, p in shapes))) | bsgs_steps))
    g.synchronize()
    keygen_s = time.perf_counter() - t0
    ct_bytes = 2 * len(pre.q_bits) * g.N * 8
    budget = 96 << 30
    waves, cur, used = [], [], 0
    for i, (m, n, p) in enumerate(shapes):
        need = (1 + max(2, api.volley_geometry(g.N // 2, m, p)[2])) * n * ct_bytes
        if cur and used + need > budget:
            waves.append(cur)
            cur, used = [], 0
        cur.append(i)
        used += need
    if cur:
        waves.append(cur)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        g.synchronize()
        ev0.record(stream)
        r = fn()
        ev1.record(stream)
        ev1.synchronize()
        return r, ev0.elapsed_time(ev1) / 1e3

    # warm-up: one small product through both paths
    wa = g.encrypt_matrix_a(np.ones((4, 4)), 0)
    wb = g.encrypt_matrix_b(np.ones((4, 4)), 100)
    g.matmul(wa, wb, 4, 4)
    g.matmul_batched([wa], [wb], [4], [4])
    g.matmul_volley(g.encrypt_matrix_a_volley(np.ones((4, 4)), 4, 0), wb)
    t_batched = t_plain = t_volley = t_bsgs = 0.0
    launches_b = launches_v = 0
    wave0_prof = {}
    max_err = max_err_v = 0.0
    rng_seed = 402
    clk = ClockSampler(local_rank).__enter__()
    for wave in waves:
        As, Bs, mats = [], [], []
        for i in wave:
            m, n, p = shapes[i]
            A, Bm = synthetic.matmul_operands(m, n, p, seed=rng_seed + i)
            As.append(g.encrypt_matrix_a(A, 10 ** 6 * i))
            Bs.append(g.encrypt_matrix_b(Bm, 10 ** 6 * i + 5 * 10 ** 5))
            mats.append(A @ Bm)
        ms = [shapes[i][0] for i in wave]
        ps = [shapes[i][2] for i in wave]
        l0 = lib.he_kernel_launches()
        outs, dt = timed(lambda: g.matmul_batched(As, Bs, ms, ps))
        launches_b += lib.he_kernel_launches() - l0
        t_batched += dt
        for t in (0, len(wave) - 1):
            max_err = max(max_err, float(np.abs(g.decrypt_matrix(outs[t], ms[t], ps[t]) - mats[t]).max()))
        del outs

        def plain():
            res = []
            for t in range(len(wave)):
                res.append(g.matmul(As[t], Bs[t], ms[t], ps[t]))
                del res[-1]
            return None
        _, dt = timed(plain)
        t_plain += dt
        if wave is waves[0]:
            # where the time goes in both revolver modes: per-kernel device time (CUDA events per
            # launch) against the elapsed time of the same call, repeated once with the profiler on
            for mode, fn in (("batched", lambda: g.matmul_batched(As, Bs, ms, ps)), ("plain", plain)):
                profile_read(lib)
                lib.he_profile_enable(1)
                r_, dt_ = timed(fn)
                del r_
                prof = profile_read(lib)
                lib.he_profile_enable(0)
                dev = sum(v["ms"] for v in prof.values())
                top = sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:4]
                wave0_prof[mode] = {"products": len(wave), "elapsed_ms": round(1e3 * dt_, 1),
                                    "kernel_ms": round(dev, 1), "busy_frac": round(dev / (1e3 * dt_), 3),
                                    "launches": int(sum(v["launches"] for v in prof.values())),
                                    "top_kernels_ms": {k: round(v["ms"], 1) for k, v in top}}

        def bsgs():
            for t in range(len(wave)):
                r = g.matmul_bsgs(As[t], Bs[t], ms[t], ps[t])
                del r
            return None
        _, dt = timed(bsgs)
        t_bsgs += dt
        del As
        # the zero-rotation form: A in the volley layout (G groups of n ciphertexts), same B
        Vs = []
        for i in wave:
            m, n, p = shapes[i]
            A, _ = synthetic.matmul_operands(m, n, p, seed=rng_seed + i)
            Vs.append(g.encrypt_matrix_a_volley(A, p, 10 ** 6 * i + 2 * 10 ** 5))
        l0 = lib.he_kernel_launches()

        def volley():
            res = []
            for t in range(len(wave)):
                res.append(g.matmul_volley(Vs[t], Bs[t]))
            return res
        vouts, dt = timed(volley)
        launches_v += lib.he_kernel_launches() - l0
        t_volley += dt
        for t in range(len(wave)):
            max_err_v = max(max_err_v, float(np.abs(g.decrypt_matrix_volley(vouts[t], ms[t], ps[t]) - mats[t]).max()))
        del vouts, Vs, Bs
    clk.__exit__()
    total = len(shapes)
    t_b = max_over_ranks(t_batched, world)
    t_p = max_over_ranks(t_plain, world)
    t_v = max_over_ranks(t_volley, world)
    rot = sum(n * (p - 1) for _, n, p in shapes)
    groups = [api.volley_geometry(g.N // 2, m, p)[2] for m, _, p in shapes]
    return {"value": total * world / t_v, "ms_per_step": 1e3 * t_v, "launches": launches_v, "max_abs_err": max_err_v,
            "revolver_batched_value": total * world / t_b, "revolver_batched_ms": 1e3 * t_b,
            "revolver_plain_value": total * world / t_p, "revolver_plain_ms": 1e3 * t_p,
            "bsgs_value": total * world / max_over_ranks(t_bsgs, world), "bsgs_ms": 1e3 * max_over_ranks(t_bsgs, world),
            "revolver_launches": launches_b, "revolver_max_abs_err": max_err, "keygen_s": keygen_s,
            "waves": len(waves), "revolver_rotations": rot, "revolver_tensors": sum(n * p for _, n, p in shapes),
            "volley_tensors": sum(G * n for G, (_, n, _) in zip(groups, shapes)), "volley_rotations": 0,
            "clocks": clk.summary(), "shapes": shapes, "revolver_wave0_profile": wave0_prof}


# ---------------------------------------------------------------------------
# many small products (--workload matmul_small): plain calls, one batched call, its CUDA graph
# ---------------------------------------------------------------------------
MATMUL_SMALL_METRIC = "HE-matmul/s (4096 matmuls A(4x8) B(8x4), N=2^13), plain vs batched vs CUDA graph"


def run_matmul_small(args, rank, world, local_rank):
    """4096 independent products of the small matmul configuration (N = 2^13, Q = 60 + 40 + 40,
    P = 60, scale 2^40, n = 8 ciphertexts per operand): one he_matmul call per product (plain),
    one he_matmul_batched call over all of them, and that call captured once into a CUDA graph
    and replayed. Operands encrypted (untimed) up front; each path timed with CUDA events on the
    context's stream over args.steps repetitions after args.warmup."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_18646_gb300 import api, load
    lib = load()
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.Stream()
    pre = synthetic.MATMUL_SMALL
    g = api.Context.from_preset(pre, seed=5000 + rank, stream=stream.cuda_stream)
    if getattr(args, 'no_tensor_cores', False):
        g.set_tensor_cores(False)  # the convolutions' multiply-accumulate on the CUDA cores
    g.keygen([1, 2, 3])
    count = args.count or 4096
    m, n, p = 4, 8, 4
    mats, As, Bs = [], [], []
    for t in range(count):
        A, Bm = synthetic.matmul_operands(m, n, p, seed=101 + 7919 * t)
        mats.append(A @ Bm)
        As.append(g.encrypt_matrix_a(A, 100 * t))
        Bs.append(g.encrypt_matrix_b(Bm, 100 * t + 50))
    ms, ps = [m] * count, [p] * count
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        g.synchronize()
        l0 = lib.he_kernel_launches()
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / 1e3 / reps, (lib.he_kernel_launches() - l0) / reps

    def plain():
        for t in range(count):
            r = g.matmul(As[t], Bs[t], m, p)
            del r

    def batched():
        r = g.matmul_batched(As, Bs, ms, ps)
        del r

    for _ in range(max(1, args.warmup)):
        batched()
    g.synchronize()
    g.graph_begin()
    outs = g.matmul_batched(As, Bs, ms, ps)
    graph = g.graph_end()
    for _ in range(max(1, args.warmup)):
        graph.launch()
    with ClockSampler(local_rank) as clk:
        t_plain, l_plain = timed(plain, 1)
        t_batched, l_batched = timed(batched, max(1, args.steps))
        t_graph, l_graph = timed(graph.launch, max(1, args.steps))
    g.synchronize()
    err = max(float(np.abs(g.decrypt_matrix(outs[t], m, p) - mats[t]).max()) for t in (0, count // 2, count - 1))
    graph.destroy()
    t_g = max_over_ranks(t_graph, world)
    return {"value": count * world / t_g, "ms_per_step": 1e3 * t_g, "graph_kernel_launches": l_graph,
            "batched_value": count * world / max_over_ranks(t_batched, world), "batched_ms": 1e3 * t_batched,
            "batched_launches": l_batched, "plain_value": count * world / max_over_ranks(t_plain, world),
            "plain_ms": 1e3 * t_plain, "plain_launches": l_plain, "max_abs_err": err, "count": count,
            "clocks": clk.summary()}


# ---------------------------------------------------------------------------
# Table I's first layer on 28x28 images (--workload layer28): the paper's single-ciphertext method
# (Alg. 4 over virtual ciphertexts) against the column layout, same layer
# ---------------------------------------------------------------------------
LAYER28_METRIC = ("encrypted-layer images/s (Table I CONV 4x3x3 stride 1 + ACT-1 on 28x28 images, N=2^16), "
                  "column layout vs single-ciphertext Alg. 4")
ACT1 = (-0.00015120704, 0.4610149, 2.0225089, -1.4511951)  # Table I, ACT-1


def run_layer28(args, rank, world, local_rank):
    """CONV (4 kernels 3x3, stride 1) + ACT-1 of Table I on synthetic 28x28 images at the CNN
    parameters (N = 2^16, Q = 60 + 12 x 45, P = 2 x 60). Single-ciphertext path (the paper's
    original method): 32 images per ciphertext in 32x32 blocks (Sec. V: 32 images per ciphertext),
    Alg. 4 per kernel with encrypted Kernelspanner ciphertexts and bias. Column path: 1024 images per
    ciphertext set (blocks of 32 rows), 28 column ciphertexts, he_conv2d with the 4 kernels. Both
    followed by ACT-1 (degree 3). Timed with CUDA events on the context's stream."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_18646_gb300 import api, load
    lib = load()
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.Stream()
    pre = synthetic.CNN_N16
    g = api.Context.from_preset(pre, seed=6000 + rank, stream=stream.cuda_stream)
    if getattr(args, 'no_tensor_cores', False):
        g.set_tensor_cores(False)  # the convolutions' multiply-accumulate on the CUDA cores
    side, k, Hb = 28, 3, 32
    g.keygen([1, 2, Hb, 2 * Hb])
    K, bias = synthetic.conv_weights(4, 1, k, 0.1, seed=202)
    S = g.N // 2
    n_vr = S // (Hb * Hb)  # 32 images per ciphertext
    n_col = S // Hb        # 1024 images per column set
    imgs_vr = synthetic.images(n_vr, side, side, seed=701)
    imgs_col = synthetic.images(n_col, side, side, seed=702)
    x_vr = g.vr_encrypt_images(imgs_vr, Hb, Hb, 0)
    kern = [g.vr_encrypt_kernels(K[o, 0], float(bias[o]), side, side, Hb, Hb, g.L1, 100 * (o + 1))
            for o in range(4)]
    x_col = g.encrypt_image(imgs_col, Hb, ct_id_base=1000)
    g.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(max(1, args.warmup)):
            fn()
        g.synchronize()
        l0 = lib.he_kernel_launches()
        ev0.record(stream)
        for _ in range(reps):
            r = fn()
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / 1e3 / reps, (lib.he_kernel_launches() - l0) / reps, r

    def single():
        outs = []
        for o in range(4):
            y = g.vr_conv2d(x_vr, kern[o][0], kern[o][1], side, side, k, Hb, Hb)
            outs.append(g.poly_act(y, ACT1))
        return outs

    def column():
        y = g.conv2d(x_col, 1, 1, K, bias, 1)
        return g.poly_act(y, ACT1)

    t_vr, l_vr, out_vr = timed(single, max(1, args.steps))
    t_col, l_col, out_col = timed(column, max(1, args.steps))
    # decrypted outputs for the CPU leg's FP64 check (first 4 images of each path)
    ho = side - k + 1
    dec_vr = np.stack([g.decrypt_slots(y)[0] for y in out_vr])  # [o][slots]
    vr_img = np.zeros((4, 4, ho, ho))
    for o in range(4):
        for b in range(4):
            for r in range(ho):
                vr_img[b, o, r] = dec_vr[o, b * Hb * Hb + r * Hb: b * Hb * Hb + r * Hb + ho]
    dec_col = g.decrypt_image(out_col, 4, Hb, 1, ho).reshape(4, 4, ho, ho).transpose(0, 1, 3, 2)
    t_c = max_over_ranks(t_col, world)
    return {"value": n_col * world / t_c, "ms_per_step": 1e3 * t_c, "launches": l_col,
            "single_value": n_vr * world / max_over_ranks(t_vr, world), "single_ms": 1e3 * t_vr,
            "single_launches": l_vr,
            "checks": [(vr_img, imgs_vr[:4], K, bias), (dec_col, imgs_col[:4], K, bias)]}


def fp64_layer_error(checks) -> float:
    """CPU leg: max |decrypted - FP64 (conv + ACT-1)| (the closed forms live with the oracle)."""
    from oracle import fp64_ref
    err = 0.0
    for got, imgs, K, bias in checks:
        x = fp64_ref.conv2d(imgs[:, None], K, bias, 1)
        ref = ACT1[0] + ACT1[1] * x + ACT1[2] * x ** 2 + ACT1[3] * x ** 3
        err = max(err, float(np.abs(got - ref).max()))
    return err


# ---------------------------------------------------------------------------
# one conv + x^2 layer at N = 2^15 (--workload layer): latency and GB/s
# ---------------------------------------------------------------------------
LAYER_METRIC = ("encrypted conv+x^2 layer images/s and latency (N=2^15, 64x64, conv 4x3x3 stride 1 + x^2, "
                "relinearised)")


def run_layer(args, rank, world, local_rank):
    """conv (4 kernels 3x3, stride 1, weights and biases N(0, 0.1)) -> x^2 -> relinearisation on 64x64
    images U[0, 1] at N = 2^15, Q = 60 + 8 x 40, P = 60, alpha = 1, scale 2^40. Two inputs through
    the same call sequence: one image per set of 64 column ciphertexts (the layer's latency) and
    256 images slot-packed per set (block stride 64, S / 64 blocks). GB/s = the library's algorithmic
    bytes of one layer call (every operand read and written once, per kernel) / its device time.
    Timed with CUDA events on the context's stream."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_18646_gb300 import api, load
    lib = load()
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.Stream()
    pre = synthetic.CONV_LAYER
    g = api.Context.from_preset(pre, seed=201 + 1000 * rank, stream=stream.cuda_stream)
    if getattr(args, 'no_tensor_cores', False):
        g.set_tensor_cores(False)  # the convolutions' multiply-accumulate on the CUDA cores
    g.keygen([1, 2])
    side, Hs = 64, 64
    K, bias = synthetic.conv_weights(4, 1, 3, 0.1, seed=202)
    n_batch = (g.N // 2) // Hs
    imgs = synthetic.images(n_batch, side, side, seed=201)
    x1 = g.encrypt_image(imgs[:1], Hs, ct_id_base=0)
    xb = g.encrypt_image(imgs, Hs, ct_id_base=100)
    g.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def layer(x):
        y = g.conv2d(x, 1, 1, K, bias, 1)
        g.square(y)
        return g.relinearize(y)

    def timed(x, reps):
        for _ in range(max(1, args.warmup)):
            y = layer(x)
            y.free()
        g.synchronize()
        l0 = lib.he_kernel_launches()
        ys = []
        ev0.record(stream)
        for _ in range(reps):
            ys.append(layer(x))
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / 1e3 / reps, (lib.he_kernel_launches() - l0) // reps, ys[-1]

    reps = max(1, args.steps)
    with ClockSampler(local_rank) as clk:
        t1, l1, y1 = timed(x1, reps)
        tb, lb, yb = timed(xb, reps)
    # algorithmic bytes of one layer call from the library's per-kernel counts
    lib.he_profile_enable(1)
    layer(xb).free()
    g.synchronize()
    prof = profile_read(lib)
    lib.he_profile_enable(0)
    alg_bytes = sum(v["bytes"] for v in prof.values())
    ho = side - 2
    dec1 = g.decrypt_image(y1, 1, Hs, 1, ho).reshape(1, 4, ho, ho).transpose(0, 1, 3, 2)
    decb = g.decrypt_image(yb, 4, Hs, 1, ho).reshape(4, 4, ho, ho).transpose(0, 1, 3, 2)
    t1m, tbm = max_over_ranks(t1, world), max_over_ranks(tb, world)
    return {"value": n_batch * world / tbm, "ms_per_step": 1e3 * tbm, "launches": lb,
            "latency_ms": 1e3 * t1m, "plain_value": world / t1m, "plain_launches": l1,
            "alg_bytes": alg_bytes, "GBps": alg_bytes / tbm / 1e9, "images_per_set": n_batch, "clocks": clk.summary(),
            "checks": [(dec1, imgs[:1], K, bias), (decb, imgs[:4], K, bias)]}


def fp64_square_layer_error(checks) -> float:
    """CPU leg: max |decrypted - FP64 (conv, then x^2)|."""
    from oracle import fp64_ref
    err = 0.0
    for got, imgs, K, bias in checks:
        ref = fp64_ref.conv2d(imgs[:, None], K, bias, 1) ** 2
        err = max(err, float(np.abs(got - ref).max()))
    return err


# ---------------------------------------------------------------------------
# Table I's whole CNN in the single-ciphertext layout (--workload table1)
# ---------------------------------------------------------------------------
TABLE1_METRIC = ("encrypted Table I CNN images/s (CONV 4x3x3, ACT-1, FC-1 2704->64, ACT-2, FC-2 64->10 on 28x28 "
                 "images, N=2^16), the paper's single-ciphertext layout")


def run_table1(args, rank, world, local_rank):
    """Table I's CNN through the paper's own method: 32 images of 28 x 28 per ciphertext in 32 x 32
    blocks, CONV by Alg. 4, ACT-1, FC-1 and FC-2 by Alg. 3 (table1.forward), at the CNN parameters
    (N = 2^16, Q = 60 + 12 x 45, P = 2 x 60), all twelve levels. One step = one inference of one
    ciphertext of 32 images; timed with CUDA events on the context's stream."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_18646_gb300 import api, load, table1
    lib = load()
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.Stream()
    g = api.Context.from_preset(synthetic.CNN_N16, seed=7000 + rank, stream=stream.cuda_stream)
    if getattr(args, 'no_tensor_cores', False):
        g.set_tensor_cores(False)  # the convolutions' multiply-accumulate on the CUDA cores
    geo = table1.Geometry(h=28, w=28, k=3, Hb=32, Wb=32, channels=4, fc1_out=64, fc2_out=10, slots=g.N // 2)
    t0 = time.perf_counter()
    g.keygen(table1.rotation_steps(geo))
    keygen_s = time.perf_counter() - t0
    wts = synthetic.table1_weights(seed=202)
    imgs = synthetic.images(geo.images, 28, 28, seed=703)
    model = table1.encrypt_model(g, geo, wts)
    x = g.vr_encrypt_images(imgs, 32, 32, 0)
    g.synchronize()
    for _ in range(max(1, args.warmup)):
        table1.forward(g, geo, x, model)
    g.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = lib.he_kernel_launches()
    reps = max(1, args.steps)
    ev0.record(stream)
    for _ in range(reps):
        out = table1.forward(g, geo, x, model)
    ev1.record(stream)
    ev1.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3 / reps
    launches = (lib.he_kernel_launches() - l0) // reps
    got = table1.logits(g, geo, out)
    tm = max_over_ranks(t, world)

    # the same network through the column layout: 1024 images per set of 28 column ciphertexts
    # (32-row blocks), he_conv2d, he_poly_act, the column-layout dense layer (he_fc_apply) twice
    H, Bc = 32, g.N // 2 // 32
    imgs_c = synthetic.images(Bc, 28, 28, seed=704)
    xc = g.encrypt_image(imgs_c, H, ct_id_base=5000)
    W1 = np.ascontiguousarray(wts.fc1_w.reshape(-1, 64).T)  # [64][4 x 26 x 26], (channel, row, column)
    W2 = np.ascontiguousarray(wts.fc2_w.T)                   # [10][64]
    pts1 = g.fc_prepare(W1, 4, 26, 26, 1, H, Bc, g.L1 - 3)
    pts2 = g.fc_prepare(W2, 64, 1, 1, 1, H, Bc, g.L1 - 6)

    def column_net():
        y = g.conv2d(xc, 1, 1, wts.conv_w[:, None], wts.conv_b, 1)
        g.poly_act(y, table1.ACT1)
        z = g.fc_apply(y, pts1, wts.fc1_b)
        g.poly_act(z, table1.ACT2)
        return g.fc_apply(z, pts2, wts.fc2_b)

    for _ in range(max(1, args.warmup)):
        column_net()
    g.synchronize()
    l0 = lib.he_kernel_launches()
    ev0.record(stream)
    for _ in range(reps):
        zc = column_net()
    ev1.record(stream)
    ev1.synchronize()
    tc = max_over_ranks(ev0.elapsed_time(ev1) / 1e3 / reps, world)
    col_launches = (lib.he_kernel_launches() - l0) // reps
    got_c = g.decrypt_slots(zc)[:, ::H][:, :8].T
    return {"value": geo.images * world / tm, "ms_per_step": 1e3 * tm, "launches": launches,
            "keygen_s": keygen_s, "rotation_keys": len(table1.rotation_steps(geo)), "images": geo.images,
            "check": (got, imgs, wts), "column_value": Bc * world / tc, "column_ms": 1e3 * tc,
            "column_launches": col_launches, "column_images": Bc, "column_check": (got_c, imgs_c[:8], wts)}


def fp64_table1_error(check) -> float:
    """CPU leg: max |decrypted logits - FP64 Table I CNN|."""
    from oracle import fp64_ref
    from paper_2512_18646_gb300 import table1
    got, imgs, wts = check
    return float(np.abs(got - fp64_ref.table1_cnn(imgs, wts, table1.ACT1, table1.ACT2)).max())


# ---------------------------------------------------------------------------
# the serving workload (--workload serve)
# ---------------------------------------------------------------------------
SERVE_METRIC = ("served encrypted-CNN images/s and p50/p99 latency (Poisson arrivals, image sides {64,128,256}, "
                "N=2^16), continuous batching vs one request at a time")
SERVE_SIDES = (64, 128, 256)


def _replay(srv, pool, arrival_s, sides, out_buf):
    """Submit request i at arrival_s[i] (seconds after the start) from a client thread; claim each
    result as soon as it is done (he_server_take_host into page-locked host memory).

    Returns per request: (scheduled arrival, submit, admit, start, done, claimed), ms of CLOCK_MONOTONIC."""
    import queue
    n = len(arrival_s)
    ids = queue.Queue()
    t0 = time.monotonic() + 0.05

    def client():
        for i in range(n):
            dt = t0 + arrival_s[i] - time.monotonic()
            if dt > 0:
                time.sleep(dt)
            ptr, words = pool[int(sides[i])][i % len(pool[int(sides[i])])]
            try:
                ids.put((i, srv.submit_ptr(ptr, words, int(sides[i]))))
            except Exception as e:  # refused (e.g. budget): reported by the claiming loop
                ids.put((i, e))
                return

    th = threading.Thread(target=client)
    th.start()
    rec = np.zeros((n, 6))
    pending = {}
    claimed = 0
    deadline = time.monotonic() + 600 + float(arrival_s[-1])
    while claimed < n:
        while True:
            try:
                i, rid = ids.get_nowait()
            except queue.Empty:
                break
            if isinstance(rid, Exception):
                th.join()
                raise rid
            pending[rid] = i
        done = [rid for rid in pending if srv.poll(rid) >= 3]
        for rid in done:
            i = pending.pop(rid)
            blk, t = srv.take_host(rid, out_buf)
            rec[i, 0] = 1e3 * (t0 + arrival_s[i])
            rec[i, 1:5] = t
            rec[i, 5] = 1e3 * time.monotonic()
            claimed += 1
        if not done:
            if time.monotonic() > deadline:
                raise RuntimeError("requests not served within the deadline")
            time.sleep(0.001)
    th.join()
    return rec


def run_serve(args, rank, world, local_rank):
    """A Poisson stream of encrypted CNN requests against the continuous-batching server and against
    the same server limited to one request per batch (plain FIFO, one request at a time)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_18646_gb300 import api, load
    lib = load()
    torch.cuda.set_device(local_rank)
    pre = synthetic.CNN_N16
    g = api.Context.from_preset(pre, seed=5000 + rank)
    if getattr(args, 'no_tensor_cores', False):
        g.set_tensor_cores(False)  # the convolutions' multiply-accumulate on the CUDA cores
    g.keygen([])
    w = {s: synthetic.cnn_weights(s, seed=302) for s in SERVE_SIDES}
    n_warm, n_meas = args.serve_warmup, args.requests
    arrival, side = synthetic.poisson_trace(n_warm + n_meas, rate=args.rate)
    # a pool of encrypted requests per side, each image repeated in every slot block, in page-locked memory
    pool, keep = {}, []
    t_enc = time.perf_counter()
    for s in SERVE_SIDES:
        pool[s] = []
        for k in range(args.pool):
            img = synthetic.images(1, s, s, seed=600 + 7 * k + s)[0]
            x = g.encrypt_image(np.repeat(img[None], g.slots // s, axis=0), s, ct_id_base=10 ** 6 * (k + 1) + s)
            buf = torch.empty(s * 2 * g.L1 * g.N, dtype=torch.int64).pin_memory()
            arr = buf.numpy().view(np.uint64)
            x.export_raw(arr)
            del x
            keep.append(buf)
            pool[s].append((arr.ctypes.data, arr.size))
    g.synchronize()
    t_enc = time.perf_counter() - t_enc
    out_words = 10 * 2 * (g.L1 - 6) * g.N
    out_buf = torch.empty(out_words, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
    res = {"encrypt_pool_s": t_enc}
    clk = ClockSampler(local_rank).__enter__()
    for mode, max_blocks, n_req in (("batched", args.max_blocks, n_meas), ("plain", 1, args.plain_requests)):
        t_c = time.perf_counter()
        srv = api.Server(g, w, hbm_budget_bytes=int(args.budget_gb * (1 << 30)), max_blocks=max_blocks)
        create_s = time.perf_counter() - t_c
        # warm-up: the first n_warm requests of the trace (untimed)
        _replay(srv, pool, arrival[:n_warm] - arrival[0], side[:n_warm], out_buf)
        l0 = lib.he_kernel_launches()
        arr = arrival[n_warm:n_warm + n_req]
        rec = _replay(srv, pool, arr - arr[0], side[n_warm:n_warm + n_req], out_buf)
        launches = lib.he_kernel_launches() - l0
        st = srv.stats()
        srv.close()
        lat = rec[:, 4] - rec[:, 0]
        e2e_lat = rec[:, 5] - rec[:, 0]
        span = (rec[:, 4].max() - rec[:, 0].min()) / 1e3
        span_e2e = (rec[:, 5].max() - rec[:, 0].min()) / 1e3
        res[mode] = {
            "requests": n_req, "images_per_s": n_req / span, "e2e_images_per_s": n_req / span_e2e,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "e2e_p99_ms": float(np.percentile(e2e_lat, 99)),
            "queue_p50_ms": float(np.percentile(rec[:, 3] - rec[:, 0], 50)),
            "submit_jitter_p99_ms": float(np.percentile(rec[:, 1] - rec[:, 0], 99)),
            "batches": st["batches"], "reserve_gb": st["reserve_bytes"] / 2 ** 30,
            "max_held_gb": st["max_held_bytes"] / 2 ** 30, "pool_high_gb": st["pool_high_bytes"] / 2 ** 30,
            "create_s": create_s, "launches": launches,
            "h2d_bytes": int(sum(int(s) * 2 * g.L1 * g.N * 8 for s in side[n_warm:n_warm + n_req])),
            "d2h_bytes": int(n_req * out_words * 8),
        }
    clk.__exit__()
    res["clocks"] = clk.summary()
    res["sides"] = [int(x) for x in side[n_warm:n_warm + n_meas]]
    # accuracy: one request per side through the batched server, against the FP64 CNN (untimed)
    srv = api.Server(g, w, hbm_budget_bytes=int(args.budget_gb * (1 << 30)), max_blocks=args.max_blocks,
                     start_paused=True)
    rids = {s: srv.submit_ptr(*pool[s][0], s) for s in SERVE_SIDES}
    srv.pause(False)
    checks = []  # (logits, image, weights) per side, checked against the FP64 CNN by the CPU leg
    for s, rid in rids.items():
        srv.wait(rid, 600_000)
        z, blk, _ = srv.take(rid)
        logit = g.decrypt_slots(z)[:, blk * s]
        img = synthetic.images(1, s, s, seed=600 + s)[0]
        checks.append((logit[None], img[None], w[s]))
    srv.close()
    res["checks"] = checks
    return res


def fp64_max_error(checks) -> float:
    """CPU leg: max |decrypted logits - FP64 CNN| over (logits, images, weights) triples. The FP64
    closed form lives with the oracle; only this CPU leg of the benchmark imports it."""
    from oracle import fp64_ref
    return max(float(np.abs(logits - fp64_ref.cnn(imgs, w)).max()) for logits, imgs, w in checks)


# ---------------------------------------------------------------------------
# CPU oracle: bounded samples of the same workloads
# ---------------------------------------------------------------------------
def ks_per_inference(side: int) -> int:
    """Key switches of one CNN inference on a side x side image in the column layout: conv-1 rotates
    each of the side input columns by 1..4; the square's output (8 h1 three-component ciphertexts) is
    relinearised as conv-2's input and rotated by 2 and 4; the dense layer takes the second square's
    three components, relinearises its 10 outputs and sums their blocks by rotations 4 .. side/2."""
    h1 = (side - 5) // 2 + 1
    return 4 * side + 8 * h1 + 16 * h1 + 10 + 10 * int(np.log2(side // 4))


class OracleCnnSample:
    """Conv-1 output column 0 (all 8 channels) of the CNN on the oracle at the full parameters.

    Set up once (keys, five encrypted input columns); each run() is 5 hoisted ModUps, 20 key switches
    at the top level, 200 ciphertext-scalar products and 8 rescales, and stands for
    20 / ks_per_inference(side) of one inference (the oracle's time is dominated by key switching)."""

    def __init__(self, batch: int, side: int = SIDE, H: int = H, preset=None):
        from oracle import Oracle, layouts
        pre = preset or synthetic.CNN_N16
        self.o = Oracle.from_preset(pre, seed=7)
        self.o.keygen([1, 2, 3, 4])
        imgs = synthetic.images(batch, side, 5, seed=301)
        z = layouts.image_columns(imgs, self.o.slots, H)
        self.X = np.stack([self.o.encrypt(self.o.encode(z[j]), self.o.L1, j) for j in range(5)])[None]
        self.w = synthetic.cnn_weights(side, seed=302)
        self.fraction = 20.0 / ks_per_inference(side)

    def run(self) -> float:
        t0 = time.perf_counter()
        self.o.conv2d(self.X, 1, self.w.conv1_w, self.w.conv1_b, 2, self.o.scale, sel=[(c, 0) for c in range(8)])
        return time.perf_counter() - t0


def _cpu(value, unit, sample):
    return {"value": value, "unit": unit, "cores": cpu_cores(), "cpu_model": cpu_model(), "kind": "oracle",
            "sample": sample}


def oracle_cnn_baseline(batch: int, preset=None):
    s = OracleCnnSample(batch, preset=preset)
    dt = s.run()
    per_inference = dt / s.fraction
    return _cpu(batch / per_inference, UNIT,
                f"conv-1 output column 0 (8 channels, 20 top-level key switches) took {dt:.2f} s; scaled to one "
                f"inference of {batch} images by key-switch count ({ks_per_inference(SIDE)}/20)")


def oracle_matmul_small_baseline(budget_s: float = 10.0):
    """The whole 4x8 . 8x4 product at N = 2^13 on the oracle (24 hoisted rotations, 32 tensor products,
    4 relinearisations and rescales), repeated for about budget_s seconds."""
    from oracle import Oracle, layouts
    o = Oracle.from_preset(synthetic.MATMUL_SMALL, seed=5)
    o.keygen([1, 2, 3])
    A, Bm = synthetic.matmul_operands(4, 8, 4, seed=101)
    Ac = np.stack([o.encrypt(o.encode(v), o.L1, i) for i, v in enumerate(layouts.matrix_a_columns(A, o.slots))])
    Bc = np.stack([o.encrypt(o.encode(v), o.L1, 50 + i) for i, v in enumerate(layouts.matrix_b_rows(Bm, o.slots))])
    reps, t0 = 0, time.perf_counter()
    while reps == 0 or time.perf_counter() - t0 < budget_s:
        o.matmul(Ac, Bc, 4)
        reps += 1
    dt = time.perf_counter() - t0
    return _cpu(reps / dt, "HE-matmul/s", f"{reps} whole products (A 4x8, B 8x4, N=2^13) in {dt:.2f} s")


def oracle_layer_baseline():
    """Output column 0 of the conv + x^2 + relinearisation layer (4 channels) at N = 2^15: 3 input columns
    rotated by 1 and 2 (6 key switches), 36 scalar products, 4 squares and 4 relinearisations; scaled to
    the whole layer (128 rotations + 248 relinearisations) by key-switch count."""
    from oracle import Oracle, layouts
    o = Oracle.from_preset(synthetic.CONV_LAYER, seed=201)
    o.keygen([1, 2])
    side, Hs = 64, 64
    imgs = synthetic.images((o.slots // Hs), side, side, seed=201)
    K, bias = synthetic.conv_weights(4, 1, 3, 0.1, seed=202)
    z = layouts.image_columns(imgs[:, :, :3], o.slots, Hs)
    X = np.stack([o.encrypt(o.encode(z[j]), o.L1, j) for j in range(3)])[None]
    t0 = time.perf_counter()
    y = o.square(o.conv2d(X, 1, K, bias, 1, o.scale, sel=[(c, 0) for c in range(4)]))
    for t in range(4):
        o.relin(y[t])
    dt = time.perf_counter() - t0
    per_layer = dt * (128 + 248) / (6 + 4)
    return _cpu((o.slots // Hs) / per_layer, "images/s",
                f"output column 0 of the 4 channels (10 key switches) took {dt:.2f} s; scaled to one layer of "
                f"{o.slots // Hs} packed images by key-switch count (376/10)")


def oracle_matmul_baseline(shapes):
    """One zero-rotation product of the 64-product workload on the oracle (the one with the fewest tensor
    products), scaled to all 64 by tensor-product count (sum of G n over the products)."""
    from oracle import Oracle, layouts
    pre = synthetic.CNN_N16
    o = Oracle.from_preset(pre, seed=7)
    o.keygen([])
    S = (1 << pre.log_n) // 2
    cost = [layouts.volley_geometry(S, m, p)[2] * n for m, n, p in shapes]
    i = int(np.argmin(cost))
    m, n, p = shapes[i]
    A, Bm = synthetic.matmul_operands(m, n, p, seed=402 + i)
    G = layouts.volley_geometry(S, m, p)[2]
    za = layouts.matrix_a_volley(A, S, p).reshape(G * n, S)
    Ac = np.stack([o.encrypt(o.encode(v), o.L1, t) for t, v in enumerate(za)]).reshape(G, n, 2, o.L1, o.N)
    Bc = np.stack([o.encrypt(o.encode(v), o.L1, 10 ** 5 + t) for t, v in enumerate(layouts.matrix_b_rows(Bm, S))])
    t0 = time.perf_counter()
    o.matmul_volley(Ac, Bc)
    dt = time.perf_counter() - t0
    total = dt * sum(cost) / cost[i]
    return _cpu(len(shapes) / total, "HE-matmul/s",
                f"product {i} (m,n,p)=({m},{n},{p}), {cost[i]} tensor products, zero-rotation layout, took "
                f"{dt:.2f} s; scaled to the {len(shapes)} products by tensor-product count ({sum(cost)}/{cost[i]})")


def oracle_serve_baseline(sides):
    """Requests served one at a time by the oracle: conv-1 output column 0 of a side-64 request timed,
    each request's time scaled by its key-switch count (ks_per_inference(side) / 20)."""
    s = OracleCnnSample(1, side=64, H=64)
    dt = s.run()
    per_ks = dt / 20.0
    lat = np.array([per_ks * ks_per_inference(int(x)) for x in sides])
    return _cpu(len(sides) / float(lat.sum()), "images/s",
                f"conv-1 output column 0 of a side-64 request (20 key switches) took {dt:.2f} s; each request "
                f"of the trace scaled by its key-switch count; serial latency p50 {np.percentile(lat, 50):.0f} s")


# ---------------------------------------------------------------------------
# small cases of the hot kernels, sized for profiler captures (--workload case --case NAME)
# ---------------------------------------------------------------------------
# Each runs one layer of the CNN at its parameters (N = 2^16, Q = 60 + 12 x 45, P = 2 x 60,
# digits of two primes) on a narrow slab, so that every launch has the shape of the full workload's
# launches per limb while the device holds a few GB and each launch's data exceeds L2; the body runs
# inside the NVTX range "case" (ncu --nvtx --nvtx-include "case/"):
#   conv1   16 image columns (256 images): hoisted rotations by 1..4, the 8-channel 5x5 stride-2
#           multiply-accumulate, rescale;
#   square  x^2 of 64 ciphertexts at the top level (tensor, rescale, relinearisation);
#   conv2   the second convolution (16 x 3 x 3, stride 2, 8 channels of 16 columns, row gap 2) on
#           128 ciphertexts at 11 limbs;
#   fc      the dense layer on 16 x 4 input ciphertexts at 9 limbs, 10 outputs.
CASES = ("conv1", "conv2", "square", "fc")


def run_case(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_18646_gb300 import api
    pre = synthetic.CNN_N16
    g = api.Context.from_preset(pre, seed=5)
    if getattr(args, 'no_tensor_cores', False):
        g.set_tensor_cores(False)  # the convolutions' multiply-accumulate on the CUDA cores
    g.keygen([1, 2, 3, 4])
    w = synthetic.cnn_weights(128, seed=302)
    if args.case == "conv2":
        rng = np.random.default_rng(4)
        x = g.encrypt_coeffs(rng.integers(-(1 << 40), 1 << 40, size=(8 * 16, g.N), dtype=np.int64), 11, g.scale)
    elif args.case == "fc":
        g.keygen([4, 8, 16, 32, 64])
        rng = np.random.default_rng(3)
        x = g.encrypt_coeffs(rng.integers(-(1 << 40), 1 << 40, size=(64, g.N), dtype=np.int64), 9, g.scale)
        pts = g.fc_prepare(rng.normal(0, 0.05, (10, 16 * 30 * 4)), 16, 30, 4, 4, 128, 256, 9)
    else:
        x = g.encrypt_image(synthetic.images(256, 128, 16 if args.case == "conv1" else 64, seed=301), 128)
    g.synchronize()
    torch.cuda.nvtx.range_push("case")
    for _ in range(max(1, args.steps)):
        if args.case == "conv1":
            y = g.conv2d(x, 1, 1, w.conv1_w, w.conv1_b, 2)
        elif args.case == "conv2":
            y = g.conv2d(x, 8, 2, w.conv2_w, w.conv2_b, 2)
        elif args.case == "fc":
            y = g.fc_apply(x, pts, None)
        else:
            y = g.relinearize(g.mul(x, x))
        del y
    g.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"case": args.case, "repeats": max(1, args.steps), "done": True}))


# ---------------------------------------------------------------------------
# the other configurations, reported beside the CNN in the default run
# ---------------------------------------------------------------------------
# (key, workload, extra arguments): the small matmul (4096 products, plain vs batched vs CUDA graph),
# the conv + x^2 layer at N = 2^15, the 64 uneven matmuls at N = 2^16 (zero-rotation, baby-step
# giant-step, batched and plain revolver), and the Poisson serving trace (continuous batching vs one
# request at a time)
EXTRA_WORKLOADS = (
    ("matmul_4x8x4_n13", "matmul_small", ["--steps", "3", "--warmup", "3"]),
    ("conv_layer_64x64_n15", "layer", ["--steps", "5", "--warmup", "3"]),
    ("matmul64_uneven_n16", "matmul", []),
    ("serving_poisson_n16", "serve", []),
    ("cnn_dnum3_5special_n16", "cnn", ["--preset", "cnn_n16_dnum3", "--steps", "5", "--warmup", "3", "--no-extra",
                                       "--no-e2e"]),
)


def run_extra_workloads(args):
    """Each configuration in a process of its own (its device memory is returned when it exits), after
    the CNN's measurement has released its device memory; its JSON line (with its own clocks and
    oracle baseline) is kept whole."""
    out = {}
    for key, wl, extra in EXTRA_WORKLOADS:
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", wl, *extra]
        if args.no_cpu_baseline:
            cmd.append("--no-cpu-baseline")
        env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
        t0 = time.perf_counter()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=1200, env=env)
            lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
            if r.returncode == 0 and lines:
                out[key] = json.loads(lines[-1])
            else:
                out[key] = {"error": f"exit {r.returncode}: " + (r.stderr.strip().splitlines() or [""])[-1][:300]}
        except subprocess.TimeoutExpired:
            out[key] = {"error": "did not finish within 1200 s"}
        out[key]["wall_s"] = round(time.perf_counter() - t0, 1)
        sys.stderr.write(f"[bench] {key}: {out[key].get('value', out[key].get('error'))} ({out[key]['wall_s']} s)\n")
    return out


def cpu_cores():
    """Threads the oracle runs on: its OpenMP thread count (OMP_NUM_THREADS when set, else one per
    core this process may use)."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    omp = os.environ.get("OMP_NUM_THREADS", "")
    if omp.isdigit() and int(omp) > 0:
        n = min(n, int(omp))
    return n


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return f"{ln.split(':', 1)[1].strip()} ({platform.machine()})"
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--batch", type=int, default=256, help="images per ciphertext set (block stride 128)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tensor-cores", action="store_true",
                    help="run the convolutions' multiply-accumulate on the CUDA cores (96-bit sums)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--preset", choices=sorted(CNN_PRESETS), default="cnn_n16",
                    help="cnn workload: prime chain and key-switching digits")
    ap.add_argument("--no-extra", action="store_true",
                    help="cnn workload: skip the other configurations (matmul, conv layer, batched matmul, serving)")
    ap.add_argument("--workload", choices=["cnn", "layer", "matmul", "matmul_small", "layer28", "table1", "serve",
                                           "case"], default="cnn")
    ap.add_argument("--case", choices=CASES, default="conv2", help="case workload: the kernel case to run")
    ap.add_argument("--count", type=int, default=0, help="matmul workload: first COUNT products only")
    ap.add_argument("--requests", type=int, default=600, help="serve workload: measured requests")
    ap.add_argument("--serve-warmup", type=int, default=20, help="serve workload: warm-up requests")
    ap.add_argument("--plain-requests", type=int, default=40,
                    help="serve workload: requests replayed on the one-at-a-time path (a prefix of the trace)")
    ap.add_argument("--rate", type=float, default=20.0, help="serve workload: Poisson arrival rate (req/s)")
    ap.add_argument("--max-blocks", type=int, default=128, help="serve workload: requests per batch")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serve workload: device-memory budget")
    ap.add_argument("--pool", type=int, default=2, help="serve workload: distinct encrypted images per side")
    args = ap.parse_args()
    rank, world, local_rank = rank_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    wl = WORKLOAD.replace(KS_DESC["cnn_n16"], KS_DESC[args.preset])
    cfg = {"workload": wl, "images_per_step": args.batch, "image_side": SIDE, "log_n": 16,
           "parallelism": f"replicas x{world} (independent inferences, no collective)",
           "l2": "inputs (128 ciphertexts, 1.7 GB) larger than L2; no flush needed",
           "conv_mac": "CUDA cores (96-bit sums)" if args.no_tensor_cores else
           "tensor cores (tcgen05: residues in byte or 7-bit chunks, products summed exactly in fp32)"}

    if args.workload == "case":
        run_case(args)
        return

    if args.workload == "layer" and args.impl == "gpu":
        res = run_layer(args, rank, world, local_rank)
        if rank == 0:
            line = {"metric": LAYER_METRIC, "value": res["value"], "unit": "images/s", "n_gpus": world,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                    "data": "synthetic",
                    "config": {"workload": "conv (4 kernels 3x3, stride 1, weights and biases N(0,0.1), seed 202) "
                                           "-> x^2 -> relinearisation on 64x64 images U[0,1] (seed 201); RNS-CKKS "
                                           "N=2^15, Q=60+8x40, P=60, alpha=1, scale 2^40",
                               "images_per_set": res["images_per_set"], "parallelism": f"replicas x{world}",
                               "l2": "input set (64 ciphertexts of 9 limbs, 0.3 GB) and its rotations exceed L2"},
                    "path": "he_conv2d (hoisted rotations by 1 and 2, scalar multiply-accumulate, rescale) + "
                            "he_poly_act x^2 + he_relinearize; 256 images slot-packed per set",
                    "gpu_launches": res["launches"],
                    "latency_ms": res["latency_ms"],
                    "plain": {"value": res["plain_value"], "ms": res["latency_ms"], "images_per_set": 1,
                              "gpu_launches": res["plain_launches"]},
                    "algorithmic_bytes_per_layer": res["alg_bytes"], "GBps": res["GBps"],
                    "max_abs_err_vs_fp64": None if args.no_cpu_baseline else fp64_square_layer_error(res["checks"]),
                    "clocks": res["clocks"],
                    "cpu_baseline": None if args.no_cpu_baseline or world > 1 else oracle_layer_baseline()}
            print(json.dumps(line))
        return

    if args.workload == "table1" and args.impl == "gpu":
        res = run_table1(args, rank, world, local_rank)
        if rank == 0:
            line = {"metric": TABLE1_METRIC, "value": res["value"], "unit": "images/s", "n_gpus": world,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                    "data": "synthetic",
                    "config": {"workload": "Table I CNN on 32 synthetic 28x28 images U[0,1] per ciphertext (32x32 "
                                           "blocks): CONV 4 kernels 3x3 stride 1 (Alg. 4), ACT-1, FC-1 2704->64 and "
                                           "FC-2 64->10 (Alg. 3, tau_b-encoded weights), ACT-2; synthetic weights "
                                           "(seed 202); RNS-CKKS N=2^16, Q=60+12x45, P=2x60, alpha=2, 12 levels",
                               "parallelism": f"replicas x{world}"},
                    "path": "paper_2512_18646_gb300.table1.forward: he_vr_conv2d, he_poly_act, he_vr_matmul, "
                            "he_rotate, he_add, he_add_slots, he_ctset_drop_levels",
                    "gpu_launches": res["launches"], "images_per_ciphertext": res["images"],
                    "rotation_keys": res["rotation_keys"], "keygen_s": res["keygen_s"],
                    "max_abs_err_vs_fp64": None if args.no_cpu_baseline else fp64_table1_error(res["check"]),
                    "column_layout": {"value": res["column_value"], "ms": res["column_ms"],
                                      "images_per_set": res["column_images"], "gpu_launches": res["column_launches"],
                                      "path": "he_conv2d, he_poly_act, he_fc_apply x2 (1024 images per set of 28 "
                                              "column ciphertexts)",
                                      "max_abs_err_vs_fp64": None if args.no_cpu_baseline
                                      else fp64_table1_error(res["column_check"])}}
            print(json.dumps(line))
        return

    if args.workload == "layer28" and args.impl == "gpu":
        res = run_layer28(args, rank, world, local_rank)
        if rank == 0:
            line = {"metric": LAYER28_METRIC, "value": res["value"], "unit": "images/s", "n_gpus": world,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                    "data": "synthetic",
                    "config": {"workload": "Table I CONV (4 kernels 3x3, stride 1, weights N(0,0.1)) + ACT-1 on "
                                           "28x28 images U[0,1]; RNS-CKKS N=2^16, Q=60+12x45, P=2x60, alpha=2",
                               "parallelism": f"replicas x{world}"},
                    "path": "column layout (1024 images per set of 28 column ciphertexts, he_conv2d + he_poly_act)",
                    "gpu_launches": res["launches"],
                    "single_ciphertext": {"value": res["single_value"], "ms": res["single_ms"],
                                          "images_per_ciphertext": 32, "gpu_launches": res["single_launches"],
                                          "path": "Alg. 4 per kernel (he_vr_conv2d) + he_poly_act"},
                    "max_abs_err_vs_fp64": None if args.no_cpu_baseline else fp64_layer_error(res["checks"])}
            print(json.dumps(line))
        return

    if args.workload == "matmul_small" and args.impl == "gpu":
        res = run_matmul_small(args, rank, world, local_rank)
        if rank == 0:
            line = {"metric": MATMUL_SMALL_METRIC, "value": res["value"], "unit": "HE-matmul/s", "n_gpus": world,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                    "data": "synthetic",
                    "config": {"workload": f"{res['count']} encrypted matmuls A(4x8) B(8x4), entries U[-1,1]; "
                                           "RNS-CKKS N=2^13, Q=60+40+40, P=60, scale 2^40 (n=8 ciphertexts "
                                           "per operand, p=4 diagonal outputs)",
                               "parallelism": f"replicas x{world}",
                               "l2": "operands 25.8 GB, larger than L2"},
                    "path": "one he_matmul_batched call captured into a CUDA graph, replayed per step",
                    "gpu_launches": res["graph_kernel_launches"], "max_abs_err_vs_fp64": res["max_abs_err"],
                    "clocks": res["clocks"],
                    "cpu_baseline": None if args.no_cpu_baseline or world > 1 else oracle_matmul_small_baseline(),
                    "batched": {"value": res["batched_value"], "ms": res["batched_ms"],
                                "gpu_launches": res["batched_launches"]},
                    "plain": {"value": res["plain_value"], "ms": res["plain_ms"],
                              "gpu_launches": res["plain_launches"]}}
            print(json.dumps(line))
        return

    if args.workload == "matmul" and args.impl == "gpu":
        res = run_matmul(args, rank, world, local_rank)
        if rank == 0:
            line = {"metric": MATMUL_METRIC, "value": res["value"], "unit": "HE-matmul/s", "n_gpus": world,
                    "steps": 1, "warmup": 1, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
                    "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                    "config": {"workload": "64 encrypted matmuls A(m x n) B(n x p), m,n,p i.i.d. uniform over "
                                           "{16,...,256} (seed 401), entries U[-1,1]; N=2^16, CNN primes, top level",
                               "parallelism": f"replicas x{world}"},
                    "path": "zero-rotation (volley) layout: A's columns replicated at blocks t*M + o_g, "
                            "M = 1 mod p; one he_matmul_volley call per product",
                    "gpu_launches": res["launches"], "max_abs_err_vs_fp64": res["max_abs_err"],
                    "rotations": res["volley_rotations"], "tensor_products": res["volley_tensors"],
                    "revolver": {"batched_value": res["revolver_batched_value"],
                                 "batched_ms": res["revolver_batched_ms"],
                                 "plain_value": res["revolver_plain_value"], "plain_ms": res["revolver_plain_ms"],
                                 "bsgs_value": res["bsgs_value"], "bsgs_ms": res["bsgs_ms"],
                                 "gpu_launches": res["revolver_launches"],
                                 "max_abs_err_vs_fp64": res["revolver_max_abs_err"],
                                 "rotations": res["revolver_rotations"],
                                 "tensor_products": res["revolver_tensors"],
                                 "wave0_profile": res["revolver_wave0_profile"]},
                    "keygen_s": res["keygen_s"], "waves": res["waves"], "clocks": res["clocks"],
                    "cpu_baseline": None if args.no_cpu_baseline or world > 1
                    else oracle_matmul_baseline(res["shapes"])}
            print(json.dumps(line))
        return

    if args.workload == "serve" and args.impl == "gpu":
        res = run_serve(args, rank, world, local_rank)
        if rank == 0:
            b, p = res["batched"], res["plain"]
            line = {"metric": SERVE_METRIC, "value": b["images_per_s"], "unit": "images/s", "n_gpus": world,
                    "steps": b["requests"], "warmup": args.serve_warmup, "ms_per_step": 1e3 / b["images_per_s"],
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                    "data": "synthetic",
                    "config": {"workload": f"Poisson stream ({args.rate} req/s, seeds 501/502) of encrypted CNN "
                                           "requests (conv5x5s2(8)-x^2-conv3x3s2(16)-x^2-fc10), square image side "
                                           "uniform over {64,128,256}; N=2^16, Q=60+12x45, P=2x60, alpha=2",
                               "max_blocks": args.max_blocks, "budget_gb": args.budget_gb,
                               "parallelism": f"replicas x{world}"},
                    "p50_ms": b["p50_ms"], "p99_ms": b["p99_ms"],
                    "plain": p, "batched": b, "gpu_launches": b["launches"],
                    "e2e": {"value": b["e2e_images_per_s"], "unit": "images/s",
                            "h2d_bytes_per_step": b["h2d_bytes"] // b["requests"],
                            "d2h_bytes_per_step": b["d2h_bytes"] // b["requests"]},
                    "max_abs_err_vs_fp64": None if args.no_cpu_baseline else fp64_max_error(res["checks"]),
                    "encrypt_pool_s": res["encrypt_pool_s"], "clocks": res["clocks"],
                    "cpu_baseline": None if args.no_cpu_baseline or world > 1
                    else oracle_serve_baseline(res["sides"])}
            print(json.dumps(line))
        return

    if args.impl == "reference":
        if rank != 0:
            return
        smp = OracleCnnSample(args.batch)
        for _ in range(args.warmup):
            smp.run()
        times = [smp.run() for _ in range(args.steps)]
        t_step = float(np.mean(times))
        val = args.batch * smp.fraction / t_step
        sample = (f"per step: conv-1 output column 0 of {args.batch} packed images (8 channels, 20 top-level key "
                  f"switches), {smp.fraction:.5f} of one inference by key-switch count "
                  f"(20/{ks_per_inference(SIDE)}); value = images represented / step time")
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic", "config": cfg,
                "cpu_baseline": _cpu(val, UNIT, sample),
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    res = run_gpu(args, rank, world, local_rank)
    if rank != 0:
        return
    extras = None
    if world == 1 and not args.no_extra:
        # the CNN's context went out of scope with run_gpu: release its device memory first
        import gc

        import torch
        gc.collect()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        free, total = torch.cuda.mem_get_info()
        sys.stderr.write(f"[bench] device memory free before the extra workloads: {free / 2**30:.1f} of "
                         f"{total / 2**30:.1f} GiB\n")
        extras = run_extra_workloads(args)
    cpu = None
    max_err = None
    if not args.no_cpu_baseline:
        max_err = fp64_max_error([(res["logits"], res["imgs"], res["weights"])])
    if not args.no_cpu_baseline and world == 1:
        cpu = oracle_cnn_baseline(args.batch, CNN_PRESETS[args.preset])
    line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": cfg,
            "roofline": res["roofline"], "cpu_baseline": cpu, "e2e": res["e2e"], "clocks": res["clocks"],
            "gpu_launches": res["launches"], "max_abs_err_vs_fp64": max_err,
            "alu_peak_modmul_per_s": res["modmul_peak"], "alu_peak_mac96_per_s": res["mac96_peak"],
            "alu_peak_butterfly_per_s": res["bfly_peak"],
            "plain": {"value": res["plain_value"], "ms_per_step": res["plain_ms"], "images_per_set": 1},
            "ntt_geometry": res["ntt_geometry"],
            "kernel_breakdown": res["breakdown"]}
    if extras is not None:
        line["workloads"] = extras
    print(json.dumps(line))


if __name__ == "__main__":
    main()
