"""Throughput of the deformed hash-grid radiance field hot path on one B300 (or N replicas).

One step = one training step over one batch of key-frame rays: ray sampling with
occupancy skipping, nearest-node dual-quaternion warp, hash encoding, MLPs, compositing,
Huber loss, the adjoint chain (compositing, MLPs, hash-table scatter) and Adam.

Headline workload (value, e2e, roofline): the batched key-frame step -- 8 key frames, each
with its own 2048-node graph pose and object pose, rays drawn log-uniformly between 2^14 and
2^18 per frame and field (human and object fields, L=16, T=2^19), 128 samples per ray --
in BF16 MLP with FP32 accumulation, launch shapes autotuned, the whole step captured in one
CUDA graph.  Beside it: the same frames as 8 sequential FP32 calls, the single-batch
training step (2^18 rays) in BF16 / FP16 / FP32, and the two-field 512x512 render.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|fp16|bf16] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas (the path has
no exchange step at one GPU per key-frame set); value = all ranks' samples / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "train samples/s (fwd+bwd) & render Mrays/s, mixed-prec vs FP32 at fixed error"
UNIT = "samples/s"
# kernels launched per TIMED record of the library (scan = 3 kernels, composite_train = 2,
# march_count = 2: the occupied-cell bounds, then the count)
KERNELS_PER_RECORD = {"scan": 3, "composite_train": 2, "march_count": 2}


def launches_per_record(n_fields):
    """Kernels per timed record for a step over n_fields fields: the encoding, fused forward
    and scatter records launch once per field."""
    return dict(KERNELS_PER_RECORD, encode=n_fields, warp_encode=n_fields, encode_bwd=n_fields)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--prec", choices=["fp32", "fp16", "bf16"], default="bf16")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rays", type=int, default=1 << 18)
    ap.add_argument("--no-render", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-interleave", action="store_true")
    ap.add_argument("--no-lut", action="store_true")
    ap.add_argument("--no-deform", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="time only the batched key-frame step (no single-batch, FP32, render, LUT sections)")
    ap.add_argument("--render-only", action="store_true",
                    help="time only the two-field 512x512 render (all three precisions; for launch lists)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--kf-frames", type=int, default=8,
                    help="key frames of the batched workload (smaller cases for ncu captures)")
    ap.add_argument("--kf-log2-rays", type=float, nargs=2, default=(14.0, 18.0),
                    help="range of log2(rays) per frame and field of the batched workload")
    ap.add_argument("--tune", type=str, default=None,
                    help="fixed launch shapes of the batched step as JSON (keys of Context.TUNE_KEYS; the "
                         "rest keep the context's defaults) instead of autotuning")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks sampling
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device, self.rows, self.proc = device, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.rows and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.05)
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ workloads
def build_train(invr, ctx, tw, prec, loss="huber"):
    import torch
    fields = {id(fp): invr.Field.from_synth(ctx, fp, prec) for fp in tw.fields}
    keep, batches = [], []
    for b in tw.batches:
        g = None
        if b.view.graph is not None:
            sg = b.view.graph
            g = invr.Graph(ctx, sg.x_canon.shape[1], sg.K, sg.radius, 1, torch.from_numpy(sg.x_canon).cuda())
            g.set_pose(0, torch.from_numpy(sg.dq).cuda(), torch.from_numpy(sg.x_live).cuda())
        occ = torch.from_numpy(b.view.occupancy).cuda() if b.view.occupancy is not None else None
        view = invr.View(fields[id(b.view.field)], g, 0, b.view.rigid_dq, occ)
        o = torch.from_numpy(b.rays.o).cuda()
        d = torch.from_numpy(b.rays.d).cuda()
        t = torch.from_numpy(b.target).cuda()
        keep.append((g, occ, view))
        if loss == "paper":      # the paper's masked colour L2 + depth L1 losses
            batches.append((o, d, view, t, torch.from_numpy(b.mask).cuda(), torch.from_numpy(b.depth).cuda()))
        else:
            batches.append((o, d, view, t))
    tb = invr.TrainBatches(batches, tw.n_samples, tw.t_eps, tw.huber_delta, tw.lr, tw.beta1, tw.beta2, tw.adam_eps,
                           loss=loss)
    return tb, fields, keep


def occupied_samples(invr, ctx, tb):
    """Occupied samples per batch (the samples the path evaluates), via the sampling step."""
    total = 0
    for (o, d, view, *_) in tb.batches:
        count, _, _ = invr.ray_samples(ctx, o, d, tb.args.batches[0].n_samples, view.occupancy)
        total += int(count.sum().item())
    return total


# algorithmic work per kernel of one training step
def kernel_work(name, R, S_occ, n_samples, L, n_params, n_w):
    """(bound, algorithmic work per launch) of one kernel of the training step: FLOPs for the
    MLPs (2 per multiply-add of the unpadded layers), bytes for the streaming/gather ones."""
    mlp_f = 2 * n_w                       # FLOPs per sample, forward
    if name == "mlp_fwd":
        return "alu", S_occ * mlp_f
    if name == "mlp_bwd":
        return "alu", S_occ * 3 * mlp_f   # recompute forward + input grads + weight grads
    if name == "mlp_fwd_tc":
        return "tensor", S_occ * mlp_f
    if name == "mlp_bwd_tc":
        return "tensor", S_occ * 3 * mlp_f
    if name == "adam":
        return "hbm", n_params * 32       # read p,g,m,v; write p,g(=0),m,v
    if name == "encode":
        return "hbm", S_occ * (12 + L * (8 * 8 + 8))    # vc in, 8 corner gathers + 2 features out per level
    if name == "warp_encode":
        return "hbm", S_occ * (24 + L * (8 * 8 + 8))   # live position in, v_c out, the encoding's gathers and out
    if name == "encode_bwd":
        return "hbm", S_occ * (12 + L * (8 + 8 * 8))    # vc, dfeat in, 8 corner atomics per level
    if name == "march_count":
        return "hbm", R * 28
    if name == "march_emit":
        return "hbm", R * 32 + S_occ * 20            # o, d, first, count in; ray id, t, position out
    if name == "composite_train":
        return "hbm", R * 48 + S_occ * 36            # per sample sigma, rgb, t in, dL/dout out
    if name == "warp":
        return "hbm", S_occ * 24                     # live position in, canonical out (latency-bound)
    return None, None


def fp32_alu_peak(sm_mhz):
    return 148 * 128 * 2 * sm_mhz * 1e6 / 1e12   # TFLOP/s, FP32 FMA pipes


PRECS = {"fp32": 0, "fp16": 1, "bf16": 2}


def aggregate_replicas(ms_local: float, samples_local: float, world: int):
    """Whole-job throughput of independent replicas: every rank's samples over the slowest
    rank's time (max over ranks of the per-step milliseconds).  Returns (value, max_ms)."""
    ms = ms_local
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * samples_local / (ms * 1e-3), ms


def time_train(invr, ctx, tb, steps, warmup, flush, world):
    """Per-step CUDA-event times (L2 flushed between steps) and the per-kernel breakdown."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        invr.train_step(ctx, tb)
    ctx.sync()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ctx.enable_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush.fill_(1)                    # L2 flush between steps (outside the timed events)
        a.record(stream)
        invr.train_step(ctx, tb)
        b.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ktime = ctx.timing()
    ctx.enable_timing(False)
    ctx.sync()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    _, ms = aggregate_replicas(ms, 1.0, world)
    return ms, ktime


def measure_l2(invr, ctx):
    """L2 ceilings measured on this device by the library's probe kernels: a read stream over
    a 64 MiB resident buffer (the size of one field's tables), and random 32-byte / float4 /
    float2 loads from it and float4 / float2 atomic adds into it (the forms the encoding's
    gathers and the hash-gradient scatter issue).  Best of 5, CUDA events."""
    import torch
    buf = torch.ones(1 << 24, dtype=torch.float32, device="cuda")        # 64 MiB < 126 MB L2
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def best(fn, nbytes):
        fn()                                                             # warm: buffer into L2
        out = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            out.append(nbytes / (a.elapsed_time(b) * 1e-3) / 1e9)
        return max(out)
    passes, n_ops = 40, 1 << 27
    res = {"read_gbs": best(lambda: invr.probe_l2_read(ctx, buf, passes, sink), passes * buf.numel() * 4),
           "atomic_v4_gbs": best(lambda: invr.probe_l2_atomic(ctx, buf, 4, n_ops), n_ops * 16),
           "atomic_v2_gbs": best(lambda: invr.probe_l2_atomic(ctx, buf, 2, n_ops), n_ops * 8),
           "gather_v8_gbs": best(lambda: invr.probe_l2_gather(ctx, buf, 8, n_ops, sink), n_ops * 32),
           "gather_v4_gbs": best(lambda: invr.probe_l2_gather(ctx, buf, 4, n_ops, sink), n_ops * 16),
           "gather_v2_gbs": best(lambda: invr.probe_l2_gather(ctx, buf, 2, n_ops, sink), n_ops * 8)}
    ctx.sync()
    return {k: round(v, 1) for k, v in res.items()}


def l2_roofline(name, kms_per_launch, S_occ, L, l2):
    """The L2 view of a gather/scatter kernel: table payload per launch (8 corners x F=2
    floats per level and sample) over its duration, against the probe's ceiling for that
    access form."""
    if l2 is None or name not in ("encode", "warp_encode", "encode_bwd"):
        return None
    payload = S_occ * L * 8 * 2 * 4
    ach = payload / (kms_per_launch * 1e-3) / 1e9
    gather = name != "encode_bwd"
    peak = l2["gather_v4_gbs"] if gather else l2["atomic_v4_gbs"]
    return {"achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
            "payload_bytes": payload,
            "peak_source": "measured by probe: random float4 " + ("loads from" if gather
                                                                  else "atomic adds into") + " a 64 MiB table"}


# The encoding's gather and the gradient scatter keep the tables (64 MiB per field) in L2:
# their bound is the L2, measured in the same run by the library's probe kernels.
L2_BOUND = {"encode": ("gather_v4_gbs", "random float4 loads from"),
            "warp_encode": ("gather_v4_gbs", "random float4 loads from"),
            "encode_bwd": ("atomic_v4_gbs", "random float4 atomic adds into")}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one step's scatter launches
# (both fields) on the batched key-frame workload, from one ncu capture of that workload,
# with a digest of the scatter's source files at the time of the capture: the bench line
# carries the figure only while the kernel is unchanged (else traffic is null).
SCATTER_SOURCES = ("paper_2304_03184_b300/csrc/k_encode.cu", "paper_2304_03184_b300/csrc/hash_grid.cuh")
SCATTER_DRAM = {"sources_sha16": "d25467f8f6c6be0c", "workload": "keyframe_batch_8frames_x2fields_s128",
                "bytes": 2_212_720_000, "l2_bytes": 53_630_000_000}


def sources_sha16(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def scatter_traffic(workload, key="bytes"):
    """The captured DRAM bytes (key "bytes") or L2 bytes ("l2_bytes") of the scatter per step, or
    None (no capture of this workload, or the kernel's sources changed since)."""
    if not SCATTER_DRAM or SCATTER_DRAM["workload"] != workload:
        return None
    return SCATTER_DRAM[key] if sources_sha16(SCATTER_SOURCES) == SCATTER_DRAM["sources_sha16"] else None


def roofline(ktime, tw, R, S_occ, peaks, l2=None):
    fp = tw.fields[0]
    n_params = fp.desc.n_table_params() + fp.desc.n_weight_params()
    name, (kms, kn) = max(ktime.items(), key=lambda kv: kv[1][0])
    bound, work = kernel_work(name, R, S_occ, tw.n_samples, fp.desc.L, n_params, fp.desc.n_weight_params())
    dur = kms / kn * 1e-3
    if name in L2_BOUND and l2:
        # algorithmic bytes: the table payload, 8 corners x F = 2 floats per level and sample
        payload = S_occ * fp.desc.L * 8 * 2 * 4
        key, form = L2_BOUND[name]
        ach, peak = payload / dur / 1e9, l2[key]
        hbm_peak = peaks.get("hbm_gbs", 6400.0)
        traffic = scatter_traffic(tw.name) if name == "encode_bwd" else None
        l2_bytes = scatter_traffic(tw.name, "l2_bytes") if name == "encode_bwd" else None
        return {"kernel": name, "bound": "l2", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": traffic,
                "l2_traffic": l2_bytes,
                "l2_traffic_gbs": round(l2_bytes / dur / 1e9, 1) if l2_bytes else None,
                "peak_source": f"measured in this run by the library's L2 probe: {form} a 64 MiB resident table",
                "algorithmic_bytes": payload, "ms": round(kms / kn, 4),
                "hbm": {"bytes": work, "achieved": round(work / dur / 1e9, 1), "peak": hbm_peak,
                        "frac": round(work / dur / 1e9 / hbm_peak, 4),
                        "note": "the kernel's per-sample inputs and outputs; the table traffic stays in L2"},
                "traffic_note": ("DRAM bytes (traffic) and L2 bytes (lts__t_bytes, l2_traffic) of the stage from "
                                 "ncu captures of this workload at the current kernel sources (the table traffic "
                                 "stays in L2)" if traffic is not None else
                                 "no ncu capture of this workload at the current kernel sources")}
    if bound == "alu":
        peak = fp32_alu_peak(peaks.get("sm_max_mhz", 2032.0))
        ach = work / dur / 1e12
        return {"kernel": name, "bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 1),
                "unit": "TFLOP/s", "frac": round(ach / peak, 4), "traffic": None,
                "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 x max SM clock"}
    if bound == "tensor":
        peak = peaks.get("bf16_tflops_sustained", 1400.0)
        ach = work / dur / 1e12
        return {"kernel": name, "bound": "tensor", "achieved": round(ach, 2), "peak": peak, "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "traffic": None,
                "peak_source": "measured (sustained dense bf16)" if "bf16_tflops_sustained" in peaks else "fallback"}
    if bound == "hbm":
        peak = peaks.get("hbm_gbs", 6400.0)
        ach = work / dur / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": None,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "l2": l2_roofline(name, kms / kn, S_occ, fp.desc.L, l2)}
    return None


def kernel_rooflines(ktime, tw, R, S_occ, peaks, l2=None):
    """Every timed kernel of the step against the roofline that bounds its work: algorithmic
    work per timed record (a step stage over all batches; Adam: one field) -- FLOPs of the
    unpadded MLP layers, or bytes -- over its CUDA-event time,
    as a fraction of the measured peak (HBM copy bandwidth, sustained dense BF16, or the FP32
    FMA peak derived from the SM count and the maximum SM clock).  The gather and the
    scatter, whose tables stay in L2, are given against the L2 probe ceilings when measured
    (table payload per second: lanes that share a vertex are served by one L2 operation, so
    the ratio can pass 1)."""
    fp = tw.fields[0]
    n_params = fp.desc.n_table_params() + fp.desc.n_weight_params()  # Adam is timed per field
    res = {}
    for name, (kms, kn) in sorted(ktime.items()):
        bound, work = kernel_work(name, R, S_occ, tw.n_samples, fp.desc.L, n_params, fp.desc.n_weight_params())
        if bound is None:
            continue
        if name in ("encode", "warp_encode", "encode_bwd") and l2:
            r = l2_roofline(name, kms / kn, S_occ, fp.desc.L, l2)
            res[name] = {"bound": "l2", **{k: r[k] for k in ("achieved", "peak", "unit", "frac")},
                         "ms": round(kms / kn, 4)}
            continue
        dur = kms / kn * 1e-3
        if bound == "hbm":
            peak, unit, ach = peaks.get("hbm_gbs", 6400.0), "GB/s", work / dur / 1e9
        elif bound == "tensor":
            peak, unit, ach = peaks.get("bf16_tflops_sustained", 1400.0), "TFLOP/s", work / dur / 1e12
        else:
            peak, unit, ach = fp32_alu_peak(peaks.get("sm_max_mhz", 2032.0)), "TFLOP/s", work / dur / 1e12
        res[name] = {"bound": bound, "achieved": round(ach, 1), "peak": round(peak, 1), "unit": unit,
                     "frac": round(ach / peak, 4), "ms": round(kms / kn, 4)}
    return res


def headline_config(tw, world):
    """The workload the headline is quoted on (both arms print the same object)."""
    return {"workload": tw.name, "rays": int(sum(b.rays.n for b in tw.batches)), "samples_per_ray": tw.n_samples,
            "batches": len(tw.batches), "fields": len(tw.fields), "parallelism": f"replicas{world}",
            "l2": "inputs and per-sample buffers larger than L2; the GPU arm also flushes L2 (256 MiB write) "
                  "between timed steps",
            "samples_counted": "nominal: rays x samples_per_ray per step (value_occupied: the occupied samples "
                               "the path evaluates)"}


def apply_batched(out, bt, invr, ctx, args, world, peaks):
    """Fill the bench line from the batched key-frame run (the headline workload)."""
    bvalue = world * bt["S_nom"] / (bt["ms"] * 1e-3)
    btw = bt["tw"]
    out["value"] = round(bvalue, 1)
    out["value_occupied"] = round(world * bt["occupied_samples"] / (bt["ms"] * 1e-3), 1)
    out["ms_per_step"] = round(bt["ms"], 3)
    out["config"] = headline_config(btw, world)
    out["run"] = {"occupied_samples": bt["occupied_samples"], "prec": args.prec,
                  "launch": "one CUDA graph per step (all batches per stage launch)", "tune": bt["tune"]}
    out["e2e"] = bt["e2e"]
    bR, bS = bt["rays"], bt["occupied_samples"]
    l2 = measure_l2(invr, ctx)
    out["l2_probe"] = l2
    out["roofline"] = roofline(bt["ktime"], btw, bR, bS, peaks, l2)
    out["l2_rooflines"] = {k: l2_roofline(k, bt["ktime"][k][0] / bt["ktime"][k][1], bS, btw.fields[0].desc.L, l2)
                           for k in ("encode", "warp_encode", "encode_bwd") if k in bt["ktime"]}
    nsteps = max(5, args.steps // 4)
    out["kernels_ms_per_step"] = {k: round(v[0] / nsteps, 4) for k, v in sorted(bt["ktime"].items())}
    out["kernel_rooflines"] = kernel_rooflines(bt["ktime"], btw, bR, bS, peaks, l2)
    per_rec = launches_per_record(len(btw.fields))
    # the per-kernel records come from eager steps with timing on (one stream); the timed graph
    # splits the MLP backward of a two-field 16-bit step in two (one launch per field)
    split_bwd = 1 if (len(btw.fields) == 2 and args.prec != "fp32") else 0
    out["gpu_launches"] = int(round(sum(n * per_rec.get(k, 1) for k, (_, n) in bt["ktime"].items())
                                    / nsteps * args.steps)) + split_bwd * args.steps
    out["gpu_launches_per_step"] = round(out["gpu_launches"] / args.steps, 1)
    out["variants"] = {args.prec + "_graph": {"value": round(bvalue, 1), "ms_per_step": round(bt["ms"], 3)},
                       args.prec + "_eager": {"value": round(world * bt["S_nom"] / (bt["eager_ms"] * 1e-3), 1),
                                              "ms_per_step": round(bt["eager_ms"], 3)},
                       "fp32_sequential": bt["fp32_sequential"]}


def run_ours(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    from paper_2304_03184_b300 import build, synth
    build.build()
    import paper_2304_03184_b300 as invr
    ctx = invr.Context(local)
    tw = synth.train_step_workload(n_rays=args.rays)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # 256 MiB > 126 MB L2
    clocks = ClockSampler(local)
    clocks.start()
    if args.headline_only:        # the batched key-frame step alone (clean launch lists)
        out = {"metric": METRIC, "value": None, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else f"{args.prec}-mlp/f32",
               "data": "synthetic", "clocks": None}
        bt = bench_batched(invr, args, flush, world, args.prec, with_fp32=False)
        apply_batched(out, bt, invr, ctx, args, world, peaks)
        out["clocks"] = clocks.stop()
        return out, bt["tw"]

    # the requested precision, then the other two for the mixed-vs-FP32 comparison
    order = [args.prec] + [p for p in ("fp32", "fp16", "bf16") if p != args.prec]
    if args.render_only:          # the two-field render alone (clean launch lists)
        render = {p: bench_render(invr, ctx, PRECS[p], args, flush) for p in order}
        out = {"metric": "render Mrays/s (two-field 512x512)", "value": render[args.prec]["value"],
               "unit": "Mrays/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": render[args.prec]["ms_per_frame"], "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else f"{args.prec}-mlp/f32",
               "data": "synthetic", "render": render, "clocks": clocks.stop()}
        return out, tw
    variants, main = {}, None
    for p in order:
        tb, fields, keep = build_train(invr, ctx, tw, PRECS[p])
        if main is None:
            R = sum(b[0].shape[1] for b in tb.batches)
            S_nom = R * tw.n_samples
            S_occ = occupied_samples(invr, ctx, tb)
        steps = args.steps if p == args.prec else max(5, args.steps // 4)
        ms, ktime = time_train(invr, ctx, tb, steps, args.warmup, flush, world)
        variants[p] = {"value": round(world * S_nom / (ms * 1e-3), 1), "ms_per_step": round(ms, 3),
                       "kernels_ms_per_step": {k: round(v[0] / steps, 4) for k, v in sorted(ktime.items())}}
        if main is None:
            main = (tb, fields, keep, ms, ktime)
    # the paper's losses (masked colour L2 + depth L1) in place of the Huber penalty
    tbp, fields_p, keep_p = build_train(invr, ctx, tw, PRECS[args.prec], loss="paper")
    steps_p = max(5, args.steps // 4)
    ms_p, ktime_p = time_train(invr, ctx, tbp, steps_p, args.warmup, flush, world)
    variants[args.prec + "_paper_loss"] = {
        "value": round(world * S_nom / (ms_p * 1e-3), 1), "ms_per_step": round(ms_p, 3),
        "kernels_ms_per_step": {k: round(v[0] / steps_p, 4) for k, v in sorted(ktime_p.items())}}
    del tbp, fields_p, keep_p
    tb, fields, keep, ms, ktime = main
    value = world * S_nom / (ms * 1e-3)
    per_rec = launches_per_record(len(tw.fields))
    launches = sum(n * per_rec.get(k, 1) for k, (_, n) in ktime.items())
    roof = roofline(ktime, tw, R, S_occ, peaks)

    # end to end through the public API with host buffers: rays + targets in, loss out, every
    # step.  Two sets of input buffers: step i+1's inputs are copied host -> device on a copy
    # stream into the other set while step i runs (eager calls, as the device timing above).
    host_in = [(b[0].cpu().pin_memory(), b[1].cpu().pin_memory(), b[3].cpu().pin_memory()) for b in tb.batches]
    loss_h = torch.empty(1, pin_memory=True)
    h2d = sum(x.numel() * 4 for trip in host_in for x in trip)
    stream = torch.cuda.current_stream()
    tb2 = invr.TrainBatches([(b[0].clone(), b[1].clone(), b[2], b[3].clone()) for b in tb.batches], tw.n_samples,
                            tw.t_eps, tw.huber_delta, tw.lr, tw.beta1, tw.beta2, tw.adam_eps)
    sets = [tb, tb2]
    cs = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def copy_in(i):
        t = sets[i % 2]
        with torch.cuda.stream(cs):
            cs.wait_event(consumed[i % 2] if i >= 2 else a)
            off = 0
            for j, (ho, hd, ht) in enumerate(host_in):
                t.batches[j][0].copy_(ho, non_blocking=True)
                t.batches[j][1].copy_(hd, non_blocking=True)
                t.targets[off:off + ht.numel()].copy_(ht.reshape(-1), non_blocking=True)  # [3][R_b] per batch
                off += ht.numel()
            copied[i % 2].record(cs)

    invr.train_step(ctx, tb2)              # the second set's first call plans outside the timed region
    torch.cuda.synchronize()
    a.record(stream)
    copy_in(0)
    for i in range(args.steps):
        if i + 1 < args.steps:
            copy_in(i + 1)
        stream.wait_event(copied[i % 2])
        flush.fill_(1)                    # L2 flushed before every step, as in the device timing
        loss = invr.train_step(ctx, sets[i % 2])
        consumed[i % 2].record(stream)
        loss_h.copy_(loss, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    e_ms = a.elapsed_time(b) / args.steps
    e2e = {"value": round(world * S_nom / (e_ms * 1e-3), 1), "unit": UNIT, "ms_per_step": round(e_ms, 3),
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4,
           "copies": "pinned host -> device on a copy stream into one of two input sets (next step's under "
                     "this one), eager calls, loss read back every step; L2 flushed before every step"}
    del tb2, sets

    render = None
    if not args.no_render:
        render = {p: bench_render(invr, ctx, PRECS[p], args, flush) for p in order}

    single = {"workload": tw.name, "rays": R, "samples_per_ray": tw.n_samples, "occupied_samples": S_occ,
              "value": round(value, 1), "ms_per_step": round(ms, 3), "e2e": e2e, "roofline": roof,
              "variants": variants}
    out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else f"{args.prec}-mlp/f32",
           "data": "synthetic",
           "config": {"workload": tw.name, "rays": R, "samples_per_ray": tw.n_samples,
                      "occupied_samples": S_occ, "fields": len(tw.fields), "parallelism": f"replicas{world}",
                      "l2": "flushed between timed steps (256 MiB write)", "prec": args.prec},
           "roofline": roof, "e2e": e2e, "render": render, "variants": variants, "clocks": None,
           "gpu_launches": launches,
           "kernels_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in sorted(ktime.items())}}
    if not args.no_batched:
        bt = bench_batched(invr, args, flush, world, args.prec)
        apply_batched(out, bt, invr, ctx, args, world, peaks)
        out["single_batch_train"] = single
        tw = bt["tw"]
    if not args.no_lut:
        out["lut_search"] = bench_lut(invr, args, flush, world, args.prec)
    if not args.no_deform:
        out["deform_net"] = bench_deform(invr, args, flush, world, args.prec)
    if not args.no_interleave:
        out["interleave"] = bench_interleave(invr, args, args.prec)
    out["clocks"] = clocks.stop()      # sampled over every timed region above
    return out, tw


def frames_of(tw):
    """Split the key-frame workload's batches (frame-major: human, object) per frame."""
    from paper_2304_03184_b300 import synth
    out = []
    for i in range(0, len(tw.batches), 2):
        out.append(synth.TrainWorkload(tw.name, tw.batches[i:i + 2], tw.fields, tw.n_samples, tw.t_eps,
                                       tw.huber_delta, tw.lr, tw.beta1, tw.beta2, tw.adam_eps))
    return out


def bench_batched(invr, args, flush, world, prec_name, with_fp32=True):
    """Headline: batched key-frame step, mixed precision, autotuned, one CUDA graph per step;
    with_fp32 adds the plain comparison (the same frames as sequential FP32 calls)."""
    import torch
    from paper_2304_03184_b300 import synth
    tw = synth.keyframe_batch_workload(n_frames=args.kf_frames, log2_rays=tuple(args.kf_log2_rays))
    R = sum(b.rays.n for b in tw.batches)
    S_nom = R * tw.n_samples
    stream = torch.cuda.current_stream()

    ctx = invr.Context(torch.cuda.current_device())
    tb, fields, keep = build_train(invr, ctx, tw, PRECS[prec_name])
    S_occ = occupied_samples(invr, ctx, tb)
    ctx.reserve(R, max(32, 2 * (S_occ // R + 1)))       # fixed workspace: capture allocates nothing
    if args.tune:
        tune = dict(ctx.tune(), **json.loads(args.tune))
        ctx.set_tune(tune)
        tune = ctx.tune()
    else:
        tune = ctx.autotune(tb)
    # eager timed steps: per-kernel breakdown (same kernels as the graph)
    eager_ms, ktime = time_train(invr, ctx, tb, max(5, args.steps // 4), args.warmup, flush, world)
    graph = invr.TrainGraph(ctx, tb, warmup=2)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in ev:
        flush.fill_(1)
        a.record(stream)
        graph.replay()
        b.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    _, ms = aggregate_replicas(ms, 1.0, world)
    ctx.sync()

    # end to end: every step's rays and targets come from pinned host memory and its loss goes
    # back to the host.  Pipelined as a caller streaming key frames would: two sets of the
    # step's input buffers, each with its own captured graph; step i+1's inputs are copied
    # host -> device on a copy stream into the other set while step i's graph runs, and each
    # step replays its set's graph and reads the loss back.  The first step's copy is inside
    # the timed region, and so is an L2 flush before every step.
    host_in = [(b[0].cpu().pin_memory(), b[1].cpu().pin_memory(), b[3].cpu().pin_memory()) for b in tb.batches]
    loss_h = torch.empty(1, pin_memory=True)
    h2d = sum(x.numel() * 4 for trip in host_in for x in trip)
    tb2 = invr.TrainBatches([(b[0].clone(), b[1].clone(), b[2], b[3].clone()) for b in tb.batches], tw.n_samples,
                            tw.t_eps, tw.huber_delta, tw.lr, tw.beta1, tw.beta2, tw.adam_eps)
    sets = [(tb, graph), (tb2, invr.TrainGraph(ctx, tb2, warmup=2))]
    cs = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]     # host -> input set done
    consumed = [torch.cuda.Event() for _ in range(2)]   # the set's step has run
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def copy_in(i):
        t = sets[i % 2][0]
        with torch.cuda.stream(cs):
            cs.wait_event(consumed[i % 2] if i >= 2 else a)
            off = 0
            for j, (ho, hd, ht) in enumerate(host_in):
                t.batches[j][0].copy_(ho, non_blocking=True)
                t.batches[j][1].copy_(hd, non_blocking=True)
                t.targets[off:off + ht.numel()].copy_(ht.reshape(-1), non_blocking=True)
                off += ht.numel()
            copied[i % 2].record(cs)

    torch.cuda.synchronize()
    a.record(stream)
    copy_in(0)
    for i in range(args.steps):
        if i + 1 < args.steps:
            copy_in(i + 1)
        stream.wait_event(copied[i % 2])
        flush.fill_(1)                    # L2 flushed before every step, as in the device timing
        loss = sets[i % 2][1].replay()
        consumed[i % 2].record(stream)
        loss_h.copy_(loss, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    e_ms = a.elapsed_time(b) / args.steps
    e2e = {"value": round(world * S_nom / (e_ms * 1e-3), 1), "unit": UNIT, "ms_per_step": round(e_ms, 3),
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4,
           "copies": "pinned host -> device on a copy stream into the inputs of one of two captured step "
                     "graphs (next step's under this one), loss read back every step; L2 flushed before "
                     "every step"}
    out = {"workload": tw.name, "rays": R, "samples_per_ray": tw.n_samples, "occupied_samples": S_occ,
           "batches": len(tw.batches), "S_nom": S_nom, "ms": ms, "eager_ms": eager_ms, "ktime": ktime,
           "tune": tune, "e2e": e2e, "tw": tw, "fp32_sequential": None}
    if not with_fp32:
        return out
    # plain path: the same frames as 8 sequential FP32 calls (2 batches each), no graph
    ctx32 = invr.Context(torch.cuda.current_device())
    per_frame = [build_train(invr, ctx32, fw, PRECS["fp32"]) for fw in frames_of(tw)]
    for _ in range(2):
        for fb in per_frame:
            invr.train_step(ctx32, fb[0])
    ctx32.sync()
    steps32 = max(3, args.steps // 8)
    ev32 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps32)]
    for a, b in ev32:
        flush.fill_(1)
        a.record(stream)
        for fb in per_frame:
            invr.train_step(ctx32, fb[0])
        b.record(stream)
    torch.cuda.synchronize()
    ms32 = float(np.mean([a.elapsed_time(b) for a, b in ev32]))
    ctx32.sync()
    out["fp32_sequential"] = {"value": round(world * S_nom / (ms32 * 1e-3), 1), "ms_per_step": round(ms32, 3),
                              "launches": "8 sequential train_step calls (2 batches each), FP32, no graph"}
    return out


def build_views(invr, ctx, w, prec):
    import torch
    keep, views = [], []
    for sv in w.views:
        f = invr.Field.from_synth(ctx, sv.field, prec)
        g = None
        if sv.graph is not None:
            gg = sv.graph
            g = invr.Graph(ctx, gg.x_canon.shape[1], gg.K, gg.radius, 1, torch.from_numpy(gg.x_canon).cuda())
            g.set_pose(0, torch.from_numpy(gg.dq).cuda(), torch.from_numpy(gg.x_live).cuda())
        occ = torch.from_numpy(sv.occupancy).cuda()
        keep.append((f, g, occ))
        views.append(invr.View(f, g, 0, sv.rigid_dq, occ))
    return views, keep


def bench_lut(invr, args, flush, world, prec_name, G=512):
    """The look-up-table neighbour search (Sec. 4.2) against the exact search on the
    single-batch train step, for two motions of the 2048-node graph: the workload's own
    (every node rotated independently about the origin) and a spatially coherent
    articulated pose.  Per motion: table build times, the warp kernel and the whole step,
    and on the occupied samples of 2^15 rays the fraction in table holes, the fraction whose
    table neighbour set equals the exact K nearest, and the canonical-position difference
    of the two warps (median, 99th percentile)."""
    import torch
    from paper_2304_03184_b300 import synth
    base = synth.train_step_workload(n_rays=args.rays)
    b0 = base.batches[0]
    g_art = synth.articulated_pose(np.random.default_rng(9), b0.view.graph)
    out = {"workload": base.name, "resolution": G, "prec": prec_name, "forward": "staged (warp timed alone)"}
    for motion, g in (("independent_nodes", b0.view.graph), ("articulated", g_art)):
        occ = b0.view.occupancy if g is b0.view.graph else synth.occupancy_near_nodes(g.x_live)
        view_s = synth.View(b0.view.field, graph=g, occupancy=occ)
        tw = synth.TrainWorkload(base.name, [synth.TrainBatch(b0.rays, view_s, b0.target)], base.fields,
                                 base.n_samples)
        ctx = invr.Context(torch.cuda.current_device())
        ctx.set_tune(dict(ctx.tune(), fused=0))   # staged forward: the warp kernel timed on its own
        tb, fields, keep = build_train(invr, ctx, tw, PRECS[prec_name])
        graph, view = keep[0][0], keep[0][2]
        steps = max(5, args.steps // 4)
        ms_exact, kt_exact = time_train(invr, ctx, tb, steps, args.warmup, flush, world)
        stream = torch.cuda.current_stream()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        dq, xl = torch.from_numpy(g.dq).cuda(), torch.from_numpy(g.x_live).cuda()
        torch.cuda.synchronize()
        a.record(stream)
        graph.enable_lut(G)                      # canonical field + this frame's live field
        b.record(stream)
        graph.set_pose(0, dq, xl)                # per frame: pack, candidate grid, live field
        c.record(stream)
        torch.cuda.synchronize()
        enable_ms, pose_ms = a.elapsed_time(b), b.elapsed_time(c)
        ms_lut, kt_lut = time_train(invr, ctx, tb, steps, args.warmup, flush, world)

        o, d = tb.batches[0][0][:, :1 << 15].contiguous(), tb.batches[0][1][:, :1 << 15].contiguous()
        count, _, pos = invr.ray_samples(ctx, o, d, tw.n_samples, view.occupancy)
        keep_s = torch.arange(tw.n_samples, device="cuda")[None, :] < count[:, None].long()
        p = pos[:, keep_s].contiguous()
        vc_lut, ids_lut = invr.warp_points(ctx, view, p, with_ids=True)
        _, live = graph.get_lut(0)
        vox = torch.clamp(torch.floor(((p + 1.0) * 0.5) * G).long(), 0, G - 1)
        hole = live[vox[0] + G * (vox[1] + G * vox[2])] == -1
        del live
        graph.disable_lut()
        vc_exact, ids_exact = invr.warp_points(ctx, view, p, with_ids=True)
        same = torch.all(torch.sort(ids_lut, dim=0)[0] == torch.sort(ids_exact, dim=0)[0], dim=0)
        err = torch.linalg.vector_norm(vc_lut - vc_exact, dim=0)
        ctx.sync()
        S_nom = tb.batches[0][0].shape[1] * tw.n_samples
        out[motion] = {
            "enable_ms": round(enable_ms, 3), "set_pose_ms": round(pose_ms, 3),
            "exact": {"value": round(world * S_nom / (ms_exact * 1e-3), 1), "ms_per_step": round(ms_exact, 3),
                      "warp_ms": round(kt_exact["warp"][0] / steps, 4)},
            "lut": {"value": round(world * S_nom / (ms_lut * 1e-3), 1), "ms_per_step": round(ms_lut, 3),
                    "warp_ms": round(kt_lut["warp"][0] / steps, 4)},
            "samples_checked": int(p.shape[1]), "hole_fraction": round(float(hole.float().mean()), 4),
            "neighbour_set_agreement": round(float(same.float().mean()), 4),
            "canonical_position_diff": {"median": float(err.median()), "p99": float(torch.quantile(err, 0.99))}}
        del tb, fields, keep, graph, view, ctx
    return out


def bench_deform(invr, args, flush, world, prec_name):
    """The pose-conditioned deformation net (32 hash features + 72 pose -> 4 x 128 -> 3, FP32)
    in front of the human field: the single-batch training step and the 512x512 human render,
    with and without the net, and the per-kernel breakdown of the training step."""
    import torch
    from paper_2304_03184_b300 import synth
    rng = np.random.default_rng(11)
    tw = synth.train_step_workload(n_rays=args.rays)
    dp, pose = synth.make_deform(rng), synth.make_pose(rng)
    ctx = invr.Context(torch.cuda.current_device())
    tb, fields, keep = build_train(invr, ctx, tw, PRECS[prec_name])
    R = tb.batches[0][0].shape[1]
    # sample slots (and the net's operand tiles) for ~12 occupied per ray, for the training
    # rays and the 512x512 render below
    ctx.reserve(max(R, 512 * 512), 32)
    steps = max(5, args.steps // 4)
    ms_plain, _ = time_train(invr, ctx, tb, steps, args.warmup, flush, world)
    net = invr.Deform.from_synth(ctx, dp)
    pose_d = torch.from_numpy(pose).cuda()
    g, occ, view = keep[0]
    dview = invr.View(view.field, g, 0, None, occ, net, pose_d)
    b = tb.batches[0]
    tbd = invr.TrainBatches([(b[0], b[1], dview, b[3])], tw.n_samples, tw.t_eps, tw.huber_delta, tw.lr, tw.beta1,
                            tw.beta2, tw.adam_eps)
    ms_def, kt = time_train(invr, ctx, tbd, steps, args.warmup, flush, world)
    # the net on the tensor cores (FP16 operands, forward and backward)
    net_tc = invr.Deform.from_synth(ctx, dp, PRECS["fp16"])
    tview = invr.View(view.field, g, 0, None, occ, net_tc, pose_d)
    tbt = invr.TrainBatches([(b[0], b[1], tview, b[3])], tw.n_samples, tw.t_eps, tw.huber_delta, tw.lr, tw.beta1,
                            tw.beta2, tw.adam_eps)
    ms_tc, kt_tc = time_train(invr, ctx, tbt, steps, args.warmup, flush, world)
    S_nom = b[0].shape[1] * tw.n_samples
    w = synth.two_field_render()
    o, d = torch.from_numpy(w.rays.o).cuda(), torch.from_numpy(w.rays.d).cuda()
    stream = torch.cuda.current_stream()

    def render_ms(v):
        for _ in range(3):
            invr.render_rays(ctx, o, d, w.n_samples, w.t_eps, [v])
        ctx.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, e in ev:
            flush.fill_(1)
            a.record(stream)
            invr.render_rays(ctx, o, d, w.n_samples, w.t_eps, [v])
            e.record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(e) for a, e in ev]))
    r_plain, r_def, r_tc = render_ms(view), render_ms(dview), render_ms(tview)
    net.close()
    net_tc.close()
    return {"workload": tw.name, "net": "32 hash features + 72 pose -> 4 x 128 -> 3 (FP32 SIMT, or FP16 tcgen05)",
            "field_prec": prec_name,
            "train": {"with_net": {"value": round(world * S_nom / (ms_def * 1e-3), 1), "ms_per_step": round(ms_def, 3)},
                      "without": {"value": round(world * S_nom / (ms_plain * 1e-3), 1),
                                  "ms_per_step": round(ms_plain, 3)},
                      "with_net_tc": {"value": round(world * S_nom / (ms_tc * 1e-3), 1),
                                              "ms_per_step": round(ms_tc, 3)},
                      "kernels_ms_per_step": {k: round(v[0] / steps, 4) for k, v in sorted(kt.items())},
                      "kernels_ms_per_step_tc": {k: round(v[0] / steps, 4) for k, v in sorted(kt_tc.items())}},
            "render_human_512x512": {"with_net_ms": round(r_def, 3), "with_net_tc_ms": round(r_tc, 3),
                                     "without_ms": round(r_plain, 3),
                                     "with_net_tc_mrays_s": round(w.rays.n / (r_tc * 1e-3) / 1e6, 3)}}


def bench_interleave(invr, args, prec_name):
    """1280x720 two-field renders (T=2^21, L=16, up to 192 samples, 4096 nodes, K=8) on one
    stream, alternating with 2^18-ray training steps of the human field on a second stream;
    the renderer reads a parameter snapshot taken after each training step.  Beside it the
    plain path: the same render and step in FP32, one after the other on one stream."""
    import torch
    from paper_2304_03184_b300 import synth
    rw = synth.two_field_render(seed=5, width=1280, height=720, n_samples=192, field_desc=synth.CFG5_FIELD,
                                n_nodes=4096, K=8)
    tw = synth.train_step_workload(seed=5, n_rays=1 << 18, field_desc=synth.CFG5_FIELD, n_nodes=4096, K=8)
    dev = torch.cuda.current_device()
    o, d = torch.from_numpy(rw.rays.o).cuda(), torch.from_numpy(rw.rays.d).cuda()
    n_iter = max(5, args.steps // 2)

    def run(prec, overlap):
        ctx_r, ctx_t = invr.Context(dev), invr.Context(dev)
        views, keep_r = build_views(invr, ctx_r, rw, prec)
        tb, fields, keep_t = build_train(invr, ctx_t, tw, prec)
        trained = list(fields.values())[0]
        snap = views[0].field                       # the renderer's copy of the human field
        ctx_r.reserve(2 * rw.rays.n, 48)
        ctx_t.reserve(sum(b[0].shape[1] for b in tb.batches), 48)
        s_r = torch.cuda.Stream() if overlap else torch.cuda.current_stream()
        s_t = torch.cuda.Stream() if overlap else torch.cuda.current_stream()
        stepped, copied = torch.cuda.Event(), torch.cuda.Event()
        for it in range(n_iter + 2):
            if it == 2:
                torch.cuda.synchronize()
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record(torch.cuda.current_stream())
                s_r.wait_stream(torch.cuda.current_stream())
                s_t.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s_t):
                s_t.wait_event(copied)              # the snapshot of the previous step is taken
                invr.train_step(ctx_t, tb)
                stepped.record(s_t)
            with torch.cuda.stream(s_r):
                s_r.wait_event(stepped)             # snapshot after this step's update
                snap.copy_params_from(trained)
                copied.record(s_r)
                invr.render_rays(ctx_r, o, d, rw.n_samples, rw.t_eps, views)
        torch.cuda.current_stream().wait_stream(s_r)
        torch.cuda.current_stream().wait_stream(s_t)
        t1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        ctx_r.sync()
        ctx_t.sync()
        ms = t0.elapsed_time(t1) / n_iter
        R = sum(b[0].shape[1] for b in tb.batches)
        return {"frames_per_s": round(1e3 / ms, 2), "train_samples_per_s": round(R * tw.n_samples / (ms * 1e-3), 1),
                "ms_per_iteration": round(ms, 3)}

    return {"render_workload": rw.name, "train_workload": tw.name, "iterations": n_iter,
            prec_name + "_two_streams": run(PRECS[prec_name], True), "fp32_one_stream": run(PRECS["fp32"], False)}


def bench_render(invr, ctx, prec, args, flush):
    import torch
    from paper_2304_03184_b300 import synth
    w = synth.two_field_render()
    keep, views = [], []
    for sv in w.views:
        f = invr.Field.from_synth(ctx, sv.field, prec)
        g = None
        if sv.graph is not None:
            gg = sv.graph
            g = invr.Graph(ctx, gg.x_canon.shape[1], gg.K, gg.radius, 1, torch.from_numpy(gg.x_canon).cuda())
            g.set_pose(0, torch.from_numpy(gg.dq).cuda(), torch.from_numpy(gg.x_live).cuda())
        occ = torch.from_numpy(sv.occupancy).cuda()
        keep.append((f, g, occ))
        views.append(invr.View(f, g, 0, sv.rigid_dq, occ))
    o, d = torch.from_numpy(w.rays.o).cuda(), torch.from_numpy(w.rays.d).cuda()
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        for _ in range(max(args.warmup, 3)):
            fn()
        ctx.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.fill_(1)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    ms = timed(lambda: invr.render_rays(ctx, o, d, w.n_samples, w.t_eps, views), args.steps)
    ms_joint = timed(lambda: invr.render_rays(ctx, o, d, w.n_samples, w.t_eps, views, joint=True),
                     max(5, args.steps // 4))
    # occupancy maintenance of the human field (2 M cell queries through warp, encoding, MLPs)
    n = invr.OCC_RES ** 3
    dens = torch.zeros(n, device="cuda")
    bits = torch.empty(n // 32, dtype=torch.int32, device="cuda")
    ms_occ = timed(lambda: invr.occupancy_update(ctx, views[0], dens, bits, 0.95, 0.01), max(5, args.steps // 4))
    return {"value": round(w.rays.n / (ms * 1e-3) / 1e6, 3), "unit": "Mrays/s", "ms_per_frame": round(ms, 3),
            "workload": w.name,
            "joint": {"value": round(w.rays.n / (ms_joint * 1e-3) / 1e6, 3), "unit": "Mrays/s",
                      "ms_per_frame": round(ms_joint, 3)},
            "occupancy_update": {"ms": round(ms_occ, 3), "cells_per_s": round(n / (ms_occ * 1e-3), 1),
                                 "cells": n}}


# ------------------------------------------------------------------ oracle (CPU) arm
def oracle_train_sample(tw, rays_per_batch):
    """The oracle's training step (loss, gradient, Adam on every field) on the first
    rays_per_batch rays of every batch of the workload; returns seconds."""
    from oracle import oracle
    ofields = {id(fp): oracle.Field.from_params(fp) for fp in tw.fields}
    obs = []
    for b in tw.batches:
        n = min(rays_per_batch, b.rays.n)
        v = oracle.View.from_synth(b.view, field=ofields[id(b.view.field)])
        obs.append(oracle.TrainBatch(b.rays.o[:, :n], b.rays.d[:, :n], v, b.target[:, :n]))
    t0 = time.perf_counter()
    _, grads = oracle.train_loss_grad(obs, tw.n_samples, tw.t_eps, tw.huber_delta)
    for f in ofields.values():
        gt, gw = grads[id(f)]
        p = np.concatenate([f.tables, f.weights])
        m, vv = np.zeros_like(p), np.zeros_like(p)
        oracle.adam(p, np.concatenate([gt, gw]), m, vv, 1, tw.lr, tw.beta1, tw.beta2, tw.adam_eps)
    return time.perf_counter() - t0, sum(min(rays_per_batch, b.rays.n) for b in tw.batches)


def cpu_baseline(tw, rays_per_batch=2048):
    from oracle import oracle
    oracle.build()
    dt, n = oracle_train_sample(tw, rays_per_batch)
    return {"value": round(n * tw.n_samples / dt, 1), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"first {rays_per_batch} rays of each of the {len(tw.batches)} batches ({n} rays), "
                      f"one training step (loss + gradient + Adam), {dt:.1f} s"}


def run_reference(args, rank, world):
    from paper_2304_03184_b300 import synth
    tw = synth.keyframe_batch_workload()
    per_batch = 64
    times = []
    for _ in range(args.warmup):
        oracle_train_sample(tw, per_batch)
    n = 0
    for _ in range(args.steps):
        dt, n = oracle_train_sample(tw, per_batch)
        times.append(dt)
    ms = float(np.mean(times)) * 1e3
    value = n * tw.n_samples / (ms * 1e-3)
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(tw, world),
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"each step: the FP64 CPU oracle's training step (loss, gradient, Adam) on "
                                       f"the first {per_batch} rays of each of the {len(tw.batches)} batches "
                                       f"({n} rays x {tw.n_samples} samples)"},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out, tw = run_ours(args, rank, world, local)
    if rank == 0:
        if world == 1 and not args.no_cpu:
            out["cpu_baseline"] = cpu_baseline(tw)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
