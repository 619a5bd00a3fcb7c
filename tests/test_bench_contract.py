"""The bench's reference arm (the FP64 oracle on the host) runs without a GPU: its one JSON
line carries the contract's keys, and the replica aggregation is the documented formula."""
import dataclasses
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_replica_aggregation_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.aggregate_replicas(2.0, 1000.0, 1)
    assert ms == 2.0 and abs(value - 1000.0 / 2e-3) < 1e-6


def test_kernel_rooflines_arithmetic():
    """The per-kernel roofline fractions: bytes (or FLOPs) of the stated algorithmic work over
    the CUDA-event duration of one record, against the measured peak the bound names; the
    gather and the scatter against the L2 probe ceilings when those were measured."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2304_03184_b300 import synth
    tw = synth.keyframe_batch_workload(n_frames=1, log2_rays=(9.0, 9.5))
    S, L = 1_000_000, tw.fields[0].desc.L
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1000.0}
    kt = {"adam": (0.2, 2), "mlp_fwd_tc": (1.0, 1), "encode": (2.0, 1), "encode_bwd": (4.0, 1)}
    r = bench.kernel_rooflines(kt, tw, 1000, S, peaks)
    n_params = tw.fields[0].desc.n_table_params() + tw.fields[0].desc.n_weight_params()
    assert abs(r["adam"]["achieved"] - n_params * 32 / 1e-4 / 1e9) < 0.1       # one launch: 0.1 ms
    assert abs(r["mlp_fwd_tc"]["achieved"] - S * 2 * tw.fields[0].desc.n_weight_params() / 1e-3 / 1e12) < 0.1
    assert r["encode"]["bound"] == "hbm" and abs(r["encode"]["frac"] - r["encode"]["achieved"] / 6000.0) < 1e-3
    l2 = {"gather_v4_gbs": 4000.0, "atomic_v4_gbs": 3000.0}
    r2 = bench.kernel_rooflines(kt, tw, 1000, S, peaks, l2)
    payload = S * L * 64                                                       # 8 corners x 2 floats per level
    assert r2["encode"]["bound"] == "l2" and abs(r2["encode"]["achieved"] - payload / 2e-3 / 1e9) < 0.1
    assert abs(r2["encode_bwd"]["achieved"] - payload / 4e-3 / 1e9) < 0.1
    assert abs(r2["encode_bwd"]["frac"] - r2["encode_bwd"]["achieved"] / 3000.0) < 1e-3


def test_headline_roofline_object():
    """The bench line's roofline: the kernel with the most time is the gradient scatter, whose
    tables stay in L2, so its bound is the L2 -- the table payload (8 corners x 2 floats per
    level and sample) per record over the record's duration, against the random float4
    atomic ceiling the probe measured in the same run; its HBM fraction (per-sample inputs)
    rides along, and DRAM traffic (an ncu-only counter) is null."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2304_03184_b300 import synth
    tw = synth.keyframe_batch_workload(n_frames=1, log2_rays=(9.0, 9.5))
    S, L = 2_000_000, tw.fields[0].desc.L
    kt = {"encode_bwd": (10.0, 2), "encode": (4.0, 2), "adam": (0.2, 2)}
    r = bench.roofline(kt, tw, 1000, S, {"hbm_gbs": 6000.0},
                       {"gather_v4_gbs": 4000.0, "atomic_v4_gbs": 3000.0})
    assert r["kernel"] == "encode_bwd" and r["bound"] == "l2" and r["peak"] == 3000.0
    want = S * L * 64 / 5e-3 / 1e9                                             # 5 ms per record
    assert abs(r["achieved"] - want) < 0.1 and abs(r["frac"] - want / 3000.0) < 1e-4
    assert r["traffic"] is None and r["l2_traffic"] is None and r["l2_traffic_gbs"] is None
    hbm = S * (12 + L * (8 + 64)) / 5e-3 / 1e9
    assert abs(r["hbm"]["achieved"] - hbm) < 0.1 and abs(r["hbm"]["frac"] - hbm / 6000.0) < 1e-4
    # without a probe measurement the scatter falls back to its HBM view
    r0 = bench.roofline(kt, tw, 1000, S, {"hbm_gbs": 6000.0})
    assert r0["bound"] == "hbm" and r0["traffic"] is None


def test_scatter_traffic_only_for_the_captured_sources():
    """The captured DRAM and L2 bytes of the scatter ride in the bench line only for the
    workload they were captured on and while the kernel's sources match the capture's digest;
    the roofline's L2 rate is those bytes over the record's duration."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2304_03184_b300 import synth
    name = bench.SCATTER_DRAM["workload"]
    assert bench.scatter_traffic("another_workload") is None
    dram, l2 = bench.scatter_traffic(name), bench.scatter_traffic(name, "l2_bytes")
    if bench.sources_sha16(bench.SCATTER_SOURCES) != bench.SCATTER_DRAM["sources_sha16"]:
        assert dram is None and l2 is None
        return
    assert dram == bench.SCATTER_DRAM["bytes"] and l2 == bench.SCATTER_DRAM["l2_bytes"] and l2 > dram
    tw = dataclasses.replace(synth.keyframe_batch_workload(n_frames=1, log2_rays=(9.0, 9.5)), name=name)
    kt = {"encode_bwd": (10.0, 2)}
    r = bench.roofline(kt, tw, 1000, 2_000_000, {"hbm_gbs": 6000.0}, {"gather_v4_gbs": 4000.0, "atomic_v4_gbs": 3000.0})
    assert r["traffic"] == dram and r["l2_traffic"] == l2
    assert abs(r["l2_traffic_gbs"] - l2 / 5e-3 / 1e9) < 0.1

