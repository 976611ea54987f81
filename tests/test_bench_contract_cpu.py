"""bench.py's reference arm (the FP64 oracle timed on the host cores) prints
one JSON line with the keys the benchmark contract names; run on a small
workload here, no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "vol64",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert "64x64x64" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_byte_model_and_rates():
    """The roofline's algorithmic bytes per voxel-iteration (each array of the
    fused step read or written once) and the whole-job rate."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.bytes_per_voxel("f32", "delta") == 32  # x, d, b, w, om1, omtv read; x, d written
    assert bench.bytes_per_voxel("f32", "prev") == 28   # x_k, x_{k-1}, b, w, om1, omtv read; x written
    assert bench.bytes_per_voxel("bf16", "delta") == 28
    assert bench.bytes_per_voxel("bf16", "prev") == 24
    # the method's own bytes (x_k, x_{k-1}, b, w, om1, omtv read once, x_{k+1}
    # written once): what the roofline fraction counts, whatever the storage
    assert bench.method_bytes_per_voxel("f32") == 28
    assert bench.method_bytes_per_voxel("bf16") == 24
    # 2 ranks x 1e9 voxel-iterations in 500 ms of the slowest rank: 4 Gvoxel-iter/s for the job
    assert abs(bench.whole_job_rate(1e8, 10, 2, 500.0) - 4.0) < 1e-12
    assert bench.max_over_ranks(12.5, 1) == 12.5


def test_roofline_counts_the_method_bytes():
    """frac = method bytes / launch time / peak; the increment write of the
    increment storage form is reported beside it, not inside it."""
    sys.path.insert(0, ROOT)
    import bench
    nvox = 512 ** 3
    r = bench.roofline_block("f32", "delta", nvox, 0.6508e-3, 6689.5, "measured", traffic=4.313e9)
    assert r["algorithmic_bytes_per_launch"] == 28 * nvox
    assert r["storage_overhead_bytes_per_launch"] == 4 * nvox
    assert r["moved_bytes_per_launch"] == 32 * nvox
    assert abs(r["achieved"] - 28 * nvox / 0.6508e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6689.5) < 1e-12
    assert abs(r["frac"] - 0.863) < 0.001          # 206.2 Gvoxel-iter/s on 28 B
    assert abs(r["moved_frac"] - 0.986) < 0.001    # the same launch on the 32 B it moves
    assert abs(r["traffic_over_algorithmic"] - 4.313e9 / (28 * nvox)) < 1e-12
    assert abs(r["frac_nominal"] - r["achieved"] / bench.NOMINAL_HBM_GBS) < 1e-12
    r = bench.roofline_block("bf16", "prev", nvox, 1e-3, 6791.0, "measured")
    assert r["algorithmic_bytes_per_launch"] == r["moved_bytes_per_launch"] == 24 * nvox
    assert r["storage_overhead_bytes_per_launch"] == 0 and r["traffic"] is None


def test_secondary_byte_models():
    """Bytes per voxel behind the adjoint and Fourier-domain lines."""
    sys.path.insert(0, ROOT)
    import bench
    # 50 iterations, checkpoints every 10: 50 adjoint steps of 84 B, a sweep of
    # 50 fused steps and 5 segments recomputed up to their last step (45), 28 B each
    assert bench.adjoint_bytes_per_voxel(50, 10) == 84 * 50 + 28 * (50 + 45)
    assert bench.adjoint_bytes_per_voxel(1, 10) == 84 + 28
    assert bench.adjoint_bytes_per_voxel(12, 5) == 84 * 12 + 28 * (12 + 9)
    assert bench.fourier_bytes_per_voxel() == 62
