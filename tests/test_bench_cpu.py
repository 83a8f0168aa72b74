"""bench.py on the CPU: the reference arm (the oracle) prints a valid JSON
line, and the helpers the GPU arm uses work."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "cavity16", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_bench_helpers():
    import bench
    from paper_1705_08019_gb300 import workloads as W
    w = W.cavity16()
    assert bench.work_of(w) == sum(2000 - j * 500 for j in range(4)) * 16 ** 3
    cfg = bench.config_of(w)
    assert cfg["workload"] == "cavity16" and cfg["K"] == 4
    rate, sec, desc = bench.oracle_sample(W.small_random(dims=(8, 8, 8)))
    assert rate > 0 and sec > 0 and "oracle" in desc
    hbm, kind = bench.peaks()
    assert hbm > 0 and kind in ("measured", "fallback")


def test_field_error_helpers():
    """Relative L2 error per probe trace (columns) and per field component, max."""
    import torch
    import bench
    ref = (torch.ones(10, 3, dtype=torch.float64), torch.ones(3, 2, 2, 2, dtype=torch.float64),
           2 * torch.ones(3, 2, 2, 2, dtype=torch.float64))
    pr = ref[0].clone()
    pr[:, 1] *= 1.001
    h = ref[2].clone()
    h[2] *= 1.0 + 1e-6
    errs = bench.field_errors(pr, ref[1], h, ref)
    assert abs(errs["probes"] - 1e-3) < 1e-12 and errs["e"] == 0.0 and abs(errs["h"] - 1e-6) < 1e-15
    assert errs["max"] == errs["probes"]
    assert bench.traffic_from_profile(64) is None
