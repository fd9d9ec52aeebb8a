"""The benchmark's reference arm (the FP64 oracle on the host cores) prints
one JSON line with the contract's keys, the same workload and metric as the
GPU arm, and zero host-device bytes; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 0
    assert d["unit"] == "MLUPS" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] and d["config"]["lattice"] == [256, 256, 512]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_stated_error_matches_the_precision_test():
    """The bench line's stated accuracy per storage is the bound the GPU
    precision test asserts on the precision tank's 128^3 sub-run."""
    import ast
    sys.path.insert(0, ROOT)
    import bench
    src = open(os.path.join(ROOT, "tests", "test_gpu_precision.py")).read()
    node = next(n for n in ast.parse(src).body
                if isinstance(n, ast.Assign) and getattr(n.targets[0], "id", "") == "BOUNDS_C4")
    bounds = ast.literal_eval(node.value)
    for st, (bu, bf) in bounds.items():
        assert bench.STATED_ERROR_C4[st]["velocity_rel_l2_max"] == bu
        assert bench.STATED_ERROR_C4[st]["force_rel_max"] == bf
