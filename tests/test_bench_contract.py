"""The JSON line bench.py prints: the reference arm (the FP64 oracle on the host
cores, CPU) and a short GPU run, checked for every key the line promises."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=600):
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=timeout)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, res.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Msamples/s"
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("gsb-")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_traffic_capture_key_ignores_comments_only(tmp_path):
    """The committed DRAM-traffic capture is keyed by a hash of the fused
    kernel's code: comments and blank lines leave the key alone, a code change
    moves it (and the bench line's traffic then reads null)."""
    sys.path.insert(0, ROOT)
    import bench
    for f in bench.KERNEL_SOURCES:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            dst.write_text(fh.read(), encoding="utf-8")
    key = bench.kernel_source_hash(str(tmp_path))
    assert key == bench.kernel_source_hash(ROOT)
    first = tmp_path / bench.KERNEL_SOURCES[0]
    first.write_text(first.read_text(encoding="utf-8") + "\n// a note\n/* a block\n   note */\n\n",
                     encoding="utf-8")
    assert bench.kernel_source_hash(str(tmp_path)) == key
    first.write_text(first.read_text(encoding="utf-8") + "static int cdd_probe_value = 1;\n",
                     encoding="utf-8")
    assert bench.kernel_source_hash(str(tmp_path)) != key


@pytest.mark.gpu
@pytest.mark.slow
def test_gpu_line(cuda_device):
    d = run_bench("--steps", "5", "--warmup", "3", "--e2e-steps", "3", "--no-cpu-baseline")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in d, key
    assert d["value"] > 0 and d["steps"] == 5 and d["warmup"] >= 3 and d["scaling"] == "weak"
    assert d["config"]["workload"] == "gsb-32MHz@325MHz-512ch-DM50-N8192-x16"
    r = d["roofline"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and 0 < r["frac"] < 1.5
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert "traffic" in r
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == 617728 * 512 * 2
    assert e["d2h_bytes_per_step"] == 512 * 38608 * 4
    assert d["gpu_launches"] == 2 * 5
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
