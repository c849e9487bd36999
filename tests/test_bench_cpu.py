"""bench.py's reference arm on CPU: the JSON line contract (keys, units, the oracle as the timed
program) for the gradient and batched-scan workloads, whose bounded samples finish in seconds;
and the measured-peaks reader's fallback."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload,unit", [("adjoint", "grads/s"), ("batch", "instances/s")])
def test_reference_line_contract(workload, unit):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        workload, "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == unit and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert abs(d["ms_per_step"] - 1000.0 / d["value"]) <= 1e-9 * d["ms_per_step"]


def test_measured_peaks_reader(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    p = bench.measured_peaks()
    assert p["source"] in ("measured", "fallback")
    assert p["bf16_sustained"] <= p["bf16"]
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))  # no peaks file there
    q = bench.measured_peaks()
    assert q == {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}
