"""bench.py's JSON line on a GPU, on the small ring workload: one line on stdout with every
key the benchmark contract names, of the right type and sign (the headline run uses the
same code on the 256-element ring)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_contract():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = subprocess.run([sys.executable, "bench.py", "--workload", "ring32", "--steps", "3", "--warmup", "3",
                        "--cpu-rows", "64"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    r = json.loads(lines[0])
    for k in ("metric", "unit", "dtype", "data", "scaling"):
        assert isinstance(r[k], str) and r[k]
    assert r["value"] > 0 and r["ms_per_step"] > 0
    assert r["n_gpus"] == 1 and r["steps"] == 3 and r["warmup"] == 3
    assert r["higher_is_better"] is True and r["vs_baseline"] is None
    assert r["config"]["workload"] == "ring32"
    rf = r["roofline"]
    assert rf["bound"] in ("alu", "hbm", "tensor") and rf["peak"] > 0 and rf["achieved"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1 and cb["sample"]
    e2e = r["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert r["gpu_launches"] > 0
    ck = r["clocks"]
    assert "sm_mhz" in ck and "sm_max_mhz" in ck and isinstance(ck["reasons"], list)
    err = r["err_vs_fp64_oracle"]
    assert err["J_rel_l2"] <= 1e-5 and err["JT_rel_l2"] <= 1e-5
