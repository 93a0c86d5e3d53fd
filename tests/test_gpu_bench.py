"""bench.py on the GPU, short: the default JSON line carries every key of the contract, and one
single-kernel case runs (catches a broken benchmark before a long run does)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bench_line_contract():
    line = _run("--steps", "3", "--warmup", "3", "--no-cpu", "--no-compare", "--no-e2e")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "gpu_launches", "clocks", "roofline"):
        assert key in line, key
    assert line["value"] > 0 and line["gpu_launches"] == 36
    roof = line["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in roof, key
    assert 0 < roof["frac"] < 1.5


def test_bench_case_runs():
    line = _run("--case", "edm:LTM:chunked:4096:3:16", "--steps", "3", "--warmup", "3")
    assert line["ms_median"] > 0
