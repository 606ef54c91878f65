"""The JSON line of bench.py's reference arm (the oracle timed on the host cores), run as a
subprocess on a small workload, and the GPU arm refusing to run without a GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args):
    return subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True,
                          timeout=900)


@pytest.mark.parametrize("workload, extra", [("circle", ()), ("batch", ("--n-scenes", "3"))])
def test_reference_arm_line(workload, extra):
    import bench
    r = _bench("--impl", "reference", "--workload", workload, "--steps", "2", "--warmup", "0", *extra)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    cb, e2e = line["cpu_baseline"], line["e2e"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    assert cb["host"]["nproc"] >= 1 and cb["host"]["cpu_model"]
    assert e2e == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cfg = line["config"]
    assert {"workload", "M", "N", "nnz", "prec", "parallelism"} <= set(cfg)
    if workload == "circle":
        assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
        assert line["ms_per_step"] == pytest.approx(1e3 * cfg["nnz"] / line["value"], rel=1e-9)
    else:
        assert line["unit"] == "scenes/s" and cfg["workload"].startswith("batch: 3 circle scenes")


def test_gpu_arm_fails_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _bench("--workload", "circle", "--steps", "1", "--warmup", "3")
    assert r.returncode != 0
    assert not r.stdout.strip() or '"value"' not in r.stdout
