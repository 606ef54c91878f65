"""The JSON line of bench.py's reference arm (the oracle timed on the host cores), run as a
subprocess on a small workload, and the GPU arm refusing to run without a GPU."""
import json
import os
import subprocess
import sys

import numpy as np
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
    assert {"workload", "M", "N", "nnz", "parallelism", "l2"} <= set(cfg)
    if workload == "circle":
        assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
        # the step is one oracle iteration over the sample: its measured time, and beside it the
        # whole workload's step at the same rate, labelled as extrapolated
        assert line["ms_per_step_whole_workload_extrapolated"] == pytest.approx(1e3 * cfg["nnz"] / line["value"],
                                                                               rel=1e-9)
        assert line["ms_per_step"] * line["steps"] < 1e3 * 120
        assert cfg == bench.tourism_config(_circle(), 1)
    else:
        assert line["unit"] == "scenes/s" and cfg["workload"].startswith("batch: 3 circle scenes")


def _circle():
    from paper_2305_07026_b300 import scenes
    return scenes.make_scene("circle")


def test_oracle_on_all_cores():
    """The all-cores leg: spawned processes, each on a disjoint camera block of the workload."""
    import bench
    sc = _circle()
    blocks = bench.camera_blocks(sc, 3, sc.nnz // 4)
    seen = np.concatenate(blocks)
    assert len(seen) == len(np.unique(seen)) and len(blocks) == 3
    out = bench.cpu_oracle_all_cores(sc, 0.02, 2, n_steps=1)
    assert out["kind"] == "oracle" and out["cores"] == 2 and out["value"] > 0 and out["sample"]


def test_gpu_arm_fails_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _bench("--workload", "circle", "--steps", "1", "--warmup", "3")
    assert r.returncode != 0
    assert not r.stdout.strip() or '"value"' not in r.stdout
