"""Parity of the objective-only evaluations on the CPU: eval_F4 (the camera-pack form that
daba_objective's kernel uses, FP64 and FP32 with FP32 high and low parts of the landmark and the
camera centre) and eval_F (the flat-pack form of the allocation-free objective, FP64), built for
the host with g++, against the oracle's Eq. Fij per loss on seeded observations with |e|^2 on
both sides of the loss scale, including a city-scale offset of the whole scene. No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import daba_oracle as O
from tests.test_host_device_math import FLAGS, HOST
from tests.test_host_blocks_parity import _inputs

LOSSES = {"trivial": 0, "huber": 1, "cauchy": 2, "welsch": 3}


@pytest.fixture(scope="module")
def objective(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("objective") / "objective")
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, "objective.cpp"), "-o", exe], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    return exe


@pytest.mark.parametrize("offset", [0.0, 3000.0])
@pytest.mark.parametrize("loss", list(LOSSES))
def test_objective_forms_match_oracle(objective, loss, offset):
    """FP64 forms within 1e-14 of |p|^2, the scale of rho's argument (measured 4e-17); the FP32
    form within 1e-6 |p| |e| (measured 1.05e-7: FP32 rounding of the ray-length vectors whose
    difference is e), the same with the whole scene 3 km from the origin, because q is formed
    from the high and low parts of the landmark and the camera centre."""
    c = 0.02
    R, t, d, l, u = _inputs(41 + LOSSES[loss], 400, c)
    t = t + offset
    l = l + offset
    rows = np.concatenate([R.reshape(-1, 9), t, d, l, u], 1)
    stdin = f"{LOSSES[loss]} {c!r} {len(rows)}\n" + "\n".join(" ".join(repr(float(x)) for x in r) for r in rows) + "\n"
    run = subprocess.run([objective], input=stdin, capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stderr[-2000:]
    out = np.array([[float(x) for x in line.split()] for line in run.stdout.splitlines()])
    F = O.F_obs(loss, c, R, t, d, l, u)
    p = np.linalg.norm(O.ray(u, d), axis=1)
    e = np.linalg.norm(O.reproj_error(R, t, l, O.ray(u, d)), axis=1)
    np.testing.assert_allclose(out[:, 0], F, rtol=0, atol=1e-14 * (p ** 2).max())
    np.testing.assert_allclose(out[:, 2], F, rtol=0, atol=1e-14 * (p ** 2).max())
    assert (np.abs(out[:, 1] - F) <= 1e-6 * p * e).all(), (np.abs(out[:, 1] - F) / (p * e)).max()
