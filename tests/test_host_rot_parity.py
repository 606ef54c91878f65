"""Parity of the library's ProjRot3D variants (Eq. proj_rot3d) on the CPU: Horn's quaternion
method with Jacobi rotations (FP64 and FP32), the scaled Newton polar factor, the warm-started
Newton on the rotation and the Newton-Schulz iteration for matrices near a rotation (FP64 and
FP32), built for the host with g++, against the oracle's SVD projection U diag(1, 1, det UV^T) V^T.
Inputs: general matrices (either sign of det), extrapolations R + gamma dR near a rotation, and
reflection-like matrices (det < 0). Errors are scaled by the conditioning of the projection,
min over pairs of (signed) singular values s_i + s_j, over s_1. No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import daba_oracle as O
from tests.test_host_device_math import FLAGS, HOST


@pytest.fixture(scope="module")
def projections(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("rot_proj") / "rot_proj")
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, "rot_proj.cpp"), "-o", exe], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    rng = np.random.default_rng(5)
    n = 600
    kind = np.arange(n) % 3
    Rt = O.so3_exp(rng.uniform(-2, 2, (n, 3)))
    K = np.empty((n, 3, 3))
    for i in range(n):
        if kind[i] == 0:
            K[i] = rng.standard_normal((3, 3))
        elif kind[i] == 1:
            K[i] = Rt[i] + 0.9 * (Rt[i] - O.so3_exp(rng.uniform(-0.05, 0.05, (1, 3)))[0] @ Rt[i])
        else:
            K[i] = Rt[i] @ np.diag([1.0, 0.8, -0.3 - 0.5 * rng.uniform()])
    ora = O.proj_rot3d(K)
    Q0 = np.einsum("nab,nbc->nac", ora, O.so3_exp(rng.uniform(-0.1, 0.1, (n, 3))))   # warm starts near the answer
    stdin = f"{n}\n" + "\n".join(" ".join(repr(float(x)) for x in np.concatenate([K[i].ravel(), Q0[i].ravel()]))
                                 for i in range(n)) + "\n"
    run = subprocess.run([exe], input=stdin, capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stderr[-2000:]
    dev = np.array([[float(x) for x in line.split()] for line in run.stdout.splitlines()])
    assert dev.shape == (n, 55)
    sv = np.linalg.svd(K, compute_uv=False)
    s3 = sv[:, 2] * np.sign(np.linalg.det(K))
    cond = np.minimum(sv[:, 0] + sv[:, 1], np.minimum(sv[:, 0] + s3, sv[:, 1] + s3)) / sv[:, 0]
    return dev, ora.reshape(n, 9), cond, np.linalg.det(K)


# (name, first column, bound on the error times the conditioning): FP64 to rounding, FP32 to a few
# tens of ulp (the host build shows 1e-14 and 3.5e-6)
VARIANTS = [("jacobi64", 0, 1e-12), ("jacobi32", 9, 3e-5), ("polar64", 18, 1e-12), ("near64", 37, 1e-12),
            ("near32", 46, 3e-5)]


@pytest.mark.parametrize("name, col, bound", VARIANTS)
def test_projection_matches_oracle(projections, name, col, bound):
    dev, ora, cond, _ = projections
    err = np.abs(dev[:, col:col + 9] - ora).max(1) * cond
    assert err.max() <= bound, f"{name}: {err.max():.2e}"


def test_warm_started_projection(projections):
    """proj_rot3d_from declines (leaving the caller to the polar factor) unless det K > 0, and
    where it accepts it is the projection to rounding."""
    dev, ora, cond, det = projections
    ok = dev[:, 27] == 1
    assert not np.any(ok & (det <= 0))
    assert ok[det > 0].mean() > 0.9
    assert (np.abs(dev[ok, 28:37] - ora[ok]).max(1) * cond[ok]).max() <= 1e-12
