"""The boundary's state conversions on the CPU: the library's k_set_cams / k_get_cams (boundary
camera [w, t, f, k1, k2] <-> internal R, t, d in units of s pixels), k_set_lms / k_get_lms (the
landmark records of the FP64 and MIXED paths, through a reversed internal numbering) and
k_check_state (the first invalid camera or landmark), and k_check_degenerate (Assumption 2 on
the current iterate), built for the host with g++ and run one element or chunk at a time. The conversions are checked against the oracle's to_internal and
to_boundary (Sec. 3's camera model with Eq. ray's radial terms scaled by s), the round trips
against the input, and the check indices against the definition. No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import daba_oracle as O
from tests.test_host_device_math import FLAGS, HOST

INT_MAX = 2 ** 31 - 1


@pytest.fixture(scope="module")
def state_io(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("state_io") / "state_io")
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, "state_io.cpp"), "-o", exe], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    return exe


def _call(exe, cams, lms, s):
    M, N = cams.shape[0], lms.shape[0]
    stdin = (f"{M} {N} {float(s)!r}\n" + "\n".join(" ".join(repr(float(x)) for x in r) for r in cams) + "\n"
             + "\n".join(" ".join(repr(float(x)) for x in r) for r in lms) + "\n")
    run = subprocess.run([exe], input=stdin, capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stderr[-2000:]
    lines = run.stdout.splitlines()
    chk = [int(x) for x in lines[0].split()]
    cam = np.array([[float(x) for x in ln.split()] for ln in lines[1:1 + M]])
    lm = np.array([[float(x) for x in ln.split()] for ln in lines[1 + M:1 + M + N]])
    return chk, cam, lm


def _cameras(rng, M):
    """Axis-angle vectors from 1e-12 rad to pi - 1e-3 rad (both ends of Exp and Log), centres,
    focal lengths 500-800 px and radial coefficients of both signs."""
    axis = rng.normal(size=(M, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = np.concatenate([[1e-12, 1e-7, 1e-3, np.pi - 1e-3, np.pi - 0.1], rng.uniform(0.0, np.pi - 1e-3, M - 5)])
    return np.concatenate([axis * ang[:, None], rng.uniform(-20, 20, (M, 3)), rng.uniform(500, 800, (M, 1)),
                           rng.normal(0, 1e-1, (M, 1)), rng.normal(0, 1e-2, (M, 1))], 1)


def test_camera_conversions_match_oracle_and_round_trip(state_io):
    rng = np.random.default_rng(31)
    M, N, s = 300, 50, 650.0
    cams = _cameras(rng, M)
    lms = rng.uniform(-10, 10, (N, 3))
    chk, cam, _ = _call(state_io, cams, lms, s)
    assert chk == [INT_MAX, INT_MAX, INT_MAX]
    R, t, d, _ = O.to_internal(cams, lms, s)
    np.testing.assert_allclose(cam[:, 0:9], R.reshape(M, 9), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(cam[:, 9:12], t)
    np.testing.assert_allclose(cam[:, 12:15], d, rtol=1e-15, atol=0)
    back = cam[:, 15:24]
    # Log(Exp(w)) = w for |w| < pi; near pi the axis is recovered from R + R^T, whose
    # sensitivity grows as 1 / (pi - |w|)
    ang = np.linalg.norm(cams[:, 0:3], axis=1)
    tol = 1e-13 / np.maximum(np.pi - ang, 1e-3) + 1e-15
    assert (np.abs(back[:, 0:3] - cams[:, 0:3]).max(axis=1) <= tol).all()
    np.testing.assert_array_equal(back[:, 3:6], cams[:, 3:6])
    np.testing.assert_allclose(back[:, 6:9], cams[:, 6:9], rtol=1e-14, atol=0)
    ob, _ = O.to_boundary(cam[:, 0:9].reshape(M, 3, 3), cam[:, 9:12], cam[:, 12:15], lms, s)
    assert (np.abs(back[:, 0:3] - ob[:, 0:3]).max(axis=1) <= tol).all()
    np.testing.assert_allclose(back[:, 6:9], ob[:, 6:9], rtol=1e-14, atol=0)


def test_landmark_records_round_trip(state_io):
    """FP64 records give the coordinates back exactly; MIXED high + low parts within 2^-48 of
    each coordinate (the FP32 low part of l - hi), through a reversed internal numbering."""
    rng = np.random.default_rng(5)
    lms = rng.uniform(-1, 1, (400, 3)) * 10.0 ** rng.uniform(-6, 4, (400, 1))
    _, _, lm = _call(state_io, _cameras(rng, 10), lms, 700.0)
    np.testing.assert_array_equal(lm[:, 0:3], lms)
    assert (np.abs(lm[:, 3:6] - lms) <= 2.0 ** -48 * np.abs(lms)).all()


def test_state_check_reports_the_first_invalid_entries(state_io):
    """k_check_state: the lowest camera index with a non-finite parameter, the lowest landmark
    index with a non-finite coordinate and the lowest finite camera with f <= 0, each
    independent of the others."""
    rng = np.random.default_rng(9)
    cams = _cameras(rng, 40)
    lms = rng.uniform(-5, 5, (60, 3))
    cams[17, 4] = np.nan
    cams[23, 0] = np.inf
    cams[9, 6] = 0.0
    cams[31, 6] = -5.0
    cams[5, 6] = np.nan        # non-finite, so not counted as a bad focal length
    lms[44, 2] = -np.inf
    lms[12, 0] = np.nan
    chk, _, _ = _call(state_io, cams, lms, 650.0)
    assert chk == [5, 12, 9]


def _degenerate(exe, t, l, cam, lm):
    order = np.argsort(cam, kind="stable")
    cam, lm = cam[order], lm[order]
    stdin = (f"{t.shape[0]} {l.shape[0]} {cam.size}\n" + "\n".join(" ".join(repr(float(x)) for x in r) for r in t)
             + "\n" + "\n".join(" ".join(repr(float(x)) for x in r) for r in l) + "\n"
             + "\n".join(f"{i} {j}" for i, j in zip(cam, lm)) + "\n")
    run = subprocess.run([exe], input=stdin, capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stderr[-2000:]
    return [int(x) for x in run.stdout.split()], cam, lm


@pytest.fixture(scope="module")
def degenerate(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("degenerate") / "degenerate")
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, "degenerate.cpp"), "-o", exe], capture_output=True,
                           text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    return exe


@pytest.mark.parametrize("centre_scale", [1.0, 1e3])
def test_assumption2_check_finds_the_first_degenerate_pair(degenerate, centre_scale):
    """Assumption 2 (a landmark away from the centre of every camera observing it), as daba_run
    checks it: an observation fails when |l - t|^2 <= 1e-24 max(1, |t|^2). Landmarks placed on a
    camera centre, 1e-13 max(1, |t|) from it (fails) and 1e-11 max(1, |t|) from it (passes): both
    paths report the smallest failing position in camera order, and nothing on a clean scene."""
    rng = np.random.default_rng(int(centre_scale))
    M, N, nnz = 20, 300, 2000
    t = rng.uniform(-1, 1, (M, 3)) * centre_scale
    l = rng.uniform(-1, 1, (N, 3)) * centre_scale + 5.0
    cam = rng.integers(0, M, nnz)
    lm = rng.integers(0, N, nnz)
    none = 2 ** 64 - 1
    got, _, _ = _degenerate(degenerate, t, l, cam, lm)
    assert got == [none, none]
    order = np.argsort(cam, kind="stable")
    unit = max(1.0, centre_scale)

    def put(pos, dist):   # landmark of the observation at camera-sorted position pos near its camera
        o = order[pos]
        d = rng.normal(size=3)
        l[lm[o]] = t[cam[o]] + dist * unit * d / np.linalg.norm(d)

    put(1500, 1e-11)           # passes
    got, _, _ = _degenerate(degenerate, t, l, cam, lm)
    assert got == [none, none]
    put(1200, 1e-13)           # fails
    put(700, 0.0)              # fails, and comes first
    got, _, lms = _degenerate(degenerate, t, l, cam, lm)
    sorted_cam = cam[order]
    q = l[lm[order]] - t[sorted_cam]
    thr = 1e-24 * np.maximum(1.0, np.sum(t[sorted_cam] ** 2, axis=1))
    first = int(np.flatnonzero(np.sum(q * q, axis=1) <= thr)[0])
    assert first <= 700
    assert got == [first, first]
