"""Parity of the camera half of one iteration on the CPU: the library's camera-pass statistics
(eval_obs + accumulate_cam, FP64) and its camera solve group (camsolve_group: Eqs. DEalpha, Fak
and lFak in slack form, the accelerated S-CAM solve of Eq. update_amm, the restart test of
Eq. Eak and the MM solve of Eq. update_mm), built for the host with g++ and fed each camera's
state and observations, against one oracle step of Algorithm 1 per camera block. The
extrapolated rotation is the oracle's (the library forms it in the previous iteration's solve,
which the ProjRot3D tests cover). No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import daba_oracle as O
from tests.conftest import cached_scene
from tests.test_host_device_math import FLAGS, HOST

LOSSES = {"trivial": 0, "huber": 1, "cauchy": 2, "welsch": 3}


@pytest.fixture(scope="module")
def cam_pass(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("cam_pass") / "cam_pass")
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, "cam_pass.cpp"), "-o", exe], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    return exe


def _run(exe, scene, opts, k, bits=64, glob=0):
    lm = int(opts.cam_solver == "lm")
    prob, R, t, d, l = O.make_problem(scene.cams, scene.lms, scene.cam_idx, scene.lm_idx, scene.uv, opts)
    st = O.init_state(prob, R, t, d, l)
    for _ in range(k):
        st, _ = O.step(prob, st)
    s_next, gamma = O.nesterov(st.s)
    _, gamma_next = O.nesterov(s_next)
    Rb = O.proj_rot3d(st.R + gamma * (st.R - st.Rp))
    new, info = O.step(prob, st)
    ci, li, u, M = prob.cam_idx, prob.lm_idx, prob.u, prob.M
    order = np.argsort(ci, kind="stable")
    ptr = np.concatenate([[0], np.cumsum(np.bincount(ci, minlength=M))])
    first = k == 0
    S = np.zeros(M) if first else st.Fbar_cam - st.E_cam
    head = (f"{bits} {glob} {lm} {LOSSES[prob.loss]} {float(prob.c)!r} {float(opts.xi)!r} {float(opts.eta)!r} {opts.cam_alternations} "
            f"{int(opts.accelerated)} {int(first)} {float(gamma)!r} {float(gamma_next)!r} {M}")
    lines = [head]
    for i in range(M):
        obs = order[ptr[i]:ptr[i + 1]]
        cam = [*st.R[i].ravel(), *st.t[i], *st.d[i], *st.Rp[i].ravel(), *st.tp[i], *st.dp[i], *Rb[i].ravel(),
               S[i], st.E_cam[i]]
        lines.append(f"{len(obs)} " + " ".join(repr(float(x)) for x in cam))
        rows = np.concatenate([st.l[li[obs]], st.lp[li[obs]], u[obs]], 1)
        lines.extend(" ".join(repr(float(x)) for x in r) for r in rows)
    run = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stderr[-2000:]
    out = np.array([[float(x) for x in line.split()] for line in run.stdout.splitlines()])
    assert out.shape == (M, 39 if glob else 21)
    Fij = O.F_obs(prob.loss, prob.c, st.R[ci], st.t[ci], st.d[ci], st.l[li], u)
    return st, new, info, out, O.segsum(ci, Fij, M)


@pytest.mark.parametrize("loss,xi,k", [("huber", 1e-10, 0), ("huber", 1e-10, 12), ("cauchy", 0.5, 6),
                                       ("huber", 0.5, 16)])
def test_camera_half_matches_oracle_iteration(cam_pass, loss, xi, k):
    """Per camera of the 20-camera circle scene: x^(k+1), F^(k), Fbar^(k), E^(k+1), the next
    slack, the F_ij sum and the restart decision against the oracle's step, at the first
    iteration (slack 0, E^(0) from the F sums) and at later ones where 6-8 of the 20 camera
    blocks restart (slack and E^(k) carried in the camera state)."""
    sc = cached_scene("circle")
    opts = O.Options(loss=loss, loss_scale_px=sc.loss_scale_px, xi=xi)
    st, new, info, out, Fsum = _run(cam_pass, sc, opts, k)
    x = out[:, :15]
    F, Fbar, E_next, S_next, rs, Fs = out[:, 15], out[:, 16], out[:, 17], out[:, 18], out[:, 19] > 0.5, out[:, 20]
    scale = np.abs(info.Fbar_cam).max()
    np.testing.assert_allclose(Fs, Fsum, rtol=1e-12)
    np.testing.assert_allclose(F, info.F_cam, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(Fbar, info.Fbar_cam, rtol=0, atol=1e-11 * scale)
    margin = np.abs(info.Etest_cam - info.Fbar_cam)
    clear = margin > 1e-8 * scale
    assert clear.mean() > 0.8
    np.testing.assert_array_equal(rs[clear], info.restart_cam[clear])
    if k > 0:   # both branches: cameras that restart (MM solve) and cameras that keep the accelerated one
        assert info.restart_cam.sum() >= 5 and (~info.restart_cam).any()
    same = rs == info.restart_cam
    want = np.concatenate([new.R.reshape(-1, 9), new.t, new.d], 1)
    np.testing.assert_allclose(x[same], want[same], rtol=0, atol=1e-9)
    np.testing.assert_allclose(E_next[same], new.E_cam[same], rtol=0, atol=1e-10 * scale)
    np.testing.assert_allclose(S_next[same], (new.Fbar_cam - new.E_cam)[same], rtol=0, atol=1e-10 * scale)


@pytest.mark.parametrize("loss,xi,k", [("huber", 1e-10, 0), ("huber", 1e-10, 12), ("cauchy", 0.5, 6),
                                       ("huber", 0.5, 16)])
def test_mixed_camera_half_within_fp32_bounds(cam_pass, loss, xi, k):
    """The MIXED instantiation (statistics evaluated and accumulated in FP32, the FP32 S-CAM
    solve on displacements added to the FP64 camera state, FP64 restart metrics) against the
    same oracle step. Bounds from the FP32 arithmetic, with the measured worst in brackets:
    camera parameters within 2e-5 (7e-6, the FP32 solve), F^(k) and Fbar^(k) within 5e-6 of the
    largest Fbar (8e-7, FP32 per-observation terms), E^(k+1) and the next slack within 1e-5
    (2e-6), the F_ij sums within 5e-6 relative (1e-6), restart decisions equal where the
    oracle's margin exceeds 1e-4 of the largest Fbar."""
    sc = cached_scene("circle")
    opts = O.Options(loss=loss, loss_scale_px=sc.loss_scale_px, xi=xi)
    st, new, info, out, Fsum = _run(cam_pass, sc, opts, k, bits=32)
    x = out[:, :15]
    F, Fbar, E_next, S_next, rs, Fs = out[:, 15], out[:, 16], out[:, 17], out[:, 18], out[:, 19] > 0.5, out[:, 20]
    scale = np.abs(info.Fbar_cam).max()
    np.testing.assert_allclose(Fs, Fsum, rtol=5e-6)
    np.testing.assert_allclose(F, info.F_cam, rtol=0, atol=5e-6 * scale)
    np.testing.assert_allclose(Fbar, info.Fbar_cam, rtol=0, atol=5e-6 * scale)
    clear = np.abs(info.Etest_cam - info.Fbar_cam) > 1e-4 * scale
    assert clear.mean() > 0.8
    np.testing.assert_array_equal(rs[clear], info.restart_cam[clear])
    same = rs == info.restart_cam
    want = np.concatenate([new.R.reshape(-1, 9), new.t, new.d], 1)
    np.testing.assert_allclose(x[same], want[same], rtol=0, atol=2e-5)
    np.testing.assert_allclose(E_next[same], new.E_cam[same], rtol=0, atol=1e-5 * scale)
    np.testing.assert_allclose(S_next[same], (new.Fbar_cam - new.E_cam)[same], rtol=0, atol=1e-5 * scale)


@pytest.mark.parametrize("loss,xi,k", [("huber", 1e-10, 0), ("huber", 1e-10, 12), ("cauchy", 0.5, 6),
                                       ("huber", 0.5, 13)])
def test_lm_camera_solver_matches_oracle_iteration(cam_pass, loss, xi, k):
    """The LM camera solver variant (one successful Levenberg-Marquardt step per camera block on
    the Gauss-Newton model of its surrogate) in the same group function, FP64, against the
    oracle's step with cam_solver="lm", at the first iteration and at ones where 6-8 camera
    blocks restart: the same quantities and tolerances as the S-CAM test."""
    sc = cached_scene("circle")
    opts = O.Options(loss=loss, loss_scale_px=sc.loss_scale_px, xi=xi, cam_solver="lm")
    st, new, info, out, Fsum = _run(cam_pass, sc, opts, k)
    x = out[:, :15]
    F, Fbar, E_next, S_next, rs = out[:, 15], out[:, 16], out[:, 17], out[:, 18], out[:, 19] > 0.5
    scale = np.abs(info.Fbar_cam).max()
    np.testing.assert_allclose(F, info.F_cam, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(Fbar, info.Fbar_cam, rtol=0, atol=1e-11 * scale)
    clear = np.abs(info.Etest_cam - info.Fbar_cam) > 1e-8 * scale
    assert clear.mean() > 0.8
    np.testing.assert_array_equal(rs[clear], info.restart_cam[clear])
    if k > 0:
        assert info.restart_cam.sum() >= 5 and (~info.restart_cam).any()
    same = rs == info.restart_cam
    want = np.concatenate([new.R.reshape(-1, 9), new.t, new.d], 1)
    np.testing.assert_allclose(x[same], want[same], rtol=0, atol=1e-9)
    np.testing.assert_allclose(E_next[same], new.E_cam[same], rtol=0, atol=1e-10 * scale)
    np.testing.assert_allclose(S_next[same], (new.Fbar_cam - new.E_cam)[same], rtol=0, atol=1e-10 * scale)
