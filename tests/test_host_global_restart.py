"""The global restart variant on the CPU: one test of Algorithm 1 on the block made of every
camera and landmark (sum of E^alpha(k+1) against the sum of Fbar^alpha(k)). The library's camera
solve group and landmark pass, built for the host with g++, keep each block's accelerated step,
its MM alternative with E and the slack after a restart, and its term E^alpha(k+1) -
Fbar^alpha(k) of the test; after the reduction the fix-up kernels copy the MM alternative
everywhere if the sum of the terms is positive. Checked against the oracle (restart="global"):
every block's accelerated step, MM alternative and test term, the decision taken from the
terms' sum, and the state that decision selects, at iterations where the test fires and where
it does not. No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import daba_oracle as O
from tests.conftest import cached_scene
from tests.test_host_device_math import FLAGS, HOST
from tests import test_host_camsolve_parity as CAM
from tests import test_host_lpass_parity as LM


def _build(tmp_path_factory, name):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp(name) / name)
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, f"{name}.cpp"), "-o", exe], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    return exe


@pytest.fixture(scope="module")
def drivers(tmp_path_factory):
    return _build(tmp_path_factory, "cam_pass"), _build(tmp_path_factory, "lm_pass")


@pytest.mark.parametrize("xi,k,fires", [(1e-10, 13, False), (1e-10, 14, True), (0.5, 18, False), (0.5, 19, True)])
def test_global_restart_matches_oracle(drivers, xi, k, fires):
    cam_exe, lm_exe = drivers
    sc = cached_scene("circle")
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, xi=xi, restart="global")
    # camera half (the driver runs the oracle's step itself, with the global option)
    st, new, info, out, _ = CAM._run(cam_exe, sc, opts, k, glob=1)
    assert bool(info.restart_cam[0]) == fires and (info.restart_cam == fires).all()
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    ci, li, u, M, N = prob.cam_idx, prob.lm_idx, prob.u, prob.M, prob.N
    _, gamma = O.nesterov(st.s)
    Rb, tb, db, lb = O.extrapolate(st.R, st.t, st.d, st.l, st.Rp, st.tp, st.dp, st.lp, gamma)
    mj_k = O.majorizer(prob.loss, prob.c, st.R[ci], st.t[ci], st.d[ci], st.l[li], u)
    mj_b = O.majorizer(prob.loss, prob.c, Rb[ci], tb[ci], db[ci], lb[li], u)
    Ra, ta, da = O.solve_cameras(opts.xi, mj_b, Rb, tb, db, ci, u, M, opts.cam_alternations)
    Rm, tm, dm = O.solve_cameras(opts.xi, mj_k, st.R, st.t, st.d, ci, u, M, opts.cam_alternations)
    E0 = O.E_cam(opts.xi, mj_k, st.R, st.t, st.d, st.R, st.t, st.d, ci, u, M)
    Emm_cam = O.E_cam(opts.xi, mj_k, Rm, tm, dm, st.R, st.t, st.d, ci, u, M) + info.F_cam - E0
    scale = np.abs(info.Fbar_cam).max()
    x, g_cam, alt = out[:, :15], out[:, 21], out[:, 22:37]
    alt_E, alt_S = out[:, 37], out[:, 38]
    np.testing.assert_allclose(x, np.concatenate([Ra.reshape(-1, 9), ta, da], 1), rtol=0, atol=1e-9)
    np.testing.assert_allclose(alt, np.concatenate([Rm.reshape(-1, 9), tm, dm], 1), rtol=0, atol=1e-9)
    np.testing.assert_allclose(g_cam, info.Etest_cam - info.Fbar_cam, rtol=0, atol=1e-10 * scale)
    np.testing.assert_allclose(alt_E, Emm_cam, rtol=0, atol=1e-10 * scale)
    np.testing.assert_allclose(alt_S, info.Fbar_cam - Emm_cam, rtol=0, atol=1e-10 * scale)
    # landmark half on records formed from the oracle's majorizer
    prob_l, st_l, gamma_l, li_l, rec, new_l, info_l = LM._iteration(sc, opts, k)
    lout = LM._device(lm_exe, prob_l, st_l, gamma_l, li_l, rec, k == 0, opts, glob=1)
    la = O.solve_landmarks(opts.xi, mj_b, lb, li, N)
    lmm = O.solve_landmarks(opts.xi, mj_k, st.l, li, N)
    E0l = O.E_lm(opts.xi, mj_k, st.l, st.l, li, N)
    Emm_lm = O.E_lm(opts.xi, mj_k, lmm, st.l, li, N) + info_l.F_lm - E0l
    scale_l = np.abs(info_l.Fbar_lm).max()
    np.testing.assert_allclose(lout[:, 0:3], la, rtol=0, atol=1e-10)
    gsum = lout[:, 11]
    np.testing.assert_allclose(gsum, info_l.Etest_lm - info_l.Fbar_lm, rtol=0, atol=1e-11 * scale_l)
    np.testing.assert_allclose(lout[:, 12:15], lmm - st.l, rtol=0, atol=1e-10)
    np.testing.assert_allclose(lout[:, 15], info_l.Fbar_lm - Emm_lm, rtol=0, atol=1e-11 * scale_l)
    np.testing.assert_allclose(lout[:, 16], Emm_lm, rtol=0, atol=1e-11 * scale_l)
    # the decision from the sum of the blocks' terms, and the state it selects (the fix-up
    # kernels copy the MM alternative; otherwise the accelerated step stays)
    total = g_cam.sum() + gsum.sum()
    assert (total > 0) == fires
    cams_next = alt if fires else x
    lms_next = st.l + lout[:, 12:15] if fires else lout[:, 0:3]
    np.testing.assert_allclose(cams_next, np.concatenate([new.R.reshape(-1, 9), new.t, new.d], 1), rtol=0, atol=1e-9)
    np.testing.assert_allclose(lms_next, new_l.l, rtol=0, atol=1e-10)
