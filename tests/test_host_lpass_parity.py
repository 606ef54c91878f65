"""Parity of the landmark pass's per-landmark work on the CPU: the library's lpass_landmark (FP64,
the code nvcc compiles into k_lpass) built for the host with g++ and given, per landmark, the
records the camera pass writes: a and b of each term Q_ij at the extrapolated iterate and at
x^k (Eq. Q written around the conditioning landmark: w |lambda l - g|^2 + a/2 =
w lambda^2 |l - l_z|^2 + 2 w lambda (lambda l_z - g) . (l - l_z) + const), F_ij(x^k) and the
surrogate gap of Eq. DEalpha. The records are formed here from the oracle's majorizer, so the
test checks the pass's own arithmetic: the sums, Eqs. DEalpha, Fak and lFak in slack form, the
accelerated update (Eq. update_amm), the restart test (Eq. Eak) and the MM update
(Eq. update_mm), against one oracle iteration of Algorithm 1 per landmark block. No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import daba_oracle as O
from tests.conftest import cached_scene
from tests.test_host_device_math import FLAGS, HOST


@pytest.fixture(scope="module")
def lm_pass(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("lm_pass") / "lm_pass")
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, "lm_pass.cpp"), "-o", exe], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    return exe


def _ab(mj, lz):
    """a = w lambda^2 and b = w lambda (lambda l_z - g) of each term, around the landmark l_z."""
    wl = mj.w * mj.lam
    return wl * mj.lam, wl[:, None] * (mj.lam[:, None] * lz - mj.g)


def _iteration(scene, opts, k):
    """The oracle's state at iteration k, the records of iteration k and its step."""
    prob, R, t, d, l = O.make_problem(scene.cams, scene.lms, scene.cam_idx, scene.lm_idx, scene.uv, opts)
    st = O.init_state(prob, R, t, d, l)
    for _ in range(k):
        st, _ = O.step(prob, st)
    ci, li, u = prob.cam_idx, prob.lm_idx, prob.u
    _, gamma = O.nesterov(st.s)
    Rb, tb, db, lb = O.extrapolate(st.R, st.t, st.d, st.l, st.Rp, st.tp, st.dp, st.lp, gamma)
    mj_k = O.majorizer(prob.loss, prob.c, st.R[ci], st.t[ci], st.d[ci], st.l[li], u)
    mj_b = O.majorizer(prob.loss, prob.c, Rb[ci], tb[ci], db[ci], lb[li], u)
    mj_p = O.majorizer(prob.loss, prob.c, st.Rp[ci], st.tp[ci], st.dp[ci], st.lp[li], u)
    Fij = O.F_obs(prob.loss, prob.c, st.R[ci], st.t[ci], st.d[ci], st.l[li], u)
    gap = Fij - O.P_obs(mj_p, st.R[ci], st.t[ci], st.d[ci], u) - O.Q_obs(mj_p, st.l[li])
    ab, bb = _ab(mj_b, lb[li])
    ak, bk = _ab(mj_k, st.l[li])
    rec = np.concatenate([ab[:, None], bb, ak[:, None], bk, Fij[:, None], gap[:, None]], 1)
    new, info = O.step(prob, st)
    return prob, st, gamma, li, rec, new, info


def _device(exe, prob, st, gamma, li, rec, first, opts, bits=64, glob=0):
    N = prob.N
    order = np.argsort(li, kind="stable")
    ptr = np.concatenate([[0], np.cumsum(np.bincount(li, minlength=N))])
    dl = st.l - st.lp
    S = np.zeros(N) if first else st.Fbar_lm - st.E_lm
    lines = [f"{bits} {glob} {N} {int(first)} {float(gamma)!r} {float(opts.xi)!r} {float(opts.eta)!r} {int(opts.accelerated)}"]
    for j in range(N):
        rows = rec[order[ptr[j]:ptr[j + 1]]]
        head = [*st.l[j], *dl[j], S[j], st.E_lm[j]]
        lines.append(f"{len(rows)} " + " ".join(repr(float(x)) for x in head))
        lines.extend(" ".join(repr(float(x)) for x in r) for r in rows)
    run = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stderr[-2000:]
    out = np.array([[float(x) for x in line.split()] for line in run.stdout.splitlines()])
    assert out.shape == (N, 17 if glob else 11)
    return out


@pytest.mark.parametrize("xi,k", [(1e-10, 0), (1e-10, 8), (0.5, 0), (0.5, 12)])
def test_landmark_pass_matches_oracle_iteration(lm_pass, k, xi):
    """Per landmark of the 20-camera circle scene, at the first iteration (k = 0, slack 0 and
    E^(0) from the records) and at a later one where hundreds of landmark blocks restart (the
    slack and E^(k) carried in the landmark record): l^(k+1), its step, F^(k), Fbar^(k),
    E^(k+1), the next slack Fbar^(k) - E^(k+1), and the restart decision, against the oracle's
    step of Algorithm 1."""
    sc = cached_scene("circle")
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, xi=xi)
    prob, st, gamma, li, rec, new, info = _iteration(sc, opts, k)
    out = _device(lm_pass, prob, st, gamma, li, rec, k == 0, opts)
    lnew, step, S_next, E_next, F, Fbar, rs = (out[:, 0:3], out[:, 3:6], out[:, 6], out[:, 7], out[:, 8], out[:, 9],
                                              out[:, 10].astype(bool))
    scale = np.abs(info.Fbar_lm).max()
    np.testing.assert_allclose(F, info.F_lm, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(Fbar, info.Fbar_lm, rtol=0, atol=1e-12 * scale)
    # restart decisions agree wherever the test is not a near-tie in FP64 sums
    margin = np.abs(info.Etest_lm - info.Fbar_lm)
    clear = margin > 1e-9 * scale
    assert clear.mean() > 0.9
    np.testing.assert_array_equal(rs[clear], info.restart_lm[clear])
    if k > 0:
        assert info.restart_lm.sum() >= 100 and (~info.restart_lm).any()   # both branches are exercised
    same = rs == info.restart_lm
    np.testing.assert_allclose(lnew[same], new.l[same], rtol=0, atol=1e-10)
    np.testing.assert_allclose(step[same], (new.l - st.l)[same], rtol=0, atol=1e-10)
    np.testing.assert_allclose(E_next[same], new.E_lm[same], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(S_next[same], (new.Fbar_lm - new.E_lm)[same], rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("xi,k", [(1e-10, 0), (1e-10, 8), (0.5, 12)])
def test_mixed_landmark_pass_within_fp32_bounds(lm_pass, k, xi):
    """The MIXED instantiation (records, slack and step in FP32; the landmark as an FP32 high
    and low part) on the same records rounded to FP32: the new landmark within 1e-5 of the
    oracle's step (measured: at most 1.7e-6, a few FP32 ulps of the step, while the landmark
    itself keeps the 48-bit precision of its high and low parts), the next slack within 1e-6
    of the largest Fbar (measured 9e-9), and the restart decisions equal wherever the oracle's
    test margin is above 1e-5 of the largest Fbar (FP32 sums cannot resolve closer calls)."""
    sc = cached_scene("circle")
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, xi=xi)
    prob, st, gamma, li, rec, new, info = _iteration(sc, opts, k)
    out = _device(lm_pass, prob, st, gamma, li, rec, k == 0, opts, bits=32)
    lnew, S_next, rs = out[:, 0:3], out[:, 6], out[:, 10].astype(bool)
    scale = np.abs(info.Fbar_lm).max()
    clear = np.abs(info.Etest_lm - info.Fbar_lm) > 1e-5 * scale
    assert clear.mean() > 0.8
    np.testing.assert_array_equal(rs[clear], info.restart_lm[clear])
    same = rs == info.restart_lm
    step = np.abs(new.l - st.l).max(axis=1, keepdims=True)
    err = np.abs(lnew - new.l)
    # the FP32 step (1e-5 of its size) added to the high and low parts without further loss
    assert (err[same] <= 1e-5 * step[same] + 1e-12).all(), (err[same] / (step[same] + 1e-30)).max()
    np.testing.assert_allclose(S_next[same], (new.Fbar_lm - new.E_lm)[same], rtol=0, atol=1e-6 * scale)
