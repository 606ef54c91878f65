"""Method variant on the CUDA path: the global adaptive restart (one test on the summed block
metrics, all blocks restart together) with and without the momentum reset, against the FP64
oracle's restatement of the same variant."""
import numpy as np
import pytest

from oracle import daba_oracle as O
from tests.conftest import cached_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_07026_b300 import build
    build.build()


def _ctx(sc, prec="fp64", **kw):
    from paper_2305_07026_b300 import _lib as L
    opts = dict(loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec=prec)
    opts.update(kw)
    d = L.Daba(sc.M, sc.N, sc.nnz, **opts)
    d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    d.set_state(sc.cams, sc.lms)
    return d


@pytest.mark.parametrize("workload,reset,eta", [("circle", False, 0.5), ("circle", True, 0.5), ("circle", False, 1.0),
                                                ("street", True, 0.5)])
def test_global_restart_matches_oracle_per_iteration(workload, reset, eta):
    """F(x^k) within 1e-10 per iteration, the all-or-nothing decisions exactly (unless the global
    test is a near-tie, after which the comparison stops), block metrics and the final iterate."""
    sc = cached_scene("circle") if workload == "circle" else cached_scene("street", scale=0.05)
    K = 30
    o = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, eta=eta, restart="global", momentum_reset=reset)
    prob, R, t, dd, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, o)
    st = O.init_state(prob, R, t, dd, l)
    d = _ctx(sc, "fp64", eta=eta, restart="global", momentum_reset=reset)
    s2 = prob.s_norm ** 2
    fired = compared = 0
    for k in range(K):
        st, info = O.step(prob, st)
        tr = np.zeros(2)
        rs = np.zeros(1, np.int32)
        d.run(1, tr, rs)
        assert tr[0] == pytest.approx(info.F * s2, rel=1e-10), f"iteration {k}"
        m = d.get_block_metrics()
        np.testing.assert_allclose(m["Fbar_cam"], info.Fbar_cam * s2, rtol=1e-9, atol=1e-12 * info.F * s2)
        np.testing.assert_allclose(m["Fbar_lm"], info.Fbar_lm * s2, rtol=1e-9, atol=1e-12 * info.F * s2)
        want = int(info.restart_cam.sum() + info.restart_lm.sum())
        gap = info.Etest_cam.sum() + info.Etest_lm.sum() - info.Fbar_cam.sum() - info.Fbar_lm.sum()
        compared = k + 1
        if abs(gap) <= 1e-9 * abs(info.F):
            break
        assert rs[0] == want, f"iteration {k}"
        assert np.all(m["rs_cam"] == (want > 0)) and np.all(m["rs_lm"] == (want > 0))
        fired += want > 0
    assert compared == K and fired > 0
    cams_o, lms_o = O.to_boundary(st.R, st.t, st.d, st.l, prob.s_norm)
    cams_g, lms_g = d.get_state()
    np.testing.assert_allclose(cams_g, cams_o, rtol=1e-8, atol=1e-8)
    np.testing.assert_allclose(lms_g, lms_o, rtol=1e-8, atol=1e-8)
    d.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_global_restart_runs_and_checkpoints_bit_exact(prec):
    """One run of 40 iterations (CUDA graphs) equals 40 runs of one (direct launches), and a
    checkpoint taken after 17 iterations resumes bit-exactly, the device Nesterov scalar included."""
    sc = cached_scene("circle")
    kw = dict(restart="global", momentum_reset=True)
    a = _ctx(sc, prec, **kw)
    ta = np.zeros(41)
    ra = np.zeros(40, np.int32)
    a.run(40, ta, ra)
    b = _ctx(sc, prec, **kw)
    tb, rb = [], []
    for k in range(40):
        t1 = np.zeros(2)
        r1 = np.zeros(1, np.int32)
        b.run(1, t1, r1)
        tb.append(t1[0])
        rb.append(r1[0])
        if k == 16:
            ck = b.export_checkpoint()
    np.testing.assert_array_equal(ta[:40], np.array(tb))
    np.testing.assert_array_equal(ra, np.array(rb))
    assert (ra > 0).any()
    c = _ctx(sc, prec, **kw)
    c.import_checkpoint(ck)
    tc = np.zeros(24)
    c.run(23, tc)
    np.testing.assert_array_equal(tc[:23], ta[17:40])
    for x in (a, b, c):
        x.close()


def _mixed_reaches_fp64(sc, **kw):
    """MIXED reaches the FP64 path's objective after 150 iterations within 1e-5, within 200
    iterations: the two take different restart decisions, so while the objective still falls
    steeply one may be a few iterations behind the other."""
    out = {}
    for prec, n in (("fp64", 150), ("mixed", 200)):
        d = _ctx(sc, prec, **kw)
        tr = np.zeros(n + 1)
        d.run(n, tr)
        out[prec] = tr
        d.close()
    assert out["mixed"].min() <= out["fp64"][-1] * (1 + 1e-5)


def test_global_restart_mixed_reaches_fp64_objective():
    _mixed_reaches_fp64(cached_scene("tourism", scale=0.005), restart="global", momentum_reset=True)


def test_global_restart_monotone_at_eta_one():
    """With eta = 1, Fbar^(k) = F(x^k), so the global test keeps F non-increasing."""
    sc = cached_scene("tourism", scale=0.005)
    d = _ctx(sc, "fp64", eta=1.0, restart="global")
    tr = np.zeros(61)
    d.run(60, tr)
    assert np.all(np.diff(tr) <= 1e-12 * tr[:-1])
    d.close()


@pytest.mark.parametrize("reset", [False, True])
def test_global_restart_unrolled_grad(reset):
    """The reverse mode replays the global decisions (set on every block by the fix-up); with the
    momentum reset, also the Nesterov scalars the device continued (s <- 1 after a restart)."""
    from oracle import daba_unrolled as U
    from paper_2305_07026_b300 import _lib as L, scenes
    sc = scenes.circle_scene(seed=3)
    K = 15
    o = O.Options(loss="huber", loss_scale_px=2.0, pixel_scale=650.0, restart="global", eta=1.0,
                  momentum_reset=reset)
    rng = np.random.default_rng(4)
    g_c, g_l = rng.normal(size=sc.cams.shape), rng.normal(size=sc.lms.shape)
    gc, gl, gu, oc, ol, res = U.unrolled_grad(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, o, K, g_c, g_l)
    assert any(i.restart_cam.all() for i in res.infos)
    opts = dict(loss="huber", loss_scale_px=2.0, pixel_scale=650.0, prec="fp64", restart="global", eta=1.0,
                momentum_reset=reset)
    with L.Daba(sc.M, sc.N, sc.nnz, **opts) as d:
        d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
        d.set_state(sc.cams, sc.lms)
        gcg, glg, gug = d.unrolled_grad(K, g_c, g_l)
        cams, lms = d.get_state()
    np.testing.assert_allclose(cams, oc, rtol=1e-8, atol=1e-8)
    np.testing.assert_allclose(lms, ol, rtol=1e-8, atol=1e-8)
    for a, b in ((gcg, gc), (glg, gl), (gug, gu)):
        assert np.max(np.abs(a - b)) <= 1e-7 * np.max(np.abs(b))


def test_variant_options_validated():
    from paper_2305_07026_b300 import _lib as L
    with pytest.raises(L.DabaError):
        L.Daba(4, 4, 8, restart="block", momentum_reset=True)
    with pytest.raises(L.DabaError):
        L.Daba(4, 4, 8, restart=7)


@pytest.mark.parametrize("workload,accel", [("circle", True), ("street", True), ("circle", False)])
def test_lm_camera_solver_matches_oracle_per_iteration(workload, accel):
    """One successful LM step per camera subproblem (the paper's reported inner solver): F(x^k)
    within 1e-10 per iteration, restart decisions exactly (unless a near-tie), final iterate."""
    sc = cached_scene("circle") if workload == "circle" else cached_scene("street", scale=0.05)
    K = 20
    o = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, accelerated=accel, cam_solver="lm")
    prob, R, t, dd, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, o)
    st = O.init_state(prob, R, t, dd, l)
    d = _ctx(sc, "fp64", accelerated=accel, cam_solver="lm")
    s2 = prob.s_norm ** 2
    for k in range(K):
        st, info = O.step(prob, st)
        tr = np.zeros(2)
        rs = np.zeros(1, np.int32)
        d.run(1, tr, rs)
        assert tr[0] == pytest.approx(info.F * s2, rel=1e-10), f"iteration {k}"
        m = d.get_block_metrics()
        flips = 0
        for which in ("cam", "lm"):
            gpu = m[f"rs_{which}"].astype(bool)
            ora = getattr(info, f"restart_{which}")
            E, Fb, F = (getattr(info, f"Etest_{which}"), getattr(info, f"Fbar_{which}"),
                        np.abs(getattr(info, f"F_{which}")))
            tie = np.abs(E - Fb) <= 1e-9 * np.maximum(F, 1e-300)
            assert not ((gpu != ora) & ~tie).any(), f"iteration {k}: {which}"
            flips += int((gpu != ora).sum())
        assert flips == 0, f"iteration {k}: near-tie restart decision"
    cams_o, lms_o = O.to_boundary(st.R, st.t, st.d, st.l, prob.s_norm)
    cams_g, lms_g = d.get_state()
    np.testing.assert_allclose(cams_g, cams_o, rtol=1e-8, atol=1e-8)
    np.testing.assert_allclose(lms_g, lms_o, rtol=1e-8, atol=1e-8)
    d.close()


def test_lm_camera_solver_mixed_reaches_fp64_objective():
    _mixed_reaches_fp64(cached_scene("tourism", scale=0.005), cam_solver="lm")


def test_lm_camera_solver_reverse_mode_mixed():
    """The reverse mode covers the LM camera solver on MIXED contexts too (FP64 parity in
    test_gpu_grad.py): along the MIXED run, its product agrees with the FP64 context's to
    FP32-level relative error; an unknown solver is refused."""
    from paper_2305_07026_b300 import _lib as L
    sc = cached_scene("circle")
    rng = np.random.default_rng(5)
    seed = (rng.normal(size=sc.cams.shape), rng.normal(size=sc.lms.shape))
    out = {}
    for prec in ("fp64", "mixed"):
        d = _ctx(sc, prec, cam_solver="lm")
        out[prec] = d.unrolled_grad(3, *seed)
        d.close()
    for a, b in zip(out["mixed"], out["fp64"]):
        assert np.all(np.isfinite(a))
        np.testing.assert_allclose(a, b, rtol=2e-3, atol=2e-3 * np.abs(b).max())
    with pytest.raises(L.DabaError):
        L.Daba(4, 4, 8, cam_solver=5)


@pytest.mark.parametrize("kw", [dict(restart="global", cam_solver="lm"),
                                dict(restart="global", momentum_reset=True, cam_solver="lm", eta=1.0),
                                dict(restart="global", accelerated=False)])
def test_variant_combinations_match_oracle(kw):
    """The variants combined (global restart with the LM camera solver, with the momentum reset at
    eta = 1, and DUBA, where the restart mode has no effect): F(x^k) within 1e-10 for 15 iterations
    and the restart counts exactly."""
    sc = cached_scene("circle")
    ok = dict(kw)
    o = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, **ok)
    res = O.daba(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, o, 15, keep_infos=15)
    d = _ctx(sc, "fp64", **kw)
    tr = np.zeros(16)
    rs = np.zeros(15, np.int32)
    d.run(15, tr, rs)
    d.close()
    np.testing.assert_allclose(tr, res.trace_px2, rtol=1e-10)
    assert rs.tolist() == res.restarts.tolist()
