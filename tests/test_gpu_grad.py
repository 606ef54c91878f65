"""Gradient of the objective through the C ABI (adjoint kernels) and the PyTorch autograd
function: against the oracle's boundary gradient (itself pinned by FP64 central differences)
and against FP64 central differences of the library's own objective along random directions."""
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


def _ctx(sc, prec, **kw):
    from paper_2305_07026_b300 import _lib as L
    o = dict(loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec=prec)
    o.update(kw)
    d = L.Daba(sc.M, sc.N, sc.nnz, **o)
    d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    d.set_state(sc.cams, sc.lms)
    return d


def _close(a, b, tol):
    a, b = np.asarray(a), np.asarray(b)
    np.testing.assert_allclose(a, b, rtol=tol, atol=tol * np.abs(b).max())


@pytest.mark.parametrize("workload,scale,prec", [("circle", 1.0, "fp64"), ("circle", 1.0, "mixed"),
                                                 ("tourism", 0.005, "fp64"), ("street", 0.05, "fp64")])
def test_objective_grad_matches_oracle(workload, scale, prec):
    sc = cached_scene(workload, scale=scale)
    F, gc, gl, gu = O.grad_objective_boundary(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv,
                                              O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px))
    d = _ctx(sc, prec)
    Fg, gcg, glg, gug = d.objective_grad()
    tol = 1e-9 if prec == "fp64" else 2e-4
    assert Fg == pytest.approx(F, rel=1e-11 if prec == "fp64" else 1e-5)
    _close(gcg, gc, tol)
    _close(glg, gl, tol)
    _close(gug, gu, tol)
    # after iterations the gradient is taken at the new iterate
    d.run(3)
    cams, lms = d.get_state()
    F3, gc3, gl3, gu3 = O.grad_objective_boundary(cams, lms, sc.cam_idx, sc.lm_idx, sc.uv,
                                                  O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px))
    Fg3, gcg3, glg3, gug3 = d.objective_grad()
    assert Fg3 == pytest.approx(F3, rel=1e-10 if prec == "fp64" else 1e-5)
    _close(glg3, gl3, tol)
    d.close()


def test_autograd_matches_central_differences():
    """Differentiation workload: 200 cameras of the street generator, Huber 1 px, FP64 path;
    autograd gradient against FP64 central differences (h = 1e-6 relative) on 64 random
    directions."""
    from paper_2305_07026_b300.autograd import objective
    sc = cached_scene("street", scale=0.2)
    d = _ctx(sc, "fp64", loss="huber", loss_scale_px=1.0)
    dev = "cuda"
    cams = torch.tensor(sc.cams, device=dev, requires_grad=True)
    lms = torch.tensor(sc.lms, device=dev, requires_grad=True)
    uv = torch.tensor(sc.uv, device=dev, requires_grad=True)
    F = objective(d, cams, lms, uv)
    F.backward()
    gc, gl, gu = cams.grad.detach().clone(), lms.grad.detach().clone(), uv.grad.detach().clone()
    rng = np.random.default_rng(7)
    cscale = torch.tensor([1e-3, 1e-3, 1e-3, 1e-2, 1e-2, 1e-2, 1.0, 1e-4, 1e-6], dtype=torch.float64, device=dev)
    h = 1e-6 / 1e-3
    with torch.no_grad():
        for k in range(64):
            vc = torch.tensor(rng.normal(size=sc.cams.shape), device=dev) * cscale * 1e-3
            vl = torch.tensor(rng.normal(size=sc.lms.shape), device=dev) * 1e-5
            vu = torch.tensor(rng.normal(size=sc.uv.shape), device=dev) * 1e-4
            fp = objective(d, cams + h * vc, lms + h * vl, uv + h * vu).item()
            fm = objective(d, cams - h * vc, lms - h * vl, uv - h * vu).item()
            fd = (fp - fm) / (2 * h)
            an = float((gc * vc).sum() + (gl * vl).sum() + (gu * vu).sum())
            assert an == pytest.approx(fd, rel=1e-5, abs=1e-10 * F.item()), k
    d.close()


def test_set_pixels_matches_set_observations():
    sc = cached_scene("circle")
    rng = np.random.default_rng(3)
    uv2 = sc.uv + rng.normal(0, 0.5, sc.uv.shape)
    from paper_2305_07026_b300 import _lib as L
    for prec in ("fp64", "mixed"):
        a = _ctx(sc, prec)
        a.set_pixels(uv2)
        b = L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec=prec)
        b.set_observations(sc.cam_idx, sc.lm_idx, uv2)
        b.set_state(sc.cams, sc.lms)
        ta, tb = np.zeros(6), np.zeros(6)
        a.run(5, ta)
        b.run(5, tb)
        np.testing.assert_array_equal(ta, tb)
        bad = uv2.copy()
        bad[4, 0] = np.nan
        with pytest.raises(L.DabaError) as e:
            a.set_pixels(bad)
        assert e.value.status == L.DABA_ERR_NONFINITE
        a.close()
        b.close()


def _rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("case", ["small-huber-6", "small-cauchy-12", "small-trivial-mm-8", "small-huber-50",
                                  "circle-tiles-12", "circle-welsch-20", "street-12", "small-huber-lm-6",
                                  "small-cauchy-mm-lm-5", "street-lm-8", "small-huber-reset-15",
                                  "small-trivial-lm-reset-14"])
def test_unrolled_grad_matches_oracle(case):
    """Vector-Jacobian product of K iterations (the CUDA adjoint kernels, states kept every 10
    iterations and recomputed) against autograd through the oracle's PyTorch restatement of the
    update, which is itself pinned by FP64 central differences of the numpy oracle."""
    from oracle import daba_unrolled as U
    from paper_2305_07026_b300 import _lib as L, scenes
    kw = {}
    if case.startswith("small"):
        sc = scenes.circle_scene(seed=11, n_cams=6, n_lms=40, cap=6)
        loss, K = case.split("-")[1], int(case.split("-")[-1])
        accel = "mm" not in case
        scale_px = 2.0
    elif case == "circle-tiles-12":   # several chunks per camera and many landmark tiles
        sc = scenes.circle_scene(seed=3)
        loss, K, accel, scale_px = "huber", 12, True, 2.0
        kw = dict(chunk_obs=64, tile_obs=128, tile_lms=16)
    elif case == "circle-welsch-20":
        sc = scenes.circle_scene(seed=5)
        loss, K, accel, scale_px = "welsch", 20, True, 60.0   # no saturated block (no exact restart ties)
    else:
        sc = cached_scene("street", scale=0.05)
        loss, K, accel, scale_px = sc.loss, int(case.split("-")[-1]), True, sc.loss_scale_px
    solver = "lm" if "-lm-" in case else "scam"   # the LM camera solver variant
    kw["cam_solver"] = solver
    ok = {}
    if "-reset-" in case:   # global restart with the momentum reset (one restart fires within K)
        kw.update(restart="global", momentum_reset=True)
        ok = dict(restart="global", momentum_reset=True)
    o = O.Options(loss=loss, loss_scale_px=scale_px, accelerated=accel, pixel_scale=650.0, cam_solver=solver, **ok)
    rng = np.random.default_rng(4)
    g_c, g_l = rng.normal(size=sc.cams.shape), rng.normal(size=sc.lms.shape)
    gc, gl, gu, oc, ol, res = U.unrolled_grad(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, o, K, g_c, g_l)
    opts = dict(loss=loss, loss_scale_px=scale_px, accelerated=accel, pixel_scale=650.0, prec="fp64", **kw)
    # the restart decisions the adjoint replays are those of the oracle's run
    with L.Daba(sc.M, sc.N, sc.nnz, **opts) as d:
        d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
        d.set_state(sc.cams, sc.lms)
        rs = np.zeros(K, np.int32)
        d.run(K, restarts=rs)
        want = [int(np.sum(i.restart_cam)) + int(np.sum(i.restart_lm)) for i in res.infos] if accel else [0] * K
        assert rs.tolist() == want
        if ok:
            assert any(want[:K - 1])
    with L.Daba(sc.M, sc.N, sc.nnz, **opts) as d:
        d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
        d.set_state(sc.cams, sc.lms)
        gcg, glg, gug = d.unrolled_grad(K, g_c, g_l)
        cams, lms = d.get_state()   # left at x^K
        np.testing.assert_allclose(cams, oc, rtol=1e-8, atol=1e-8)
        np.testing.assert_allclose(lms, ol, rtol=1e-8, atol=1e-8)
        errs = {"cams": _rel_err(gcg, gc), "lms": _rel_err(glg, gl), "uv": _rel_err(gug, gu)}
        assert max(errs.values()) < 1e-7, errs
        with pytest.raises(L.DabaError):   # iterations have run since the state was set
            d.unrolled_grad(K, g_c, g_l)


def test_unrolled_grad_linear_in_seed():
    """The product is linear in the seed and K = 1 of a seed on one landmark touches only what
    that landmark's update reads."""
    from paper_2305_07026_b300 import _lib as L, scenes
    sc = scenes.circle_scene(seed=11, n_cams=6, n_lms=40, cap=6)
    rng = np.random.default_rng(9)
    s1 = (rng.normal(size=sc.cams.shape), rng.normal(size=sc.lms.shape))
    s2 = (rng.normal(size=sc.cams.shape), rng.normal(size=sc.lms.shape))

    def vjp(seed, K):
        with L.Daba(sc.M, sc.N, sc.nnz, loss="huber", loss_scale_px=2.0, prec="fp64") as d:
            d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
            d.set_state(sc.cams, sc.lms)
            return d.unrolled_grad(K, *seed)
    a, b = vjp(s1, 5), vjp(s2, 5)
    c = vjp((2.0 * s1[0] - s2[0], 2.0 * s1[1] - s2[1]), 5)
    for x, y, z in zip(a, b, c):
        np.testing.assert_allclose(z, 2.0 * x - y, rtol=1e-9, atol=1e-9 * np.abs(z).max())
    seed = (np.zeros_like(sc.cams), np.zeros_like(sc.lms))
    seed[1][7] = [1.0, -2.0, 0.5]
    gc, gl, gu = vjp(seed, 1)
    obs = np.flatnonzero(sc.lm_idx == 7)
    others = np.setdiff1d(np.arange(sc.nnz), obs)
    assert np.all(gu[others] == 0.0) and np.any(gu[obs] != 0.0)
    assert np.all(np.delete(gl, 7, axis=0) == 0.0)
    assert np.all(np.delete(gc, np.unique(sc.cam_idx[obs]), axis=0) == 0.0)


def test_unrolled_autograd_matches_central_differences():
    """torch.autograd through K iterations of the library (backward: the CUDA adjoint) against
    FP64 central differences of the library's own K-iteration map along random directions."""
    from paper_2305_07026_b300 import _lib as L, autograd as A, scenes
    sc = scenes.circle_scene(seed=11, n_cams=6, n_lms=40, cap=6)
    K = 7
    dev = torch.device("cuda:0")
    d = L.Daba(sc.M, sc.N, sc.nnz, loss="huber", loss_scale_px=2.0, pixel_scale=650.0, prec="fp64")
    d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    d.set_state(sc.cams, sc.lms)
    c0 = torch.tensor(sc.cams, device=dev, requires_grad=True)
    l0 = torch.tensor(sc.lms, device=dev, requires_grad=True)
    u0 = torch.tensor(sc.uv, device=dev, requires_grad=True)
    rng = np.random.default_rng(2)
    wc = torch.tensor(rng.normal(size=sc.cams.shape), device=dev)
    wl = torch.tensor(rng.normal(size=sc.lms.shape), device=dev)
    oc, ol = A.unrolled(d, c0, l0, u0, K)
    y = (oc * wc).sum() + (ol * wl).sum()
    gc, gl, gu = torch.autograd.grad(y, (c0, l0, u0))

    def J(c, l, u):
        with torch.no_grad():
            a, b = A.unrolled(d, c, l, u, K)
            return float((a * wc).sum() + (b * wl).sum())
    cscale = torch.tensor([1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 0.5, 1e-4, 1e-6], device=dev, dtype=torch.float64)
    for part in range(3):
        for rep in range(3):
            v = [torch.zeros_like(c0), torch.zeros_like(l0), torch.zeros_like(u0)]
            r = torch.tensor(rng.normal(size=tuple(v[part].shape)), device=dev)
            v[part] = r * (cscale if part == 0 else (1e-3 if part == 1 else 1e-2))
            h = (1e-3, 1e-2, 1e-2)[part]
            c, l, u = c0.detach(), l0.detach(), u0.detach()
            fd = (J(c + h * v[0], l + h * v[1], u + h * v[2]) - J(c - h * v[0], l - h * v[1], u - h * v[2])) / (2 * h)
            an = float((gc * v[0]).sum() + (gl * v[1]).sum() + (gu * v[2]).sum())
            assert an == pytest.approx(fd, rel=1e-5, abs=1e-9), (part, rep)
    d.close()


def test_unrolled_grad_differentiation_workload_k50():
    """The differentiation workload (street generator scaled to 200 cameras, ~150k observations)
    with K = 50 (five checkpoint segments): the product is finite and linear in the seed, and the
    state left after it is bit-identical to daba_run(50). (Element-wise comparison with the
    oracle's autograd is done on the smaller scenes above: at this size the oracle's graph needs
    tens of GB and some restart decisions sit within 1e-11 of a tie.)"""
    from paper_2305_07026_b300 import _lib as L
    sc = cached_scene("street", scale=0.2)
    opts = dict(loss="huber", loss_scale_px=1.0, prec="fp64")
    rng = np.random.default_rng(8)
    s1 = (rng.normal(size=sc.cams.shape), rng.normal(size=sc.lms.shape))
    s2 = (rng.normal(size=sc.cams.shape), rng.normal(size=sc.lms.shape))

    def vjp(seed):
        with L.Daba(sc.M, sc.N, sc.nnz, **opts) as d:
            d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
            d.set_state(sc.cams, sc.lms)
            g = d.unrolled_grad(50, *seed)
            return g, d.get_state()
    (a, st_a), (b, _) = vjp(s1), vjp(s2)
    (c, _) = vjp((s1[0] + 3.0 * s2[0], s1[1] + 3.0 * s2[1]))
    for x, y, z in zip(a, b, c):
        assert np.all(np.isfinite(x))
        np.testing.assert_allclose(z, x + 3.0 * y, rtol=1e-9, atol=1e-9 * np.abs(z).max())
    with L.Daba(sc.M, sc.N, sc.nnz, **opts) as d:
        d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
        d.set_state(sc.cams, sc.lms)
        d.run(50)
        cams, lms = d.get_state()
    np.testing.assert_array_equal(st_a[0], cams)
    np.testing.assert_array_equal(st_a[1], lms)


@pytest.mark.parametrize("accel,K,reset", [(False, 8, False), (True, 4, False), (True, 12, False), (True, 15, True)])
def test_unrolled_grad_mixed_context(accel, K, reset):
    """Reverse mode of a MIXED context: the product along the MIXED run's iterates and decisions
    with FP64 adjoint arithmetic. Its trajectory differs from the FP64 one by FP32 rounding only
    (checked: the same restart counts), so the two products agree to FP32-level relative error;
    the product is linear in the seed, and the context is left at x^K bit for bit as run(K)."""
    from paper_2305_07026_b300 import _lib as L, scenes
    sc = scenes.circle_scene(seed=11, n_cams=6, n_lms=40, cap=6)
    rng = np.random.default_rng(21)
    g_c, g_l = rng.normal(size=sc.cams.shape), rng.normal(size=sc.lms.shape)
    opts = dict(loss="huber", loss_scale_px=2.0, accelerated=accel, pixel_scale=650.0)
    if reset:   # global restart with the momentum reset
        opts.update(restart="global", momentum_reset=True)

    def ctx(prec):
        d = L.Daba(sc.M, sc.N, sc.nnz, prec=prec, **opts)
        d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
        d.set_state(sc.cams, sc.lms)
        return d

    rs = {}
    for prec in ("fp64", "mixed"):
        with ctx(prec) as d:
            r = np.zeros(K, np.int32)
            d.run(K, restarts=r)
            rs[prec] = r
    assert rs["mixed"].tolist() == rs["fp64"].tolist()
    with ctx("fp64") as d:
        gc64, gl64, gu64 = d.unrolled_grad(K, g_c, g_l)
    with ctx("mixed") as d:
        gcm, glm, gum = d.unrolled_grad(K, g_c, g_l)
        cams_m, lms_m = d.get_state()
        gcm2, glm2, gum2 = None, None, None
    with ctx("mixed") as d:
        d.run(K)
        cams_r, lms_r = d.get_state()
    np.testing.assert_array_equal(cams_m, cams_r)
    np.testing.assert_array_equal(lms_m, lms_r)
    errs = {"cams": _rel_err(gcm, gc64), "lms": _rel_err(glm, gl64), "uv": _rel_err(gum, gu64)}
    assert max(errs.values()) < 2e-3, errs
    with ctx("mixed") as d:   # linear in the seed
        gcm2, glm2, gum2 = d.unrolled_grad(K, 2.0 * g_c, -3.0 * g_l)
    with ctx("mixed") as d:
        gcl, gll, gul = d.unrolled_grad(K, g_c, np.zeros_like(g_l))
    with ctx("mixed") as d:
        gcr, glr, gur = d.unrolled_grad(K, np.zeros_like(g_c), g_l)
    for a, b, c in ((gcm2, gcl, gcr), (glm2, gll, glr), (gum2, gul, gur)):
        np.testing.assert_allclose(a, 2.0 * b - 3.0 * c, rtol=1e-9, atol=1e-9 * np.max(np.abs(a)))
