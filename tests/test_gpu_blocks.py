"""Coarse blocks on the GPU (daba_set_partition: contiguous groups of one to BLK_MAX_CAMS cameras
and the landmarks they see first; the block scratch in shared memory up to 16 cameras per block,
in global memory above, Eq. Ealpha with the intra-block pairs exact, one successful LM step
per block) against the oracle of Algorithm 1 with the same blocks (oracle/daba_blocks.py), per
iteration: the objective trace, the per-block restart metrics F^alpha and Fbar^alpha, the restart
decisions and the iterate."""
import numpy as np
import pytest

from oracle import daba_blocks as B
from oracle import daba_oracle as O
from tests.conftest import cached_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NEAR_TIE = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_07026_b300 import build
    build.build()


def _residuals(prob, cams, lms):
    """The reprojection error vectors (Eq. error) of every observation at a boundary state."""
    R, t, d, l = O.to_internal(cams, lms, prob.s_norm)
    ci, li = prob.cam_idx, prob.lm_idx
    return O.reproj_error(R[ci], t[ci], l[li], O.ray(prob.u, d[ci]))


def _scene(name):
    from paper_2305_07026_b300 import scenes
    if name == "circle":
        return cached_scene("circle")
    if name == "circle_small":
        return scenes.circle_scene(n_lms=300)
    return cached_scene(name, scale={"street": 0.05, "tourism": 0.005}[name])


@pytest.mark.parametrize("name,accel,K,n_blocks,ctas", [(*c, 0) if len(c) == 4 else c for c in [
    ("circle", True, 20, None), ("circle_small", False, 12, None), ("street", True, 12, None),
    ("tourism", True, 20, None), ("tourism", True, 12, None, 1),
    # several cameras per block: the Schur complement couples the block's cameras. Such a block
    # is a small bundle adjustment whose gauge only the inter pairs and xi hold, and two correct
    # solves of its damped system part at ~1e-10 after one step; the parting grows about threefold
    # per iteration, so the trajectory is compared for 12 iterations and the iterate not at all
    # (test_multi_camera_blocks_step_from_common_state compares every step from the GPU's state)
    ("circle", True, 12, 4), ("circle", True, 12, 8), ("circle_small", False, 12, 3), ("circle_small", True, 12, 6),
    ("street", True, 8, 25), ("tourism", True, 12, 8), ("tourism", True, 12, 32),
    # blocks of 10 and 15 cameras on one CTA each (shared-memory scratch) and on clusters; 20 and
    # 25 cameras on one CTA (global scratch) and on clusters; the oracle takes seconds per
    # iteration on the larger ones
    ("circle", True, 12, 4, 1), ("circle", True, 12, 2, 1), ("circle", True, 12, 2), ("tourism", True, 4, 4, 1),
    ("tourism", True, 4, 4), ("circle", True, 12, 1, 1), ("circle", True, 12, 1), ("circle", True, 12, 1, 4),
    ("street", True, 4, 2)]])
def test_blocks_match_oracle_per_iteration(name, accel, K, n_blocks, ctas):
    from paper_2305_07026_b300 import _lib as L
    sc = _scene(name)
    part = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, n_blocks or sc.M)
    assert np.bincount(part.cam_block).max() <= L.BLK_MAX_CAMS
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, accelerated=accel)
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    st = B.init_state(prob, part, R, t, d, l)
    s2 = prob.s_norm ** 2
    g = L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec="fp64", accelerated=accel)
    g.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    g.set_block_ctas(ctas)
    g.set_partition(part.cam_block, part.lm_block, part.S)
    g.set_state(sc.cams, sc.lms)
    compared = 0
    for k in range(K):
        st, info = B.step(prob, part, st)
        tr = np.zeros(2)
        rs = np.zeros(1, np.int32)
        g.run(1, tr, rs)
        assert tr[0] == pytest.approx(info.F * s2, rel=1e-10), f"iteration {k}"
        F_blk, Fb_blk, rs_blk = g.get_partition_metrics()
        # Lemma 1a on the GPU's own block metrics
        assert F_blk.sum() == pytest.approx(tr[0], rel=1e-10)
        np.testing.assert_allclose(F_blk, info.F_blk * s2, rtol=1e-9, atol=1e-12 * info.F * s2)
        np.testing.assert_allclose(Fb_blk, info.Fbar_blk * s2, rtol=1e-9, atol=1e-12 * info.F * s2)
        tie = np.abs(info.Etest - info.Fbar_blk) <= NEAR_TIE * np.abs(info.F_blk)
        bad = (rs_blk.astype(bool) != info.restart) & ~tie
        assert not bad.any(), f"iteration {k}: restart decisions differ at {np.flatnonzero(bad)[:10]}"
        compared = k + 1
        if (rs_blk.astype(bool) != info.restart).any():
            break
    assert compared >= min(K, 10)
    if compared == K and (n_blocks is None or name == "circle_small"):
        cams_o, lms_o = O.to_boundary(st.R, st.t, st.d, st.l, prob.s_norm)
        cams_g, lms_g = g.get_state()
        np.testing.assert_allclose(cams_g, cams_o, rtol=1e-8, atol=1e-8)
        np.testing.assert_allclose(lms_g, lms_o, rtol=1e-8, atol=1e-8)
    g.close()


@pytest.mark.parametrize("ctas,reset", [(1, False), (1, True), (4, True)])
def test_blocks_global_restart_trajectory(ctas, reset):
    """The global restart over coarse blocks (one camera each, with the landmarks it sees first):
    the objective trace, block metrics and the one decision per iteration against the block
    oracle for 16 iterations (a restart fires at iteration 12), with and without the momentum
    reset (s <- 1 after it), on one CTA per block and on clusters; then the iterate."""
    from paper_2305_07026_b300 import _lib as L
    sc = _scene("circle_small")
    part = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, sc.M)
    kw = dict(restart="global", momentum_reset=reset)
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, **kw)
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    st = B.init_state(prob, part, R, t, d, l)
    s2 = prob.s_norm ** 2
    g = L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec="fp64", **kw)
    g.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    g.set_block_ctas(ctas)
    g.set_partition(part.cam_block, part.lm_block, part.S)
    g.set_state(sc.cams, sc.lms)
    n_cam_blocks = len(np.unique(part.cam_block))
    fired = []
    for k in range(16):
        st, info = B.step(prob, part, st)
        tr = np.zeros(2)
        rs = np.zeros(1, np.int32)
        g.run(1, tr, rs)
        assert tr[0] == pytest.approx(info.F * s2, rel=1e-10), f"iteration {k}"
        F_blk, Fb_blk, rs_blk = g.get_partition_metrics()
        np.testing.assert_allclose(F_blk, info.F_blk * s2, rtol=1e-9, atol=1e-12 * info.F * s2)
        np.testing.assert_allclose(Fb_blk, info.Fbar_blk * s2, rtol=1e-9, atol=1e-12 * info.F * s2)
        np.testing.assert_array_equal(rs_blk.astype(bool), info.restart)
        assert rs[0] == (n_cam_blocks if info.restart.any() else 0)
        if info.restart.any():
            fired.append(k)
    assert fired and fired[0] < 15
    cams_o, lms_o = O.to_boundary(st.R, st.t, st.d, st.l, prob.s_norm)
    cams_g, lms_g = g.get_state()
    np.testing.assert_allclose(cams_g, cams_o, rtol=1e-8, atol=1e-8)
    np.testing.assert_allclose(lms_g, lms_o, rtol=1e-8, atol=1e-8)
    g.close()


@pytest.mark.parametrize("name,n_blocks,iters,ctas,restart", [(*c, "block") if len(c) == 4 else c for c in [
    ("circle", 4, 20, 1), ("circle", 8, 20, 0), ("tourism", 8, 20, 1), ("tourism", 8, 6, 0), ("tourism", 32, 20, 0),
    ("circle", 2, 20, 0), ("circle", 1, 20, 1), ("circle", 1, 20, 0), ("street", 2, 4, 0), ("tourism", 1, 3, 0),
    # the global restart (fires at iteration 12 on this scene), with and without the momentum reset
    ("circle_small", 4, 16, 1, "global"), ("circle_small", 2, 16, 0, "reset")]])
def test_multi_camera_blocks_step_from_common_state(name, n_blocks, iters, ctas, restart):
    """Every one of `iters` iterations (blocks of up to 60 cameras) from the same state: before each GPU iteration the oracle takes
    the GPU's x^k and x^(k-1) (through the boundary) and its Fbar^alpha(k-1); the oracle's Nesterov
    scalar and E^alpha carry over from its own previous step. Compared after the step: the block
    metrics F^alpha(k), Fbar^alpha(k) (which hold the previous step's E^alpha(x^k | x^(k-1))), the
    restart decisions and x^(k+1)."""
    import dataclasses
    from paper_2305_07026_b300 import _lib as L
    sc = _scene(name)
    part = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, n_blocks)
    kw = {"block": {}, "global": {"restart": "global"}, "reset": {"restart": "global", "momentum_reset": True}}[restart]
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, **kw)
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    st = B.init_state(prob, part, R, t, d, l)
    s2 = prob.s_norm ** 2
    fired = 0
    g = L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec="fp64", **kw)
    g.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    g.set_block_ctas(ctas)
    g.set_partition(part.cam_block, part.lm_block, part.S)
    g.set_state(sc.cams, sc.lms)
    prev = g.get_state()
    worst = {"F_blk": 0.0, "cams": 0.0, "lms": 0.0}
    for k in range(iters):
        if k > 0:   # the oracle continues from the GPU's state
            cur = g.get_state()
            Rk, tk, dk, lk = O.to_internal(*cur, prob.s_norm)
            Rp, tp, dp, lp = O.to_internal(*prev, prob.s_norm)
            st = dataclasses.replace(st, R=Rk, t=tk, d=dk, l=lk, Rp=Rp, tp=tp, dp=dp, lp=lp, Fbar=Fb_blk / s2)
            prev = cur
        st, info = B.step(prob, part, st)
        tr = np.zeros(2)
        g.run(1, tr)
        assert tr[0] == pytest.approx(info.F * s2, rel=1e-12), f"iteration {k}"
        F_blk, Fb_blk, rs_blk = g.get_partition_metrics()
        np.testing.assert_allclose(F_blk, info.F_blk * s2, rtol=1e-10, atol=1e-13 * info.F * s2)
        np.testing.assert_allclose(Fb_blk, info.Fbar_blk * s2, rtol=1e-10, atol=1e-13 * info.F * s2)
        tie = np.abs(info.Etest - info.Fbar_blk) <= NEAR_TIE * np.abs(info.F_blk)
        if restart != "block":   # one decision for all blocks
            tie[:] = abs(info.Etest.sum() - info.Fbar_blk.sum()) <= NEAR_TIE * abs(info.F_blk.sum())
            fired += int(info.restart.any())
        assert not ((rs_blk.astype(bool) != info.restart) & ~tie).any(), f"iteration {k}"
        cams_o, lms_o = O.to_boundary(st.R, st.t, st.d, st.l, prob.s_norm)
        cams_g, lms_g = g.get_state()
        # landmarks in the residual space: a landmark that two near-parallel rays fix has a depth
        # the objective hardly sees, and the two solves may place it ~1e-8 apart along the rays
        e_o, e_g = _residuals(prob, cams_o, lms_o), _residuals(prob, cams_g, lms_g)
        rms = np.sqrt(np.mean(np.sum(e_o ** 2, axis=1)))
        worst["F_blk"] = max(worst["F_blk"], float(np.max(np.abs(F_blk / (info.F_blk * s2) - 1))))
        worst["cams"] = max(worst["cams"], float(np.max(np.abs(cams_g - cams_o) / (1 + np.abs(cams_o)))))
        worst["lms"] = max(worst["lms"], float(np.max(np.abs(lms_g - lms_o) / (1 + np.abs(lms_o)))))
        worst["resid"] = max(worst.get("resid", 0.0), float(np.max(np.abs(e_g - e_o)) / rms))
        np.testing.assert_allclose(cams_g, cams_o, rtol=1e-9, atol=1e-9, err_msg=f"iteration {k}")
        assert np.max(np.abs(e_g - e_o)) <= 1e-7 * rms, f"iteration {k}"
        np.testing.assert_allclose(lms_g, lms_o, rtol=1e-6, atol=1e-6, err_msg=f"iteration {k}")
    print(name, n_blocks, worst)
    assert restart == "block" or fired > 0
    g.close()


def test_blocks_run_segments_and_clear():
    """One run of 12 iterations equals 5 + 7; clearing the partition returns to the singleton
    blocks (the default iteration, bit for bit)."""
    from paper_2305_07026_b300 import _lib as L
    sc = _scene("circle_small")
    part = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, sc.M)

    def ctx():
        d = L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec="fp64")
        d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
        return d
    a, b = ctx(), ctx()
    for d in (a, b):
        d.set_partition(part.cam_block, part.lm_block)
        d.set_state(sc.cams, sc.lms)
    ta, tb1, tb2 = np.zeros(13), np.zeros(6), np.zeros(8)
    a.run(12, ta)
    b.run(5, tb1)
    b.run(7, tb2)
    np.testing.assert_array_equal(ta, np.concatenate([tb1[:5], tb2]))
    np.testing.assert_array_equal(a.get_state()[1], b.get_state()[1])
    c, e = ctx(), ctx()
    c.set_partition(part.cam_block, part.lm_block)
    c.set_partition(None)
    for d in (c, e):
        d.set_state(sc.cams, sc.lms)
    tc, te = np.zeros(6), np.zeros(6)
    c.run(5, tc)
    e.run(5, te)
    np.testing.assert_array_equal(tc, te)
    for d in (a, b, c, e):
        d.close()


def test_blocks_arguments():
    from paper_2305_07026_b300 import _lib as L
    with L.Daba(4, 4, 8, prec="fp64") as d:
        for bad in (-1, 17):
            with pytest.raises(L.DabaError) as e:
                d.set_block_ctas(bad)
            assert e.value.status == L.DABA_ERR_ARG
    sc = _scene("circle_small")
    part = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, sc.M)
    m = L.Daba(sc.M, sc.N, sc.nnz, prec="mixed")
    m.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    with pytest.raises(L.DabaError) as e:
        m.set_partition(part.cam_block, part.lm_block)
    assert e.value.status == L.DABA_ERR_ARG
    m.close()
    from paper_2305_07026_b300 import scenes
    big = scenes.circle_scene(n_cams=L.BLK_MAX_CAMS + 100, n_lms=2000, cap=4)
    assert big.M > L.BLK_MAX_CAMS
    with L.Daba(big.M, big.N, big.nnz, prec="fp64") as d:
        d.set_observations(big.cam_idx, big.lm_idx, big.uv)
        with pytest.raises(L.DabaError) as e:   # all cameras in one block: more than BLK_MAX_CAMS
            d.set_partition(np.zeros(big.M, np.int32), np.zeros(big.N, np.int32), 1)
        assert e.value.status == L.DABA_ERR_ARG
    d = L.Daba(sc.M, sc.N, sc.nnz, prec="fp64")
    d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    bad = part.lm_block.copy()
    bad[3] = sc.M
    with pytest.raises(L.DabaError) as e:   # a landmark's block out of range
        d.set_partition(part.cam_block, bad, sc.M)
    assert e.value.status == L.DABA_ERR_ARG
    with pytest.raises(L.DabaError) as e:   # more blocks than cameras and landmarks
        d.set_partition(part.cam_block, part.lm_block, sc.M + sc.N + 1)
    assert e.value.status == L.DABA_ERR_ARG
    d.close()


def test_large_block_cluster_matches_one_cta():
    """A block beyond the oracle's reach (street at a quarter size: 250 cameras and all landmarks
    in one block, a 2250 x 2250 Schur matrix): a cluster of 16 CTAs against one CTA per block (the
    same arithmetic up to the rounding order of the block sums) for 3 iterations, Lemma 1a
    (F^alpha sums to F), and the unaccelerated iteration's monotone objective."""
    from paper_2305_07026_b300 import _lib as L, partition, scenes
    sc = scenes.make_scene("street", scale=0.25)
    cb, lb = partition.camera_groups(sc.M, sc.cam_idx, sc.lm_idx, sc.N, 1)
    out = {}
    for ctas, accel in ((16, True), (1, True), (16, False)):
        with L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec="fp64",
                    accelerated=accel) as d:
            d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
            d.set_block_ctas(ctas)
            d.set_partition(cb, lb)
            d.set_state(sc.cams, sc.lms)
            tr = np.zeros(4)
            d.run(3, tr)
            F_blk, _, _ = d.get_partition_metrics()
            assert F_blk.sum() == pytest.approx(tr[2], rel=1e-11)   # F^alpha(k) of the last iteration
            out[(ctas, accel)] = (tr, d.get_state())
    t16, s16 = out[(16, True)]
    t1, s1 = out[(1, True)]
    np.testing.assert_allclose(t16, t1, rtol=1e-9)
    for a, b in zip(s16, s1):
        np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-6)
    tm = out[(16, False)][0]
    assert np.all(np.diff(tm) < 0.0)


@pytest.mark.parametrize("n_blocks,ctas", [(20, 1), (3, 1), (2, 0)])
def test_blocks_checkpoint_resume(n_blocks, ctas):
    """A checkpoint taken after 5 iterations with a partition (state, Nesterov scalar and the
    per-block E^alpha, Fbar^alpha, F^alpha and restart flags) resumes bit for bit in another
    context with the same partition; a context with another partition, or none, refuses it."""
    from paper_2305_07026_b300 import _lib as L
    sc = _scene("circle_small")
    part = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, n_blocks)

    def ctx(p):
        d = L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec="fp64")
        d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
        d.set_block_ctas(ctas)
        if p is not None:
            d.set_partition(p.cam_block, p.lm_block, p.S)
        d.set_state(sc.cams, sc.lms)
        return d
    a = ctx(part)
    ta = np.zeros(13)
    ra = np.zeros(12, np.int32)
    a.run(5, ta[:6], ra[:5])
    ck = a.export_checkpoint()
    F5, Fb5, rs5 = a.get_partition_metrics()
    t7 = np.zeros(8)
    r7 = np.zeros(7, np.int32)
    a.run(7, t7, r7)
    b = ctx(part)
    b.import_checkpoint(ck)
    F, Fb, rs = b.get_partition_metrics()
    np.testing.assert_array_equal(F, F5)
    np.testing.assert_array_equal(Fb, Fb5)
    np.testing.assert_array_equal(rs, rs5)
    tb = np.zeros(8)
    rb = np.zeros(7, np.int32)
    b.run(7, tb, rb)
    np.testing.assert_array_equal(tb, t7)
    np.testing.assert_array_equal(rb, r7)
    for x, y in zip(a.get_state(), b.get_state()):
        np.testing.assert_array_equal(x, y)
    other = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, 5 if n_blocks != 5 else 4)
    for p in (other, None):
        c = ctx(p)
        with pytest.raises(L.DabaError) as e:
            c.import_checkpoint(ck)
        assert e.value.status == L.DABA_ERR_ARG
        c.close()
    for x in (a, b):
        x.close()


def test_blocks_without_cameras_and_regrown_partition():
    """Landmark-only and empty blocks (n_blocks above the largest id), then a partition with
    larger blocks on the same context (its buffers grow): both against the oracle."""
    from paper_2305_07026_b300 import _lib as L
    sc = _scene("circle_small")
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px)
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    s2 = prob.s_norm ** 2
    g = L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec="fp64")
    g.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    one = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, sc.M)
    lm_only = one.lm_block.copy()
    lm_only[::3] = sc.M + (np.arange(sc.N)[::3] % 4)   # a third of the landmarks in four camera-less blocks
    parts = [(B.Partition(one.cam_block, lm_only, sc.M + 6), 1),   # the last two blocks hold nothing
             (B.Partition(one.cam_block, lm_only, sc.M + 6), 8),   # ... on clusters of 8 CTAs
             (B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, 3), 1),
             (B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, 1), 1),   # global-memory scratch
             (B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, 2), 1)]   # and back to shared memory
    for part, ctas in parts:
        g.set_block_ctas(ctas)
        g.set_partition(part.cam_block, part.lm_block, part.S)
        g.set_state(sc.cams, sc.lms)
        st = B.init_state(prob, part, R, t, d, l)
        for k in range(6):
            st, info = B.step(prob, part, st)
            tr = np.zeros(2)
            g.run(1, tr)
            assert tr[0] == pytest.approx(info.F * s2, rel=1e-10), f"iteration {k}"
            F_blk, Fb_blk, _ = g.get_partition_metrics()
            np.testing.assert_allclose(F_blk, info.F_blk * s2, rtol=1e-9, atol=1e-12 * info.F * s2)
        cams_o, lms_o = O.to_boundary(st.R, st.t, st.d, st.l, prob.s_norm)
        cams_g, lms_g = g.get_state()
        np.testing.assert_allclose(cams_g, cams_o, rtol=1e-8, atol=1e-8)
        np.testing.assert_allclose(lms_g, lms_o, rtol=1e-8, atol=1e-8)
    g.close()
