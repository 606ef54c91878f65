"""Coarse blocks on the GPU (daba_set_partition: contiguous groups of one to eight cameras and
the landmarks they see first, Eq. Ealpha with the intra-block pairs exact, one successful LM step
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


def _scene(name):
    from paper_2305_07026_b300 import scenes
    if name == "circle":
        return cached_scene("circle")
    if name == "circle_small":
        return scenes.circle_scene(n_lms=300)
    return cached_scene(name, scale={"street": 0.05, "tourism": 0.005}[name])


@pytest.mark.parametrize("name,accel,K,n_blocks", [
    ("circle", True, 20, None), ("circle_small", False, 12, None), ("street", True, 12, None),
    ("tourism", True, 10, None),
    # several cameras per block: the Schur complement couples the block's cameras
    ("circle", True, 12, 4), ("circle_small", False, 12, 3), ("circle_small", True, 12, 6),
    ("street", True, 4, 25), ("tourism", True, 3, 30)])
def test_blocks_match_oracle_per_iteration(name, accel, K, n_blocks):
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
    assert compared >= min(K, 3 if n_blocks else 10)
    if compared == K:
        cams_o, lms_o = O.to_boundary(st.R, st.t, st.d, st.l, prob.s_norm)
        cams_g, lms_g = g.get_state()
        np.testing.assert_allclose(cams_g, cams_o, rtol=1e-8, atol=1e-8)
        np.testing.assert_allclose(lms_g, lms_o, rtol=1e-8, atol=1e-8)
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
    sc = _scene("circle_small")
    part = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, sc.M)
    m = L.Daba(sc.M, sc.N, sc.nnz, prec="mixed")
    m.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    with pytest.raises(L.DabaError) as e:
        m.set_partition(part.cam_block, part.lm_block)
    assert e.value.status == L.DABA_ERR_ARG
    m.close()
    d = L.Daba(sc.M, sc.N, sc.nnz, prec="fp64")
    d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    with pytest.raises(L.DabaError) as e:   # all cameras in one block: more than BLK_MAX_CAMS
        d.set_partition(np.zeros(sc.M, np.int32), part.lm_block)
    assert e.value.status == L.DABA_ERR_ARG
    bad = part.lm_block.copy()
    bad[3] = sc.M
    with pytest.raises(L.DabaError) as e:   # a landmark's block out of range
        d.set_partition(part.cam_block, bad, sc.M)
    assert e.value.status == L.DABA_ERR_ARG
    with pytest.raises(L.DabaError) as e:   # more blocks than cameras and landmarks
        d.set_partition(part.cam_block, part.lm_block, sc.M + sc.N + 1)
    assert e.value.status == L.DABA_ERR_ARG
    d.set_partition(part.cam_block, part.lm_block)
    d.set_state(sc.cams, sc.lms)
    with pytest.raises(L.DabaError) as e:
        d.export_checkpoint()
    assert e.value.status == L.DABA_ERR_STATE
    d.close()


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
    parts = [B.Partition(one.cam_block, lm_only, sc.M + 6),   # the last two blocks hold nothing
             B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, 3)]
    for part in parts:
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
