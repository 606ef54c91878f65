"""A batch of independent scenes run as one problem (scene partition of the C ABI) against
separate runs of each scene: with every camera and landmark a block of its own, scenes share
no term and the Nesterov scalars depend only on k, so the per-block arithmetic is the same
and the iterates agree bit for bit (same pixel_scale); per-scene objectives agree to rounding
of their final sums. Also the oracle's objective for one scene of the batch."""
import numpy as np
import pytest

from oracle import daba_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PIXEL_SCALE = 650.0


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_07026_b300 import build
    build.build()


def _scenes():
    from paper_2305_07026_b300 import scenes
    sizes = [(5, 100), (40, 900), (12, 300), (120, 2500), (7, 150), (60, 1200)]
    return [scenes.small_scene(100 + i, m, n) for i, (m, n) in enumerate(sizes)]


def _ctx(L, M, N, nnz, prec):
    return L.Daba(M, N, nnz, loss="huber", loss_scale_px=1.0, prec=prec, pixel_scale=PIXEL_SCALE)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_separate_runs(prec):
    from paper_2305_07026_b300 import _lib as L
    from paper_2305_07026_b300 import batch
    scs = _scenes()
    b = batch.merge(scs)
    K = 12
    d = _ctx(L, b.M, b.N, b.nnz, prec)
    d.set_observations(b.cam_idx, b.lm_idx, b.uv)
    d.set_state(b.cams, b.lms)
    d.set_scenes(b.cam_begin)
    f0 = d.scene_objectives()
    d.run(K)
    fK = d.scene_objectives()
    cams, lms = d.get_state()
    d.close()
    for i, (sc, (cb, lb)) in enumerate(zip(scs, batch.split(b, cams, lms))):
        e = _ctx(L, sc.M, sc.N, sc.nnz, prec)
        e.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
        e.set_state(sc.cams, sc.lms)
        g0 = e.objective()
        e.run(K)
        gK = e.objective()
        c1, l1 = e.get_state()
        e.close()
        np.testing.assert_array_equal(cb, c1, err_msg=f"scene {i}")
        np.testing.assert_array_equal(lb, l1, err_msg=f"scene {i}")
        assert f0[i] == pytest.approx(g0, rel=1e-12)
        assert fK[i] == pytest.approx(gK, rel=1e-12)


def test_scene_objective_matches_oracle():
    from paper_2305_07026_b300 import _lib as L
    from paper_2305_07026_b300 import batch
    scs = _scenes()
    b = batch.merge(scs)
    d = _ctx(L, b.M, b.N, b.nnz, "fp64")
    d.set_observations(b.cam_idx, b.lm_idx, b.uv)
    d.set_state(b.cams, b.lms)
    d.set_scenes(b.cam_begin)
    f = d.scene_objectives()
    d.close()
    for i, sc in enumerate(scs):
        o = O.Options(loss="huber", loss_scale_px=1.0, pixel_scale=PIXEL_SCALE)
        prob, R, t, dd, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, o)
        F = O.objective(prob.loss, prob.c, R, t, dd, l, prob.cam_idx, prob.lm_idx, prob.u) * prob.s_norm ** 2
        assert f[i] == pytest.approx(F, rel=1e-11), i


def test_scene_partition_is_validated():
    from paper_2305_07026_b300 import _lib as L
    from paper_2305_07026_b300 import batch
    scs = _scenes()[:2]
    b = batch.merge(scs)
    d = _ctx(L, b.M, b.N, b.nnz, "mixed")
    d.set_observations(b.cam_idx, b.lm_idx, b.uv)
    d.set_state(b.cams, b.lms)
    with pytest.raises(L.DabaError) as e:     # scene 0 ends one camera early: its last camera's
        d.set_scenes(np.array([0, b.cam_begin[1] - 1, b.M]))   # landmarks are seen from both sides
    assert e.value.status == L.DABA_ERR_ARG
    with pytest.raises(L.DabaError) as e:
        d.set_scenes(np.array([0, b.M - 1]))
    assert e.value.status == L.DABA_ERR_ARG
    d.set_scenes(b.cam_begin)
    assert d.scene_objectives().shape == (2,)
    d.close()


def test_large_batch_equals_separate_runs():
    """4,400 five-camera scenes (22,000 cameras: more camera-solve CTAs than one wave holds);
    sampled scenes equal their separate runs bit for bit."""
    from paper_2305_07026_b300 import _lib as L
    from paper_2305_07026_b300 import batch, scenes
    scs = [scenes.small_scene(1000 + i, 5, 60) for i in range(4400)]
    b = batch.merge(scs)
    K = 6
    d = _ctx(L, b.M, b.N, b.nnz, "mixed")
    d.set_observations(b.cam_idx, b.lm_idx, b.uv)
    d.set_state(b.cams, b.lms)
    d.set_scenes(b.cam_begin)
    d.run(K)
    cams, lms = d.get_state()
    d.close()
    parts = batch.split(b, cams, lms)
    for i in range(0, len(scs), 440):
        sc = scs[i]
        e = _ctx(L, sc.M, sc.N, sc.nnz, "mixed")
        e.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
        e.set_state(sc.cams, sc.lms)
        e.run(K)
        c1, l1 = e.get_state()
        e.close()
        np.testing.assert_array_equal(parts[i][0], c1, err_msg=f"scene {i}")
        np.testing.assert_array_equal(parts[i][1], l1, err_msg=f"scene {i}")


def test_schedule_changes_only_sum_order():
    """Other chunk and tile sizes give the same iteration up to the order of FP64 sums, and the
    autotuner returns one of its candidates with a time for each schedule it tried."""
    from paper_2305_07026_b300 import _lib as L
    from paper_2305_07026_b300 import autotune
    from tests.conftest import cached_scene
    sc = cached_scene("tourism", scale=0.005)
    traces = []
    for sched in ({}, {"chunk_obs": 96, "tile_obs": 64, "tile_lms": 7}, {"chunk_obs": 4096, "tile_obs": 2048}):
        d = L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec="fp64", **sched)
        d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
        d.set_state(sc.cams, sc.lms)
        tr = np.zeros(11)
        d.run(10, tr)
        d.close()
        traces.append(tr)
    np.testing.assert_allclose(traces[1], traces[0], rtol=1e-10)
    np.testing.assert_allclose(traces[2], traces[0], rtol=1e-10)
    best, tried = autotune.tune(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv,
                                dict(loss=sc.loss, loss_scale_px=sc.loss_scale_px), iters=3)
    assert best["chunk_obs"] in autotune.CHUNKS and best["tile_obs"] in autotune.TILE_OBS
    assert len(tried) >= 6 and all(v > 0 for v in tried.values())
    with pytest.raises(L.DabaError):
        L.Daba(sc.M, sc.N, sc.nnz, tile_lms=129)


@pytest.mark.parametrize("K", [12, 260])
def test_timing_mode_changes_nothing(K):
    """With per-kernel timing on (events recorded inside the run graph, or direct launches for
    runs longer than one graph) a run gives the same bits as without, and positive kernel times."""
    from paper_2305_07026_b300 import _lib as L
    from tests.conftest import cached_scene
    sc = cached_scene("tourism", scale=0.005)
    outs = []
    for timing in (False, True):
        d = L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec="mixed")
        d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
        d.set_state(sc.cams, sc.lms)
        d.set_timing(timing)
        tr = np.zeros(K + 1)
        d.run(K, tr)
        outs.append((tr, *d.get_state(), d.get_timing()))
        d.close()
    for a, b in zip(outs[0][:3], outs[1][:3]):
        np.testing.assert_array_equal(a, b)
    assert np.all(outs[0][3] == 0.0)
    assert np.all(outs[1][3] > 0.0)
