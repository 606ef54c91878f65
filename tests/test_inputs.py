"""The seeded synthetic workloads follow their stated recipes (the inputs of every parity test and
of the bench): observation list invariants, outlier fractions, the circle's geometry, the
tourism tracks' power law and camera degrees, the batch's size distributions, and
reproducibility from the seed. No GPU."""
import numpy as np
import pytest

from paper_2305_07026_b300 import scenes


def _invariants(sc):
    # every landmark seen at least twice, every camera at least once, indices in range
    assert sc.cam_idx.dtype == np.int32 and sc.lm_idx.dtype == np.int32
    assert sc.cam_idx.min() >= 0 and sc.cam_idx.max() < sc.M
    assert sc.lm_idx.min() >= 0 and sc.lm_idx.max() < sc.N
    assert np.bincount(sc.lm_idx, minlength=sc.N).min() >= 2
    assert np.bincount(sc.cam_idx, minlength=sc.M).min() >= 1
    # one observation per (landmark, camera) pair, in (landmark, camera) order
    key = sc.lm_idx.astype(np.int64) * sc.M + sc.cam_idx
    assert np.all(np.diff(key) > 0)
    assert np.all(np.isfinite(sc.uv)) and np.all(np.isfinite(sc.cams)) and np.all(np.isfinite(sc.lms))
    assert sc.cams.shape == (sc.M, 9) and sc.lms.shape == (sc.N, 3) and sc.uv.shape == (sc.nnz, 2)


@pytest.mark.parametrize("workload, scale", [("circle", 1.0), ("street", 0.02), ("tourism", 0.005)])
def test_observation_list_invariants(workload, scale):
    _invariants(scenes.make_scene(workload, scale=scale))


def test_circle_recipe():
    sc = scenes.make_scene("circle")
    assert sc.M == 20 and sc.loss == "huber" and sc.loss_scale_px == 1.0 and sc.iters == 200
    assert 12_000 <= sc.nnz <= 16_000
    centres = sc.cams_gt[:, 3:6]
    np.testing.assert_allclose(np.linalg.norm(centres[:, :2], axis=1), 10.0, rtol=1e-12)
    np.testing.assert_allclose(centres[:, 2], 0.0, atol=1e-12)
    assert np.all(np.abs(sc.lms_gt) <= 2.0)
    assert np.bincount(sc.lm_idx).max() <= 8
    assert sc.outlier_mask.mean() == pytest.approx(0.03, abs=0.5 / sc.nnz)


def test_tourism_recipe():
    sc = scenes.make_scene("tourism", scale=0.02)
    assert sc.loss == "huber" and sc.iters == 100
    ldeg = np.bincount(sc.lm_idx, minlength=sc.N)
    assert ldeg.min() >= 2 and ldeg.max() <= 200
    assert np.bincount(sc.cam_idx, minlength=sc.M).min() >= 20
    assert sc.outlier_mask.mean() == pytest.approx(0.05, abs=0.5 / sc.nnz)


def test_tourism_track_law():
    """The track-length source of the tourism generator is P(L) ~ L^-2.2 on [2, 200] (before the
    site's camera count and visibility cap it; at full size the achieved slope is -2.37)."""
    L = scenes._powerlaw_tracks(np.random.default_rng(0), 2_000_000)
    assert L.min() == 2 and L.max() == 200
    v, cnt = np.unique(L, return_counts=True)
    m = (v >= 4) & (v <= 60)
    slope = np.polyfit(np.log(v[m]), np.log(cnt[m]), 1)[0]
    assert slope == pytest.approx(-2.2, abs=0.05)


def test_batch_recipe():
    scs = scenes.batch_scenes(16)
    for sc in scs:
        _invariants(sc)
        assert 5 <= sc.M <= 200
        assert sc.N <= 20_000
    tl = np.concatenate([np.bincount(sc.lm_idx, minlength=sc.N) for sc in scs])
    assert 3.5 < tl.mean() < 5.0   # geometric tracks of mean 4, at least 2


def test_seeded_reproducibility():
    a, b = scenes.make_scene("tourism", scale=0.005), scenes.make_scene("tourism", scale=0.005)
    for k in ("cams", "lms", "cam_idx", "lm_idx", "uv"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    c = scenes.make_scene("tourism", scale=0.005, seed=3)
    assert c.nnz != a.nnz or not np.array_equal(c.uv, a.uv)
