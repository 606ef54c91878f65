"""Host-side logic that needs no GPU: option validation in daba_create (before any device
call), the batch merge/split of independent scenes, the autotuner's coordinate descent and the
coarse-block partition helper."""
import numpy as np
import pytest


@pytest.mark.parametrize("bad", [dict(restart=7), dict(restart="block", momentum_reset=True), dict(cam_solver=5),
                                 dict(chunk_obs=16), dict(tile_obs=4096), dict(tile_lms=200), dict(eta=0.0),
                                 dict(eta=1.5), dict(xi=0.0), dict(cam_alternations=0), dict(prec=3),
                                 dict(loss=9), dict(loss="huber", loss_scale_px=0.0)])
def test_invalid_options_rejected_before_device_work(bad):
    from paper_2305_07026_b300 import build
    build.build()
    from paper_2305_07026_b300 import _lib as L
    with pytest.raises(L.DabaError) as e:
        L.Daba(4, 4, 8, **bad)
    assert e.value.status == L.DABA_ERR_ARG


def test_variant_option_values():
    from paper_2305_07026_b300 import _lib as L
    o = L.options(restart="global", momentum_reset=True, cam_solver="lm")
    assert (o.restart_mode, o.momentum_reset, o.cam_solver) == (1, 1, 1)
    o = L.options()
    assert (o.restart_mode, o.momentum_reset, o.cam_solver) == (0, 0, 0)


def test_batch_merge_split_round_trip():
    from paper_2305_07026_b300 import batch, scenes
    scs = scenes.batch_scenes(7)
    b = batch.merge(scs)
    assert b.M == sum(s.cams.shape[0] for s in scs) and b.N == sum(s.lms.shape[0] for s in scs)
    assert b.nnz == sum(s.cam_idx.size for s in scs)
    for i, s in enumerate(scs):
        o0, o1 = b.obs_begin[i], b.obs_begin[i + 1]
        np.testing.assert_array_equal(b.cam_idx[o0:o1] - b.cam_begin[i], s.cam_idx)
        np.testing.assert_array_equal(b.lm_idx[o0:o1] - b.lm_begin[i], s.lm_idx)
        np.testing.assert_array_equal(b.uv[o0:o1], s.uv)
        # every observation of scene i refers to scene i's cameras and landmarks only
        assert b.cam_idx[o0:o1].min() >= b.cam_begin[i] and b.cam_idx[o0:o1].max() < b.cam_begin[i + 1]
        assert b.lm_idx[o0:o1].min() >= b.lm_begin[i] and b.lm_idx[o0:o1].max() < b.lm_begin[i + 1]
    parts = batch.split(b, b.cams, b.lms)
    for (c, l), s in zip(parts, scs):
        np.testing.assert_array_equal(c, s.cams)
        np.testing.assert_array_equal(l, s.lms)


def test_autotune_coordinate_descent(monkeypatch):
    """The tuner walks chunk, then observations per tile, then landmarks per tile, then the
    number of camera ranges, keeping the best of each and timing every schedule once."""
    from paper_2305_07026_b300 import autotune
    cost = {}

    def fake(L, cams, lms, cam_idx, lm_idx, uv, opts, sched, iters=8, warmup=2, repeats=1):
        key = (sched["chunk_obs"], sched["tile_obs"], sched["tile_lms"], sched["ranges"])
        cost[key] = cost.get(key, 0) + 1
        return abs(key[0] - 4096) / 1e3 + abs(key[1] - 256) / 1e2 + abs(key[2] - 64) / 10.0 + abs(key[3] - 4)
    monkeypatch.setattr(autotune, "time_schedule", fake)
    z = np.zeros((1, 9))
    best, tried = autotune.tune(z, np.zeros((1, 3)), np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros((1, 2)))
    assert best == {"chunk_obs": 4096, "tile_obs": 256, "tile_lms": 64, "ranges": 4}
    assert all(v == 1 for v in cost.values())
    assert len(tried) == len(cost)


def test_autotune_sweeps_until_no_axis_changes(monkeypatch):
    """Interacting axes: the best chunk depends on the number of ranges, which the first sweep
    settles last. A second sweep moves the chunk, a third changes nothing and ends the search;
    the result is the grid's optimum and no schedule is timed twice."""
    from paper_2305_07026_b300 import autotune
    cost = {}

    def fake(L, cams, lms, cam_idx, lm_idx, uv, opts, sched, iters=8, warmup=2, repeats=1):
        key = (sched["chunk_obs"], sched["tile_obs"], sched["tile_lms"], sched["ranges"])
        cost[key] = cost.get(key, 0) + 1
        want_chunk = 2048 if key[3] < 4 else 4096
        return abs(key[3] - 4) + abs(key[0] - want_chunk) / 1e4 + abs(key[1] - 512) / 1e5 + abs(key[2] - 128) / 1e5
    monkeypatch.setattr(autotune, "time_schedule", fake)
    z = np.zeros((1, 9))
    args = (z, np.zeros((1, 3)), np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros((1, 2)))
    best, tried = autotune.tune(*args)
    assert best == {"chunk_obs": 4096, "tile_obs": 512, "tile_lms": 128, "ranges": 4}
    assert all(v == 1 for v in cost.values()) and len(tried) == len(cost)
    cost.clear()
    one, _ = autotune.tune(*args, max_sweeps=1)   # a single sweep stops at the first chunk
    assert one == {"chunk_obs": 2048, "tile_obs": 512, "tile_lms": 128, "ranges": 4}


def test_autotune_context_takes_the_cut(monkeypatch):
    """A schedule's camera ranges go to daba_set_pipeline, its sizes to the context options."""
    from paper_2305_07026_b300 import autotune
    calls = []

    class FakeDaba:
        def __init__(self, M, N, nnz, **kw):
            calls.append(("create", kw))

        def set_pipeline(self, ranges):
            calls.append(("pipeline", ranges))

    class FakeL:
        Daba = FakeDaba
    autotune.make_context(FakeL, 1, 1, 1, {"prec": "mixed"}, {"chunk_obs": 1024, "ranges": 4})
    assert calls == [("create", {"prec": "mixed", "chunk_obs": 1024}), ("pipeline", 4)]
    calls.clear()
    autotune.make_context(FakeL, 1, 1, 1, {}, {})
    assert calls == [("create", {})]


def test_camera_group_partition_helper():
    """The package's partition helper gives the blocks the block oracle's helper gives, and
    refuses blocks of more cameras than the library takes."""
    import numpy as np
    from oracle import daba_blocks as B
    from paper_2305_07026_b300 import partition, scenes
    sc = scenes.circle_scene(n_lms=300)
    for n in (1, 2, 3, 4, 20):
        cb, lb = partition.camera_groups(sc.M, sc.cam_idx, sc.lm_idx, sc.N, n)
        ref = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, n)
        np.testing.assert_array_equal(cb, ref.cam_block)
        np.testing.assert_array_equal(lb, ref.lm_block)
    big = scenes.circle_scene(n_cams=1100, n_lms=2000, cap=4)
    assert big.M > 2 * partition.BLK_MAX_CAMS
    partition.camera_groups(big.M, big.cam_idx, big.lm_idx, big.N, 3)   # at most 512 cameras per block
    with pytest.raises(ValueError):
        partition.camera_groups(big.M, big.cam_idx, big.lm_idx, big.N, 2)   # more than 512
