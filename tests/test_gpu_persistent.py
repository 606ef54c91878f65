"""The persistent path (daba_set_persistent: a run's iterations as one cooperative launch with
grid barriers) against the default path (CUDA graphs of the separate kernels) through the C ABI:
the objective trace, restart counts, per-block metrics and iterate must be the same bits, on a
single scene and on a batch of scenes run as one problem; the batch's scenes are also compared
with the oracle run on each scene alone."""
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


def _run(prob, K, persistent, scenes_begin=None, **opts):
    from paper_2305_07026_b300 import _lib as L
    cams, lms, ci, li, uv = prob
    d = L.Daba(cams.shape[0], lms.shape[0], ci.size, prec="mixed", **opts)
    d.set_observations(ci, li, uv)
    if scenes_begin is not None:
        d.set_scenes(scenes_begin)
    d.set_state(cams, lms)
    d.set_persistent(persistent)
    tr, rs = np.zeros(K + 1), np.zeros(K, np.int32)
    d.run(K, tr, rs)
    # a second run continues from the first (start parity, first-iteration flag, Nesterov s)
    tr2 = np.zeros(K + 1)
    d.run(K, tr2)
    c, l = d.get_state()
    m = d.get_block_metrics(landmarks=False)
    f = d.scene_objectives() if scenes_begin is not None else None
    d.close()
    return tr, rs, tr2, c, l, m, f


def _same(a, b):
    tr, rs, tr2, c, l, m, f = a
    tr_, rs_, tr2_, c_, l_, m_, f_ = b
    np.testing.assert_array_equal(tr, tr_)
    np.testing.assert_array_equal(rs, rs_)
    np.testing.assert_array_equal(tr2, tr2_)
    np.testing.assert_array_equal(c, c_)
    np.testing.assert_array_equal(l, l_)
    for k in m:
        np.testing.assert_array_equal(m[k], m_[k])
    if f is not None:
        np.testing.assert_array_equal(f, f_)


@pytest.mark.parametrize("workload,scale,K", [("circle", 1.0, 12), ("tourism", 0.005, 9), ("street", 0.05, 13)])
def test_persistent_equals_graph_path(workload, scale, K):
    sc = cached_scene(workload, scale=scale)
    prob = (sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv)
    kw = dict(loss=sc.loss, loss_scale_px=sc.loss_scale_px)
    _same(_run(prob, K, False, **kw), _run(prob, K, True, **kw))
    # DUBA, and a schedule with small tiles and chunks (many CTAs' items per phase)
    _same(_run(prob, K, False, accelerated=False, **kw), _run(prob, K, True, accelerated=False, **kw))
    small = dict(chunk_obs=256, tile_obs=64, tile_lms=16)
    _same(_run(prob, K, False, **small, **kw), _run(prob, K, True, **small, **kw))


def test_persistent_long_tracks():
    """Tracks longer than a small tile take the one-landmark tiles inside the persistent launch."""
    from tests.test_gpu_parity import _long_track_scene
    sc, ci, li, uv = _long_track_scene()
    prob = (sc.cams, sc.lms, ci, li, uv)
    _same(_run(prob, 6, False, loss=sc.loss, loss_scale_px=sc.loss_scale_px),
          _run(prob, 6, True, loss=sc.loss, loss_scale_px=sc.loss_scale_px))


def test_persistent_batch_equals_graph_and_oracle():
    from paper_2305_07026_b300 import batch, scenes
    scs = scenes.batch_scenes(48)
    b = batch.merge(scs)
    prob = (b.cams, b.lms, b.cam_idx, b.lm_idx, b.uv)
    kw = dict(loss="huber", loss_scale_px=1.0, pixel_scale=650.0)
    K = 12
    g = _run(prob, K, False, scenes_begin=b.cam_begin, **kw)
    p = _run(prob, K, True, scenes_begin=b.cam_begin, **kw)
    _same(g, p)
    # each scene's objective after the first K iterations against the oracle on that scene alone
    from paper_2305_07026_b300 import _lib as L
    d = L.Daba(b.M, b.N, b.nnz, prec="mixed", **kw)
    d.set_observations(b.cam_idx, b.lm_idx, b.uv)
    d.set_scenes(b.cam_begin)
    d.set_state(b.cams, b.lms)
    d.set_persistent(True)
    d.run(K)
    fK = d.scene_objectives()
    d.close()
    sizes = np.array([sc.nnz for sc in scs])
    for i in [int(np.argmin(sizes)), int(np.argmax(sizes)), 7, 23]:
        sc = scs[i]
        res = O.daba(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv,
                     O.Options(loss="huber", loss_scale_px=1.0, pixel_scale=650.0), K)
        assert fK[i] == pytest.approx(res.trace_px2[-1], rel=1e-4), f"scene {i}"


def test_persistent_rejects_unsupported_contexts():
    from paper_2305_07026_b300 import _lib as L
    sc = cached_scene("circle")
    for kw in (dict(prec="fp64"), dict(prec="mixed", restart="global"), dict(prec="mixed", cam_solver="lm")):
        d = L.Daba(sc.M, sc.N, sc.nnz, **kw)
        with pytest.raises(L.DabaError) as e:
            d.set_persistent(True)
        assert e.value.status == L.DABA_ERR_ARG
        d.close()
