"""The range schedule (daba_set_pipeline) against the one-range iteration through the C ABI.

Camera ranges only change which kernels run beside one another: every camera solve and landmark
tile still reads the camera-pass chunks it read before, in the same order. So the objective trace,
restart counts, per-block metrics and iterate must be the same bits for every number of ranges,
grid bound and priority order, on single scenes (FP64 and MIXED, every loss), on a batch of
scenes, across the 8-iteration graphs of long runs, and on a run that fails and restores its entry
state."""
import numpy as np
import pytest

from tests.conftest import cached_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ONE = (1, 0, 0, (1, 0, 1))
CUTS = [
    (2, 0, 0, (1, 0, 1)),          # the default for large problems
    (3, 0, 0, (1, 0, 0)),
    (4, 4, 2, (2, 1, 0)),          # both bounded grids
    (64, 0, 3, (0, 2, 2)),         # more ranges than small scenes have cameras to cut at
    (9, 8, 0, (0, 0, 0)),
]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_07026_b300 import build
    build.build()


def _run(sc, K, pipe, prec="mixed", scenes_begin=None, loss=None, **opts):
    from paper_2305_07026_b300 import _lib as L
    d = L.Daba(sc.M, sc.N, sc.nnz, loss=loss or sc.loss, loss_scale_px=sc.loss_scale_px, prec=prec, **opts)
    d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    if scenes_begin is not None:
        d.set_scenes(scenes_begin)
    d.set_pipeline(*pipe)
    d.set_state(sc.cams, sc.lms)
    tr, rs = np.zeros(K + 1), np.zeros(K, np.int32)
    d.run(K, tr, rs)
    tr2 = np.zeros(4)   # a second run continues from the first
    d.run(3, tr2)
    c, l = d.get_state()
    m = d.get_block_metrics(landmarks=prec == "fp64")
    f = d.scene_objectives() if scenes_begin is not None else None
    d.close()
    return tr, rs, tr2, c, l, m, f


def _same(a, b):
    for x, y in zip(a[:5], b[:5]):
        np.testing.assert_array_equal(x, y)
    for k in a[5]:
        np.testing.assert_array_equal(a[5][k], b[5][k], err_msg=k)
    if a[6] is not None:
        np.testing.assert_array_equal(a[6], b[6])


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("workload,scale,K", [("tourism", 0.005, 20), ("street", 0.05, 14), ("circle", 1.0, 10)])
def test_cut_gives_the_same_bits(workload, scale, K, prec):
    sc = cached_scene(workload, scale=scale)
    ref = _run(sc, K, ONE, prec)
    if workload == "tourism":
        assert ref[1].sum() > 0   # restarts happen, so the restart decisions are compared too
    for pipe in CUTS:
        _same(_run(sc, K, pipe, prec), ref)


@pytest.mark.parametrize("loss", ["trivial", "cauchy", "welsch"])
def test_cut_other_losses(loss):
    sc = cached_scene("tourism", scale=0.005)
    _same(_run(sc, 8, CUTS[0], loss=loss), _run(sc, 8, ONE, loss=loss))


def test_cut_batch_of_scenes():
    from paper_2305_07026_b300 import batch as B
    from paper_2305_07026_b300.scenes import batch_scenes
    b = B.merge(batch_scenes(n_scenes=24, seed=11))
    ref = _run(b_as_scene(b), 10, ONE, scenes_begin=b.cam_begin, pixel_scale=650.0)
    for pipe in CUTS[:3]:
        _same(_run(b_as_scene(b), 10, pipe, scenes_begin=b.cam_begin, pixel_scale=650.0), ref)


def b_as_scene(b):
    class S:
        pass
    s = S()
    s.M, s.N, s.nnz = b.M, b.N, b.nnz
    s.cams, s.lms, s.cam_idx, s.lm_idx, s.uv = b.cams, b.lms, b.cam_idx, b.lm_idx, b.uv
    s.loss, s.loss_scale_px = "huber", 1.0
    return s


def test_cut_long_run_graphs():
    """Runs longer than one run graph use the 8-iteration graphs; the cut applies there too."""
    sc = cached_scene("circle")
    _same(_run(sc, 261, CUTS[0]), _run(sc, 261, ONE))


def test_cut_with_timing_and_failure():
    """Per-kernel timing runs the one-range iteration (same bits); a run whose landmark-pass waits
    all run out fails with DABA_ERR_TIMEOUT and leaves the state of before the call."""
    from paper_2305_07026_b300 import _lib as L
    sc = cached_scene("tourism", scale=0.005)
    ref = _run(sc, 6, ONE)
    d = L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec="mixed")
    d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    d.set_pipeline(*CUTS[0])
    d.set_timing(True)
    d.set_state(sc.cams, sc.lms)
    tr = np.zeros(7)
    d.run(6, tr)
    np.testing.assert_array_equal(tr, ref[0][:7])
    assert all(t > 0 for t in d.get_timing()[1:])
    d.set_timing(False)
    c0, l0 = d.get_state()
    d.set_wait_limit(0)
    with pytest.raises(L.DabaError) as e:
        d.run(5)
    assert e.value.status == L.DABA_ERR_TIMEOUT
    c1, l1 = d.get_state()
    np.testing.assert_array_equal(c0, c1)
    np.testing.assert_array_equal(l0, l1)
    d.set_wait_limit(1_000_000_000)
    d.run(2)   # the context stays usable
    d.close()


def test_pipeline_argument_checks():
    from paper_2305_07026_b300 import _lib as L
    sc = cached_scene("circle")
    d = L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px)
    for bad in [(0, 0, 0, ONE[3]), (65, 0, 0, ONE[3]), (2, 65, 0, ONE[3]), (2, 0, -1, ONE[3]),
                (2, 0, 0, (0, 0, 3)), (2, 0, 0, (0, -1, 0))]:
        with pytest.raises(L.DabaError) as e:
            d.set_pipeline(*bad)
        assert e.value.status == L.DABA_ERR_ARG
    d.set_pipeline(2)   # before the observations: the ranges are cut when they come
    d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
    d.set_state(sc.cams, sc.lms)
    d.run(3)
    d.close()
