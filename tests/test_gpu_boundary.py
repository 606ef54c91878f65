"""Failure statuses of daba_run through the C ABI: a bounded wait that runs out
(DABA_ERR_TIMEOUT) and an iterate that becomes non-finite (DABA_ERR_NONFINITE). Both
failures are made on the host: the first by setting the landmark pass's first-wait limit
to zero (every CTA then gives up before polling, lets its copies land and skips its tile),
the second by an observation whose pixel is so large that its ray overflows. In both cases
the call must leave the state exactly as it was (the iterate, s^k, k and the restart
metrics, compared through the checkpoint bytes) and the context must stay usable.
"""
import numpy as np
import pytest

from tests.conftest import cached_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_07026_b300 import build
    build.build()


def _ctx(sc, prec, uv=None):
    from paper_2305_07026_b300 import _lib as L
    d = L.Daba(sc.M, sc.N, sc.nnz, loss=sc.loss, loss_scale_px=sc.loss_scale_px, prec=prec)
    d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv if uv is None else uv)
    d.set_state(sc.cams, sc.lms)
    return d


def _snapshot(d):
    cams, lms = d.get_state()
    m = d.get_block_metrics(landmarks=False)
    return d.export_checkpoint(), cams, lms, m


def _same(a, b):
    assert a[0] == b[0]   # checkpoint: x^k, x^k - x^(k-1), s^k, k, per-block restart slack
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])
    for key in a[3]:
        np.testing.assert_array_equal(a[3][key], b[3][key])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("iters", [1, 4])
def test_timeout_leaves_state_and_context_usable(prec, iters):
    from paper_2305_07026_b300 import _lib as L
    sc = cached_scene("tourism", scale=0.005)
    ref = _ctx(sc, prec)
    tr_ref = np.zeros(7)
    ref.run(3)
    ref.run(6, tr_ref)
    d = _ctx(sc, prec)
    d.run(3)
    before = _snapshot(d)
    d.set_wait_limit(0)
    with pytest.raises(L.DabaError) as e:
        d.run(iters, np.zeros(iters + 1))
    assert e.value.status == L.DABA_ERR_TIMEOUT
    assert "wait" in str(e.value)
    _same(before, _snapshot(d))
    # the default limit again: the run continues as if the failed call had not happened
    d.set_wait_limit(1_000_000_000)
    tr = np.zeros(7)
    d.run(6, tr)
    np.testing.assert_array_equal(tr, tr_ref)
    np.testing.assert_array_equal(d.get_state()[0], ref.get_state()[0])
    np.testing.assert_array_equal(d.get_state()[1], ref.get_state()[1])
    d.close()
    ref.close()


def test_wait_limit_argument():
    from paper_2305_07026_b300 import _lib as L
    sc = cached_scene("circle")
    d = _ctx(sc, "fp64")
    with pytest.raises(L.DabaError) as e:
        d.set_wait_limit(-1)
    assert e.value.status == L.DABA_ERR_ARG
    d.set_wait_limit(5_000_000)   # 5 ms is ample for a tile's copies
    d.run(2)
    d.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("iters", [1, 5])
def test_nonfinite_iterate_leaves_state(prec, iters):
    """One pixel of 1e150 px passes the finiteness check of the input, but the ray of Eq. ray
    overflows (|u|^4 in its third component), so F_ij, the iterate and the objective become
    non-finite in the first iteration. The failed run restores its entry state; with the pixel
    replaced, the context runs on as a fresh one."""
    from paper_2305_07026_b300 import _lib as L
    sc = cached_scene("circle")
    uv = sc.uv.copy()
    uv[17] = (1e150, -3e149)
    d = _ctx(sc, prec, uv=uv)
    before = _snapshot(d)
    with pytest.raises(L.DabaError) as e:
        d.run(iters, np.zeros(iters + 1))
    assert e.value.status == L.DABA_ERR_NONFINITE
    _same(before, _snapshot(d))
    d.set_pixels(sc.uv)
    tr = np.zeros(5)
    d.run(4, tr)
    ref = _ctx(sc, prec)
    tr_ref = np.zeros(5)
    ref.run(4, tr_ref)
    np.testing.assert_array_equal(tr, tr_ref)
    np.testing.assert_array_equal(d.get_state()[1], ref.get_state()[1])
    d.close()
    ref.close()


def test_device_bytes_count_the_context_buffers():
    """daba_device_bytes: the buffers a context allocates are at least the observation arrays
    and both landmark buffers, the device's free memory falls by at least that much when they
    are allocated, daba_run allocates nothing, a coarse-block partition and the reverse mode
    add their buffers, and the peak never falls below what is held."""
    from paper_2305_07026_b300 import _lib as L
    from paper_2305_07026_b300 import partition
    import gc
    sc = cached_scene("street", scale=0.2)
    gc.collect()   # no earlier context is freed by a finalizer between the two readings below
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    d = _ctx(sc, "fp64")
    try:
        b0, p0 = d.device_bytes()
        free1 = torch.cuda.mem_get_info()[0]
        # per observation at least its landmark index and pixel; per landmark two FP64 records
        assert b0 >= sc.nnz * (4 + 16) + sc.N * 2 * 3 * 8
        assert free0 - free1 >= b0
        assert p0 == b0
        d.run(12)
        assert d.device_bytes() == (b0, p0)
        cb, lb = partition.camera_groups(sc.M, sc.cam_idx, sc.lm_idx, sc.N, (sc.M + 7) // 8)
        d.set_partition(cb, lb)
        b1, p1 = d.device_bytes()
        assert b1 > b0 and p1 >= b1
        d.set_partition(None)   # the block buffers stay for the next partition
        rng = np.random.default_rng(0)
        d.set_state(sc.cams, sc.lms)   # the reverse mode starts from a state just set
        d.unrolled_grad(10, rng.normal(size=(sc.M, 9)), rng.normal(size=(sc.N, 3)))
        b2, p2 = d.device_bytes()
        assert b2 > b1 and p2 == max(p1, b2)
    finally:
        d.close()
    assert L.daba_device_bytes(None, None, None) == L.DABA_ERR_ARG
