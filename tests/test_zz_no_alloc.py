"""daba_objective_noalloc, the entry point for callers that cannot allocate device memory,
against the library's regular objective entry point (daba_objective through a context).

This file is collected last so that a run stopping at the first failure has already run
every other test. It passes both alone in a fresh process and after the other tests.
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


def _regular(sc, loss, scale):
    from paper_2305_07026_b300 import _lib as L
    with L.Daba(sc.M, sc.N, sc.nnz, loss=loss, loss_scale_px=scale, prec="fp64") as d:
        d.set_observations(sc.cam_idx, sc.lm_idx, sc.uv)
        d.set_state(sc.cams, sc.lms)
        return d.objective()


def _noalloc(sc, loss, scale, pixel_scale):
    from paper_2305_07026_b300 import _lib as L
    dev = "cuda"
    args = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv)]
    out = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    st = L.daba_objective_noalloc(sc.M, sc.N, sc.nnz, *[L.ptr(a) for a in args], L.LOSSES[loss], scale, pixel_scale,
                                  L.ptr(out), L.current_stream())
    assert st == L.DABA_OK
    torch.cuda.synchronize()
    return out.item()


@pytest.mark.parametrize("workload,scale,loss,c", [("circle", 1.0, "huber", 1.0), ("tourism", 0.01, "cauchy", 2.0)])
def test_noalloc_matches_regular_objective_twice(workload, scale, loss, c):
    sc = cached_scene(workload, scale=scale)
    ref = _regular(sc, loss, c)
    s = float(np.median(sc.cams[:, 6]))
    first = _noalloc(sc, loss, c, s)
    second = _noalloc(sc, loss, c, s)
    assert first == pytest.approx(ref, rel=1e-12)
    assert second == pytest.approx(ref, rel=1e-12)


def test_noalloc_rejects_what_it_cannot_hold():
    from paper_2305_07026_b300 import _lib as L
    sc = cached_scene("circle")
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv)]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = [L.ptr(a) for a in dev]
    # more cameras than the static scratch holds
    assert L.daba_objective_noalloc(20000, sc.N, sc.nnz, *p, 1, 1.0, 600.0, L.ptr(out), 0) == L.DABA_ERR_ARG
    # host memory is not accepted (nothing is staged)
    assert L.daba_objective_noalloc(sc.M, sc.N, sc.nnz, L.ptr(sc.cams), *p[1:], 1, 1.0, 600.0, L.ptr(out),
                                    0) == L.DABA_ERR_ARG
    # an out-of-range index yields NaN, not a fault
    bad = dev[2].clone()
    bad[7] = sc.M + 3
    st = L.daba_objective_noalloc(sc.M, sc.N, sc.nnz, p[0], p[1], L.ptr(bad), p[3], p[4], 1, 1.0, 600.0, L.ptr(out), 0)
    assert st == L.DABA_OK
    torch.cuda.synchronize()
    assert np.isnan(out.item())
