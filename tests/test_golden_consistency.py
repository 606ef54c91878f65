"""The stored oracle results that the GPU tests compare with (tests/golden/street_oracle_*.json,
written by tests/golden/make_street_golden.py) are still what the oracle computes: the scene they
name is the one the seeded generator builds now, and the first iterations of the oracle on it
reproduce the stored objective trace and restart counts (at full size, F(x^0) only). Guards against the oracle, the
generator or the stored file drifting apart. No GPU."""
import json
import os

import numpy as np
import pytest

from oracle import daba_oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name,iters", [("street_oracle_0.2.json", 4), ("street_oracle_1.json", 0)])
def test_stored_oracle_results_reproduce(name, iters):
    from paper_2305_07026_b300 import scenes
    g = json.load(open(os.path.join(GOLDEN, name)))
    w = g["workload"]
    sc = scenes.make_scene(w["name"], scale=w["scale"])
    assert (sc.M, sc.N, sc.nnz, sc.seed, sc.loss, sc.loss_scale_px) == (
        w["M"], w["N"], w["nnz"], w["seed"], w["loss"], w["loss_scale_px"])
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, xi=w["xi"], eta=w["eta"])
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    s2 = prob.s_norm ** 2
    F0 = O.objective(prob.loss, prob.c, R, t, d, l, prob.cam_idx, prob.lm_idx, prob.u) * s2
    assert F0 == pytest.approx(g["trace_px2"][0], rel=1e-13)
    st = O.init_state(prob, R, t, d, l)
    for k in range(iters):
        st, info = O.step(prob, st)
        assert info.F * s2 == pytest.approx(g["trace_px2"][k], rel=1e-13), k
        assert int(info.restart_cam.sum() + info.restart_lm.sum()) == g["restarts"][k], k
    assert len(g["trace_px2"]) == g["iters"] + 1 and np.all(np.diff(g["trace_px2"][:iters + 1]) < 0)
