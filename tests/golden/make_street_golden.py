"""Writes the oracle's results on the street workload (1,000 cameras on a 1 km street grid,
200k facade landmarks, about 1M observations, Cauchy loss 2 px, 300 iterations of Algorithm 1)
to tests/golden/street_oracle_<scale>.json, for the GPU tests that compare the CUDA path with
the oracle at the full size of this workload.

Only oracle/ computes here: the scene comes from the seeded generator (no arithmetic of the
method), every stored value from oracle.daba_oracle. The full-size run takes about 40 minutes
on one core; `--scale 0.2` (200 cameras, ~150k observations) about 5 minutes.

Stored: the objective trace F(x^0) .. F(x^300) in pixel^2, the number of restarted blocks per
iteration, the smallest restart-test margin |E^alpha(k+1) - Fbar^alpha(k)| / |F^alpha(k)| of
each iteration (a margin near 1e-12 marks a near-tie, where two correct FP64 evaluation orders
may decide differently), and the boundary parameters of 24 seeded cameras and 400 seeded
landmarks after 20 iterations and after the last one.

Usage: python tests/golden/make_street_golden.py [--scale 1.0] [--iters 300]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import daba_oracle as O  # noqa: E402
from paper_2305_07026_b300 import scenes  # noqa: E402


def sample_ids(M, N, seed=11):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(M, min(24, M), replace=False)), np.sort(rng.choice(N, min(400, N), replace=False))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    sc = scenes.make_scene("street", scale=a.scale)
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px)
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    st = O.init_state(prob, R, t, d, l)
    cs, ls = sample_ids(sc.M, sc.N)
    s2 = prob.s_norm ** 2
    trace, restarts, margins, at20 = [], [], [], None
    t0 = time.time()
    for k in range(a.iters):
        st, info = O.step(prob, st)
        trace.append(info.F * s2)
        restarts.append(int(info.restart_cam.sum() + info.restart_lm.sum()))
        mc = np.abs(info.Etest_cam - info.Fbar_cam) / np.maximum(np.abs(info.F_cam), 1e-300)
        ml = np.abs(info.Etest_lm - info.Fbar_lm) / np.maximum(np.abs(info.F_lm), 1e-300)
        margins.append(float(min(mc.min(), ml.min())))
        if k + 1 == 20:
            cams_b, lms_b = O.to_boundary(st.R, st.t, st.d, st.l, prob.s_norm)
            at20 = {"cams": cams_b[cs].tolist(), "lms": lms_b[ls].tolist()}
        if (k + 1) % 25 == 0:
            print(f"iteration {k + 1}: F = {trace[-1]:.10e}  ({time.time() - t0:.0f} s)", flush=True)
    trace.append(O.objective(prob.loss, prob.c, st.R, st.t, st.d, st.l, prob.cam_idx, prob.lm_idx, prob.u) * s2)
    cams_b, lms_b = O.to_boundary(st.R, st.t, st.d, st.l, prob.s_norm)
    out = {
        "what": "oracle (oracle/daba_oracle.py, FP64) on the street workload, Algorithm 1 with singleton blocks",
        "written_by": "tests/golden/make_street_golden.py",
        "workload": {"name": sc.name, "scale": a.scale, "seed": sc.seed, "M": sc.M, "N": sc.N, "nnz": sc.nnz,
                     "loss": sc.loss, "loss_scale_px": sc.loss_scale_px, "xi": opts.xi, "eta": opts.eta},
        "iters": a.iters,
        "trace_px2": trace,
        "restarts": restarts,
        "min_restart_margin": margins,
        "sample_cams": cs.tolist(),
        "sample_lms": ls.tolist(),
        "at_20": at20,
        "final": {"cams": cams_b[cs].tolist(), "lms": lms_b[ls].tolist()},
        "oracle_seconds": time.time() - t0,
    }
    path = a.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), f"street_oracle_{a.scale:g}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print(path)


if __name__ == "__main__":
    main()
