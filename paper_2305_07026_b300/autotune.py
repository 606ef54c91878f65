"""Schedule autotuner: picks the camera-pass chunk size, the landmark-tile sizes and the cut of
the range schedule (daba_set_pipeline: camera ranges per iteration) of a problem by timing a few
iterations of each candidate on the GPU (coordinate descent: chunk, then observations per tile,
then landmarks per tile, then the ranges). The schedule changes only how the work is cut into warps and CTAs and
ordered on the GPU, not the method (results differ at most in the order of FP sums).
"""
from __future__ import annotations

import numpy as np

CHUNKS = (1024, 2048, 4096)
TILE_OBS = (256, 512, 1024)
TILE_LMS = (64, 128)
RANGES = (1, 2, 4, 6)
OPTION_KEYS = ("chunk_obs", "tile_obs", "tile_lms")


def make_context(L, M, N, nnz, opts, sched):
    """A context with the schedule's options, and its two-range cut when the schedule has one."""
    d = L.Daba(M, N, nnz, **opts, **{k: v for k, v in sched.items() if k in OPTION_KEYS})
    if "ranges" in sched:
        d.set_pipeline(sched["ranges"])
    return d


def time_schedule(L, cams, lms, cam_idx, lm_idx, uv, opts, sched, iters=8, warmup=2):
    """Milliseconds per iteration of one schedule (CUDA events around ``iters`` iterations)."""
    import torch
    d = make_context(L, cams.shape[0], lms.shape[0], cam_idx.size, opts, sched)
    try:
        d.set_observations(cam_idx, lm_idx, uv)
        d.set_state(cams, lms)
        d.run(max(warmup, iters))   # a warm-up of the timed length captures its graph
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        d.run(iters)
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / iters
    finally:
        d.close()


def tune(cams, lms, cam_idx, lm_idx, uv, opts=None, iters=8, log=None):
    """Returns (best schedule dict, {schedule: ms per iteration}) for this problem."""
    from paper_2305_07026_b300 import _lib as L
    opts = dict(opts or {})
    best = {"chunk_obs": 2048, "tile_obs": 512, "tile_lms": 128, "ranges": 2 if cam_idx.size >= 1 << 20 else 1}
    seen = {}

    def measure(s):
        key = (s["chunk_obs"], s["tile_obs"], s["tile_lms"], s["ranges"])
        if key not in seen:
            seen[key] = time_schedule(L, cams, lms, cam_idx, lm_idx, uv, opts, s, iters)
            if log:
                log(f"schedule {key}: {seen[key]:.4f} ms/iteration")
        return seen[key]

    for name, cands in (("chunk_obs", CHUNKS), ("tile_obs", TILE_OBS), ("tile_lms", TILE_LMS), ("ranges", RANGES)):
        times = {c: measure(dict(best, **{name: c})) for c in cands}
        best[name] = min(times, key=times.get)
    return best, {"/".join(str(x) for x in k): v for k, v in seen.items()}
