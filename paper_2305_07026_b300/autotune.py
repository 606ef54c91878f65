"""Schedule autotuner: picks the camera-pass chunk size, the landmark-tile sizes and the cut of
the range schedule (daba_set_pipeline: camera ranges per iteration) of a problem by timing a few
iterations of each candidate on the GPU. The search is coordinate descent (chunk, then
observations per tile, then landmarks per tile, then the ranges), repeated until a whole sweep
changes no axis: the axes interact (the best chunk depends on how many ranges split the camera
pass, the best tile on the chunk's partial sums), so one sweep can stop short of the optimum of
the grid. Each schedule is timed once and remembered; with ``repeats`` > 1 the best of several
timings is kept, which damps run-to-run noise between near-equal schedules. The schedule changes
only how the work is cut into warps and CTAs and ordered on the GPU, not the method (results
differ at most in the order of FP sums).
"""
from __future__ import annotations

CHUNKS = (1024, 1536, 2048, 3072, 4096)
TILE_OBS = (256, 512, 1024, 2048)
TILE_LMS = (32, 64, 128)
RANGES = (1, 2, 4, 6)
AXES = (("chunk_obs", CHUNKS), ("tile_obs", TILE_OBS), ("tile_lms", TILE_LMS), ("ranges", RANGES))
OPTION_KEYS = ("chunk_obs", "tile_obs", "tile_lms")


def make_context(L, M, N, nnz, opts, sched):
    """A context with the schedule's options, and its two-range cut when the schedule has one."""
    d = L.Daba(M, N, nnz, **opts, **{k: v for k, v in sched.items() if k in OPTION_KEYS})
    if "ranges" in sched:
        d.set_pipeline(sched["ranges"])
    return d


def time_schedule(L, cams, lms, cam_idx, lm_idx, uv, opts, sched, iters=8, warmup=2, repeats=1):
    """Milliseconds per iteration of one schedule (CUDA events around ``iters`` iterations; the
    best of ``repeats`` timings of the same context)."""
    import torch
    d = make_context(L, cams.shape[0], lms.shape[0], cam_idx.size, opts, sched)
    try:
        d.set_observations(cam_idx, lm_idx, uv)
        d.set_state(cams, lms)
        d.run(max(warmup, iters))   # a warm-up of the timed length captures its graph
        best = float("inf")
        for _ in range(max(1, repeats)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            d.run(iters)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / iters)
        return best
    finally:
        d.close()


def default_schedule(nnz):
    """The library's defaults (the starting point of the search)."""
    return {"chunk_obs": 2048, "tile_obs": 512, "tile_lms": 128, "ranges": 2 if nnz >= 1 << 20 else 1}


def tune(cams, lms, cam_idx, lm_idx, uv, opts=None, iters=8, log=None, max_sweeps=3, repeats=1):
    """Returns (best schedule dict, {schedule: ms per iteration}) for this problem."""
    from paper_2305_07026_b300 import _lib as L
    opts = dict(opts or {})
    best = default_schedule(cam_idx.size)
    seen = {}

    def measure(s):
        key = (s["chunk_obs"], s["tile_obs"], s["tile_lms"], s["ranges"])
        if key not in seen:
            seen[key] = time_schedule(L, cams, lms, cam_idx, lm_idx, uv, opts, s, iters, repeats=repeats)
            if log:
                log(f"schedule {key}: {seen[key]:.4f} ms/iteration")
        return seen[key]

    for _ in range(max(1, max_sweeps)):
        changed = False
        for name, cands in AXES:
            times = {c: measure(dict(best, **{name: c})) for c in cands}
            pick = min(times, key=times.get)
            changed |= pick != best[name]
            best[name] = pick
        if not changed:
            break
    return best, {"/".join(str(x) for x in k): v for k, v in seen.items()}
