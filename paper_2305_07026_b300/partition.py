"""Coarse-block partitions for `Daba.set_partition` (host-side index bookkeeping only).

A partition gives every camera and every landmark a block id; the pairs whose camera and
landmark share a block are kept exact in that block's surrogate (Eq. Ealpha), the others are
split by the majorizer of Proposition 1. The library takes blocks of at most BLK_MAX_CAMS
cameras.
"""
from __future__ import annotations

import numpy as np

from paper_2305_07026_b300._lib import BLK_MAX_CAMS


def camera_groups(M, cam_idx, lm_idx, N, n_blocks):
    """Contiguous groups of cameras (camera i in block i * n_blocks // M); every landmark joins
    the block of its lowest-index observing camera (a landmark nobody observes joins block 0).
    Returns (cam_block, lm_block) as int32 arrays."""
    if n_blocks < 1 or n_blocks > M:
        raise ValueError("n_blocks must lie in 1 .. M")
    if -(-M // n_blocks) > BLK_MAX_CAMS:
        raise ValueError(f"blocks of more than {BLK_MAX_CAMS} cameras: use at least {-(-M // BLK_MAX_CAMS)} blocks")
    cam_block = (np.arange(M, dtype=np.int64) * n_blocks) // M
    first = np.full(N, M, dtype=np.int64)
    np.minimum.at(first, np.asarray(lm_idx, dtype=np.int64), np.asarray(cam_idx, dtype=np.int64))
    lm_block = np.where(first < M, cam_block[np.minimum(first, M - 1)], 0)
    return cam_block.astype(np.int32), lm_block.astype(np.int32)
