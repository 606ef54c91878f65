"""Batches of independent scenes as one problem for the library's scene partition.

Scenes are concatenated with their camera and landmark indices offset, so that each scene's
cameras form one contiguous range (the partition given to ``daba_set_scenes``); results are
split back per scene. Pure data movement: no arithmetic of the method happens here.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Batch:
    cams: np.ndarray        # (sum M, 9)
    lms: np.ndarray         # (sum N, 3)
    cam_idx: np.ndarray     # (sum nnz,) int32
    lm_idx: np.ndarray      # (sum nnz,) int32
    uv: np.ndarray          # (sum nnz, 2)
    cam_begin: np.ndarray   # (n + 1,) int32 camera range of each scene
    lm_begin: np.ndarray    # (n + 1,) int32 landmark range of each scene
    obs_begin: np.ndarray   # (n + 1,) int64 observation range of each scene

    @property
    def M(self):
        return int(self.cams.shape[0])

    @property
    def N(self):
        return int(self.lms.shape[0])

    @property
    def nnz(self):
        return int(self.cam_idx.size)


def merge(scenes) -> Batch:
    """Concatenate scenes (objects with cams, lms, cam_idx, lm_idx, uv) into one problem."""
    M = np.array([s.cams.shape[0] for s in scenes])
    N = np.array([s.lms.shape[0] for s in scenes])
    E = np.array([s.cam_idx.size for s in scenes])
    cb = np.concatenate([[0], np.cumsum(M)]).astype(np.int32)
    lb = np.concatenate([[0], np.cumsum(N)]).astype(np.int32)
    ob = np.concatenate([[0], np.cumsum(E)]).astype(np.int64)
    return Batch(cams=np.concatenate([s.cams for s in scenes]), lms=np.concatenate([s.lms for s in scenes]),
                 cam_idx=np.concatenate([s.cam_idx + c for s, c in zip(scenes, cb[:-1])]).astype(np.int32),
                 lm_idx=np.concatenate([s.lm_idx + l for s, l in zip(scenes, lb[:-1])]).astype(np.int32),
                 uv=np.concatenate([s.uv for s in scenes]), cam_begin=cb, lm_begin=lb, obs_begin=ob)


def split(batch: Batch, cams, lms):
    """Per-scene (cams, lms) from the batch's state arrays."""
    return [(cams[batch.cam_begin[i]:batch.cam_begin[i + 1]], lms[batch.lm_begin[i]:batch.lm_begin[i + 1]])
            for i in range(len(batch.cam_begin) - 1)]
