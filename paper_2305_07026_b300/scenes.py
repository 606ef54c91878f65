"""Seeded synthetic bundle-adjustment scenes.

This module only *creates data*: camera poses, intrinsics, landmarks, and the
observed distorted pixels those would produce under the division (undistortion)
model of the paper's reprojection ray (Sec. 3, Eq. reprojection1/ray), plus
noise, outliers and a perturbed initial iterate. It evaluates none of the
method's quantities (no reprojection error, robust loss, majorizer or solve), so
the FP64 oracle and the CUDA path can both consume its output without sharing
any of the method's arithmetic.

Boundary conventions (shared by the oracle and the C ABI):

* ``cams``: float64 (M, 9) rows ``[w0, w1, w2, t0, t1, t2, f, k1, k2]``.
  ``w`` is the axis-angle vector of the camera-to-world rotation ``R_i``; a
  world point ``l`` has camera-frame coordinates ``R_i^T (l - t_i)`` and ``t_i``
  is the camera centre. The camera looks along +z of its frame.
  ``f`` is the focal length in pixels; ``k1, k2`` are dimensionless radial
  undistortion coefficients on the normalised radius ``|u| / f``, i.e. the
  undistorted ray is ``[u / f, 1 + k1 |u/f|^2 + k2 |u/f|^4]``.
* ``lms``: float64 (N, 3) world landmark positions.
* ``cam_idx``/``lm_idx``: int32 (nnz,) observation endpoints.
* ``uv``: float64 (nnz, 2) observed pixels relative to the principal point.

Workloads (sizes follow the configurations the method is benchmarked on; the
real BAL / 1DSfM data of the paper's Sec. 7 is not available, so these
synthetic scenes stand in for it):

* ``circle``  : 20 cameras on a 10 m circle around a 4 m cube of 2,000 points.
* ``street``  : 1,000 cameras along a street-grid trajectory, 200k facade points.
* ``tourism`` : 10k cameras around photo-tourism sites, 4M points, power-law
  tracks (~25M observations).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

IMG_W = 1024
IMG_H = 768


@dataclasses.dataclass
class Scene:
    name: str
    cams: np.ndarray       # (M, 9) initial iterate x^(0) (boundary parameters)
    lms: np.ndarray        # (N, 3) initial landmarks
    cam_idx: np.ndarray    # (nnz,) int32
    lm_idx: np.ndarray     # (nnz,) int32
    uv: np.ndarray         # (nnz, 2) float64 pixels
    cams_gt: np.ndarray    # (M, 9) ground truth
    lms_gt: np.ndarray     # (N, 3) ground truth
    loss: str              # "trivial" | "huber" | "cauchy" | "welsch"
    loss_scale_px: float
    iters: int
    seed: int
    outlier_mask: np.ndarray = None

    @property
    def M(self) -> int:
        return int(self.cams.shape[0])

    @property
    def N(self) -> int:
        return int(self.lms.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.cam_idx.shape[0])

    def describe(self) -> dict:
        cdeg = np.bincount(self.cam_idx, minlength=self.M)
        ldeg = np.bincount(self.lm_idx, minlength=self.N)
        return {
            "name": self.name, "M": self.M, "N": self.N, "nnz": self.nnz,
            "loss": self.loss, "loss_scale_px": self.loss_scale_px,
            "cam_degree_min": int(cdeg.min()), "cam_degree_median": float(np.median(cdeg)),
            "cam_degree_max": int(cdeg.max()),
            "track_min": int(ldeg.min()), "track_mean": float(ldeg.mean()),
            "track_max": int(ldeg.max()),
        }


# ----------------------------------------------------------------------------
# rotation parameterisation helpers (data layer only)
# ----------------------------------------------------------------------------

def _skew(v):
    z = np.zeros(v.shape[:-1])
    return np.stack([
        np.stack([z, -v[..., 2], v[..., 1]], -1),
        np.stack([v[..., 2], z, -v[..., 0]], -1),
        np.stack([-v[..., 1], v[..., 0], z], -1)], -2)


def axis_angle_to_matrix(w: np.ndarray) -> np.ndarray:
    """Rodrigues' formula, batched over leading axes."""
    w = np.asarray(w, dtype=np.float64)
    th = np.linalg.norm(w, axis=-1)[..., None, None]
    K = _skew(w)
    small = th < 1e-8
    ths = np.where(small, 1.0, th)
    a = np.where(small, 1.0 - th ** 2 / 6.0, np.sin(ths) / ths)
    b = np.where(small, 0.5 - th ** 2 / 24.0, (1.0 - np.cos(ths)) / ths ** 2)
    return np.eye(3) + a * K + b * (K @ K)


def matrix_to_axis_angle(R: np.ndarray) -> np.ndarray:
    """Rotation matrix -> axis-angle through a unit quaternion (Shepperd)."""
    R = np.asarray(R, dtype=np.float64)
    shp = R.shape[:-2]
    R = R.reshape(-1, 3, 3)
    n = R.shape[0]
    q = np.empty((n, 4))
    tr = np.trace(R, axis1=1, axis2=2)
    d = np.stack([tr, R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], 1)
    k = np.argmax(d, axis=1)
    for case in range(4):
        m = k == case
        if not np.any(m):
            continue
        Rm = R[m]
        if case == 0:
            s = np.sqrt(1.0 + tr[m]) * 2
            q[m] = np.stack([0.25 * s, (Rm[:, 2, 1] - Rm[:, 1, 2]) / s,
                             (Rm[:, 0, 2] - Rm[:, 2, 0]) / s, (Rm[:, 1, 0] - Rm[:, 0, 1]) / s], 1)
        elif case == 1:
            s = np.sqrt(1.0 + Rm[:, 0, 0] - Rm[:, 1, 1] - Rm[:, 2, 2]) * 2
            q[m] = np.stack([(Rm[:, 2, 1] - Rm[:, 1, 2]) / s, 0.25 * s,
                             (Rm[:, 0, 1] + Rm[:, 1, 0]) / s, (Rm[:, 0, 2] + Rm[:, 2, 0]) / s], 1)
        elif case == 2:
            s = np.sqrt(1.0 + Rm[:, 1, 1] - Rm[:, 0, 0] - Rm[:, 2, 2]) * 2
            q[m] = np.stack([(Rm[:, 0, 2] - Rm[:, 2, 0]) / s, (Rm[:, 0, 1] + Rm[:, 1, 0]) / s,
                             0.25 * s, (Rm[:, 1, 2] + Rm[:, 2, 1]) / s], 1)
        else:
            s = np.sqrt(1.0 + Rm[:, 2, 2] - Rm[:, 0, 0] - Rm[:, 1, 1]) * 2
            q[m] = np.stack([(Rm[:, 1, 0] - Rm[:, 0, 1]) / s, (Rm[:, 0, 2] + Rm[:, 2, 0]) / s,
                             (Rm[:, 1, 2] + Rm[:, 2, 1]) / s, 0.25 * s], 1)
    q *= np.where(q[:, :1] < 0, -1.0, 1.0)
    v = q[:, 1:]
    nv = np.linalg.norm(v, axis=1)
    ang = 2.0 * np.arctan2(nv, q[:, 0])
    scale = np.where(nv < 1e-12, 2.0, ang / np.where(nv < 1e-12, 1.0, nv))
    return (v * scale[:, None]).reshape(shp + (3,))


def look_at(centres: np.ndarray, targets: np.ndarray, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera-to-world rotations whose +z axis points from centre to target."""
    z = targets - centres
    z /= np.linalg.norm(z, axis=-1, keepdims=True)
    upv = np.broadcast_to(np.asarray(up, dtype=np.float64), z.shape)
    x = np.cross(z, upv)
    x /= np.linalg.norm(x, axis=-1, keepdims=True)
    y = np.cross(z, x)
    return np.stack([x, y, z], axis=-1)   # columns are the camera axes in world


def _random_unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


# ----------------------------------------------------------------------------
# image formation (data model): ideal projection -> distorted pixel
# ----------------------------------------------------------------------------

def distort(m: np.ndarray, f: np.ndarray, k1: np.ndarray, k2: np.ndarray):
    """Distorted pixel u for an ideal normalised projection m = X_c,xy / X_c,z.

    With the division model the undistorted ray is [u/f, 1 + k1 r^2 + k2 r^4]
    (r = |u|/f), so |m| = r / (1 + k1 r^2 + k2 r^4). The radius r is found by
    Newton's method started at |m|; returns (u, ok) where ok flags convergence
    to a root close to |m| (outside that, the model is not invertible there).
    """
    rm = np.sqrt(m[..., 0] ** 2 + m[..., 1] ** 2)
    r = rm.copy()
    act = np.arange(r.size)
    rf, rmf, k1f, k2f = r.reshape(-1), rm.reshape(-1), np.broadcast_to(k1, rm.shape).reshape(-1), \
        np.broadcast_to(k2, rm.shape).reshape(-1)
    for _ in range(30):
        ra, rma, k1a, k2a = rf[act], rmf[act], k1f[act], k2f[act]
        h = ra - rma * (1.0 + k1a * ra ** 2 + k2a * ra ** 4)
        dh = 1.0 - rma * (2.0 * k1a * ra + 4.0 * k2a * ra ** 3)
        step = h / np.where(np.abs(dh) > 1e-6, dh, 1e-6)
        rf[act] = np.clip(ra - step, 0.0, 10.0)
        act = act[np.abs(step) > 1e-15 * np.maximum(1.0, ra)]
        if act.size == 0:
            break
    r = rf.reshape(rm.shape)
    g = 1.0 + k1 * r ** 2 + k2 * r ** 4
    ok = (np.abs(r - rm * g) <= 1e-12 * np.maximum(1.0, r)) & (r >= 0) & (r < 3.0 * rm + 1e-9) & (g > 0.2)
    safe = np.where(rm > 0, rm, 1.0)
    u = (f * r / safe)[..., None] * m
    u = np.where((rm > 0)[..., None], u, 0.0)
    return u, ok


def project(R, t, f, k1, k2, X):
    """Distorted pixel of world points X for cameras (R, t, f, k1, k2) and a visibility mask.

    Only points in front of the camera whose ideal projection lies near the image
    are run through the Newton inversion of the division model.
    """
    Xc = np.einsum("...ji,...j->...i", R, X - t)
    shp = Xc.shape[:-1]
    Xc = Xc.reshape(-1, 3)
    fb = np.broadcast_to(f, shp).reshape(-1)
    k1b = np.broadcast_to(k1, shp).reshape(-1)
    k2b = np.broadcast_to(k2, shp).reshape(-1)
    z = Xc[:, 2]
    zs = np.where(z > 1e-3, z, 1.0)
    m = Xc[:, :2] / zs[:, None]
    cand = (z > 1e-3) & (np.linalg.norm(m, axis=1) * fb < 2.0 * math.hypot(IMG_W, IMG_H))
    u = np.zeros((Xc.shape[0], 2))
    vis = np.zeros(Xc.shape[0], dtype=bool)
    if np.any(cand):
        uc, ok = distort(m[cand], fb[cand], k1b[cand], k2b[cand])
        inside = (np.abs(uc[:, 0]) <= IMG_W / 2) & (np.abs(uc[:, 1]) <= IMG_H / 2)
        u[cand] = uc
        vis[cand] = ok & inside
    return u.reshape(shp + (2,)), vis.reshape(shp)


def _intrinsics(rng, M):
    f = rng.uniform(500.0, 800.0, M)
    k1 = rng.normal(0.0, 1e-2, M)
    k2 = rng.normal(0.0, 1e-4, M)
    return f, k1, k2


def _finish(name, rng, R, t, f, k1, k2, L, cam_idx, lm_idx, outlier_frac, loss, scale, iters, seed,
            rot_deg=2.0, trans_m=0.1, lm_sigma=0.05, min_cam=1, uv_clean=None):
    """Drop landmarks with fewer than 2 observations, add noise/outliers, perturb x^(0)."""
    # prune until every landmark has >= 2 and every camera >= min_cam observations
    while True:
        ldeg = np.bincount(lm_idx, minlength=L.shape[0])
        cdeg = np.bincount(cam_idx, minlength=R.shape[0])
        lkeep = ldeg >= 2
        ckeep = cdeg >= min_cam
        if lkeep.all() and ckeep.all():
            break
        sel = lkeep[lm_idx] & ckeep[cam_idx]
        if uv_clean is not None:
            uv_clean = uv_clean[sel]
        lmap = -np.ones(L.shape[0], dtype=np.int64)
        lmap[lkeep] = np.arange(int(lkeep.sum()))
        cmap = -np.ones(R.shape[0], dtype=np.int64)
        cmap[ckeep] = np.arange(int(ckeep.sum()))
        cam_idx = cmap[cam_idx[sel]]
        lm_idx = lmap[lm_idx[sel]]
        L = L[lkeep]
        R, t, f, k1, k2 = R[ckeep], t[ckeep], f[ckeep], k1[ckeep], k2[ckeep]
    M = R.shape[0]
    # observations in (landmark, camera) order: ordering is part of the input
    order = np.lexsort((cam_idx, lm_idx))
    cam_idx = cam_idx[order].astype(np.int32)
    lm_idx = lm_idx[order].astype(np.int32)
    nnz = cam_idx.shape[0]
    if uv_clean is not None:
        uv = uv_clean[order]
    else:
        uv = np.empty((nnz, 2))
        B = 1 << 22
        for b0 in range(0, nnz, B):
            ci, li = cam_idx[b0:b0 + B], lm_idx[b0:b0 + B]
            uv[b0:b0 + B], ok = project(R[ci], t[ci], f[ci], k1[ci], k2[ci], L[li])
            assert ok.all(), "generator produced an observation outside the image"
    uv = uv + rng.normal(0.0, 1.0, size=(nnz, 2))
    n_out = int(round(outlier_frac * nnz))
    out_mask = np.zeros(nnz, dtype=bool)
    if n_out:
        oi = rng.choice(nnz, size=n_out, replace=False)
        out_mask[oi] = True
        uv[oi, 0] = rng.uniform(-IMG_W / 2, IMG_W / 2, n_out)
        uv[oi, 1] = rng.uniform(-IMG_H / 2, IMG_H / 2, n_out)
    w_gt = matrix_to_axis_angle(R)
    cams_gt = np.concatenate([w_gt, t, f[:, None], k1[:, None], k2[:, None]], 1)
    dR = axis_angle_to_matrix(_random_unit(rng, M) * math.radians(rot_deg))
    R0 = dR @ R
    t0 = t + trans_m * _random_unit(rng, M)
    cams0 = np.concatenate([matrix_to_axis_angle(R0), t0, f[:, None], k1[:, None], k2[:, None]], 1)
    lms0 = L + rng.normal(0.0, lm_sigma, size=L.shape)
    return Scene(name=name, cams=cams0, lms=lms0, cam_idx=cam_idx, lm_idx=lm_idx, uv=uv,
                 cams_gt=cams_gt, lms_gt=L.copy(), loss=loss, loss_scale_px=scale, iters=iters,
                 seed=seed, outlier_mask=out_mask)


# ----------------------------------------------------------------------------
# circle workload: cameras on a circle around a cube of points
# ----------------------------------------------------------------------------

def circle_scene(seed=0, n_cams=20, n_lms=2000, radius=10.0, half=2.0, cap=8,
                 outlier_frac=0.03, loss="huber", scale=1.0, iters=200, noise_free=False):
    rng = np.random.default_rng(seed)
    ang = 2 * np.pi * np.arange(n_cams) / n_cams
    t = np.stack([radius * np.cos(ang), radius * np.sin(ang), np.zeros(n_cams)], 1)
    R = look_at(t, np.zeros_like(t))
    f, k1, k2 = _intrinsics(rng, n_cams)
    L = rng.uniform(-half, half, size=(n_lms, 3))
    _, vis = project(R[None], t[None], f[None], k1[None], k2[None], L[:, None, :])
    cam_list, lm_list = [], []
    for j in range(n_lms):
        v = np.flatnonzero(vis[j])
        if v.size > cap:
            v = rng.choice(v, size=cap, replace=False)
        cam_list.append(v)
        lm_list.append(np.full(v.size, j))
    cam_idx = np.concatenate(cam_list)
    lm_idx = np.concatenate(lm_list)
    sc = _finish("circle", rng, R, t, f, k1, k2, L, cam_idx, lm_idx, 0.0 if noise_free else outlier_frac,
                 loss, scale, iters, seed)
    if noise_free:
        sc.uv, _ = project(R[sc.cam_idx], t[sc.cam_idx], f[sc.cam_idx], k1[sc.cam_idx], k2[sc.cam_idx],
                           sc.lms_gt[sc.lm_idx])
    return sc


# ----------------------------------------------------------------------------
# workload 1: street-grid trajectory, facade points
# ----------------------------------------------------------------------------

def street_scene(seed=1, n_cams=1000, n_lms=200_000, grid=1000.0, spacing=100.0, path_blocks=30,
                 vis_range=60.0, outlier_frac=0.05, loss="cauchy", scale=2.0, iters=300):
    rng = np.random.default_rng(seed)
    nline = int(round(grid / spacing)) + 1
    # random walk on the grid intersections (no immediate reversal)
    node = np.array([rng.integers(0, nline), rng.integers(0, nline)])
    path = [node.copy()]
    prev = None
    dirs = np.array([[1, 0], [-1, 0], [0, 1], [0, -1]])
    while len(path) <= path_blocks:
        cand = [d for d in dirs if 0 <= node[0] + d[0] < nline and 0 <= node[1] + d[1] < nline
                and (prev is None or not np.array_equal(d, -prev))]
        d = cand[rng.integers(0, len(cand))]
        node = node + d
        prev = d
        path.append(node.copy())
    P = np.array(path, dtype=np.float64) * spacing - grid / 2
    seg_len = np.linalg.norm(np.diff(P, axis=0), axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg_len)])
    s = (np.arange(n_cams) + 0.5) * cum[-1] / n_cams
    si = np.clip(np.searchsorted(cum, s, side="right") - 1, 0, len(seg_len) - 1)
    a = (s - cum[si]) / seg_len[si]
    pos = P[si] + a[:, None] * (P[si + 1] - P[si])
    t = np.concatenate([pos, np.full((n_cams, 1), 1.5)], 1)
    yaw = rng.uniform(0, 2 * np.pi, n_cams)
    fwd = np.stack([np.cos(yaw), np.sin(yaw), np.zeros(n_cams)], 1)
    R = look_at(t, t + fwd)
    f, k1, k2 = _intrinsics(rng, n_cams)
    # facades along the traversed street segments (both sides)
    n_fac = 14 * path_blocks
    fseg = rng.integers(0, len(seg_len), n_fac)
    fa = rng.uniform(0, 1, n_fac)
    base = P[fseg] + fa[:, None] * (P[fseg + 1] - P[fseg])
    along = (P[fseg + 1] - P[fseg]) / seg_len[fseg][:, None]
    normal = np.stack([-along[:, 1], along[:, 0]], 1) * rng.choice([-1.0, 1.0], n_fac)[:, None]
    off = rng.uniform(5, 15, n_fac)
    width = rng.uniform(10, 40, n_fac)
    height = rng.uniform(5, 30, n_fac)
    area = width * height
    fid = rng.choice(n_fac, size=n_lms, p=area / area.sum())
    ua = rng.uniform(-0.5, 0.5, n_lms)
    ub = rng.uniform(0, 1, n_lms)
    xy = base[fid] + normal[fid] * off[fid][:, None] + along[fid] * (width[fid] * ua)[:, None]
    L = np.concatenate([xy, (height[fid] * ub)[:, None]], 1)
    # visibility: cameras within range, in front, inside the image
    # visibility: cameras within range, in front, inside the image; a camera whose
    # random yaw shows (almost) no facade points gets its yaw re-drawn
    from scipy.spatial import cKDTree
    pairs = cKDTree(t[:, :2]).sparse_distance_matrix(cKDTree(L[:, :2]), vis_range, output_type="ndarray")
    order = np.argsort(pairs["i"], kind="stable")
    pc = pairs["i"][order].astype(np.int64)
    pl = pairs["j"][order].astype(np.int64)
    del pairs, order
    vis = np.zeros(pc.size, dtype=bool)
    uvp = np.zeros((pc.size, 2))
    todo = np.arange(n_cams)
    start = np.searchsorted(pc, np.arange(n_cams + 1))
    for attempt in range(20):
        sel = np.concatenate([np.arange(start[c], start[c + 1]) for c in todo]) if todo.size < n_cams \
            else np.arange(pc.size)
        B = 1 << 22
        for b0 in range(0, sel.size, B):
            sb = sel[b0:b0 + B]
            ci, li = pc[sb], pl[sb]
            uvp[sb], vis[sb] = project(R[ci], t[ci], f[ci], k1[ci], k2[ci], L[li])
        cnt = np.bincount(pc[vis], minlength=n_cams)
        todo = np.flatnonzero(cnt < 50)
        if todo.size == 0 or attempt == 19:
            break
        yaw[todo] = rng.uniform(0, 2 * np.pi, todo.size)
        fwd = np.stack([np.cos(yaw), np.sin(yaw), np.zeros(n_cams)], 1)
        R[todo] = look_at(t[todo], t[todo] + fwd[todo])
    cam_rep, lm_rep, uvp = pc[vis], pl[vis], uvp[vis]
    # track length L = 2 + Geom(1/4) (mean 5), capped by visibility
    track = 1 + rng.geometric(0.25, n_lms)
    key = rng.random(lm_rep.size)
    order = np.lexsort((key, lm_rep))
    lm_rep, cam_rep, uvp = lm_rep[order], cam_rep[order], uvp[order]
    start = np.searchsorted(lm_rep, np.arange(n_lms))
    rank = np.arange(lm_rep.size) - start[lm_rep]
    take = rank < track[lm_rep]
    return _finish("street", rng, R, t, f, k1, k2, L, cam_rep[take], lm_rep[take], outlier_frac,
                   loss, scale, iters, seed, uv_clean=uvp[take])


# ----------------------------------------------------------------------------
# workload 2: photo-tourism sites, power-law tracks
# ----------------------------------------------------------------------------

def _powerlaw_tracks(rng, n, alpha=2.2, lo=2.0, hi=200.0):
    """Continuous P(L) ~ L^-alpha on [lo, hi] by inverse CDF, rounded to integers."""
    a1 = 1.0 - alpha
    u = rng.random(n)
    x = (lo ** a1 + u * (hi ** a1 - lo ** a1)) ** (1.0 / a1)
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def tourism_scene(seed=2, n_cams=10_000, n_lms=4_000_000, n_sites=100, site_spacing=200.0,
                  outlier_frac=0.05, loss="huber", scale=1.0, iters=100, min_cam_degree=20):
    rng = np.random.default_rng(seed)
    # site popularity: Pareto with density exponent 2.2, clipped
    w = np.minimum(rng.pareto(1.2, n_sites) + 1.0, 60.0)
    cams_per = np.maximum(30, np.floor(n_cams * w ** 0.6 / (w ** 0.6).sum())).astype(np.int64)
    while cams_per.sum() > n_cams:
        cams_per[np.argmax(cams_per)] -= 1
    cams_per[np.argmin(cams_per)] += n_cams - cams_per.sum()
    lms_per = np.floor(n_lms * w / w.sum()).astype(np.int64)
    lms_per[np.argmax(lms_per)] += n_lms - lms_per.sum()
    g = int(math.ceil(math.sqrt(n_sites)))
    centres = np.stack([(np.arange(n_sites) % g) * site_spacing, (np.arange(n_sites) // g) * site_spacing,
                        np.zeros(n_sites)], 1)
    centres[:, :2] -= centres[:, :2].mean(0)
    rad = rng.uniform(8.0, 20.0, n_sites)
    hgt = rng.uniform(8.0, 25.0, n_sites)
    Rs, ts, Ls, Ns, cam_all, lm_all = [], [], [], [], [], []
    cam_off = 0
    lm_off = 0
    for s in range(n_sites):
        m, n = int(cams_per[s]), int(lms_per[s])
        caz = np.sort(rng.uniform(0, 2 * np.pi, m))
        cdist = rad[s] + rng.uniform(25.0, 60.0, m)
        tc = centres[s] + np.stack([cdist * np.cos(caz), cdist * np.sin(caz), rng.uniform(1.4, 1.8, m)], 1)
        tgt = centres[s] + np.array([0.0, 0.0, 0.5 * hgt[s]]) + rng.normal(0, 1.5, (m, 3))
        Rc = look_at(tc, tgt)
        laz = rng.uniform(0, 2 * np.pi, n)
        Lc = centres[s] + np.stack([rad[s] * np.cos(laz), rad[s] * np.sin(laz),
                                    rng.uniform(0.0, hgt[s], n)], 1)
        # a landmark is seen by a window of cameras nearest to it in azimuth
        tl = np.minimum(_powerlaw_tracks(rng, n), m)
        pos = np.searchsorted(caz, laz) % m
        first = (pos - tl // 2) % m
        rep = np.repeat(np.arange(n), tl)
        k = np.arange(rep.size) - np.repeat(np.cumsum(tl) - tl, tl)
        ci = (first[rep] + k) % m
        Rs.append(Rc)
        ts.append(tc)
        Ls.append(Lc)
        Ns.append(np.stack([np.cos(laz), np.sin(laz)], 1))
        cam_all.append(ci + cam_off)
        lm_all.append(rep + lm_off)
        cam_off += m
        lm_off += n
    R = np.concatenate(Rs)
    t = np.concatenate(ts)
    L = np.concatenate(Ls)
    Nrm = np.concatenate(Ns)
    cam_idx = np.concatenate(cam_all)
    lm_idx = np.concatenate(lm_all)
    f, k1, k2 = _intrinsics(rng, R.shape[0])
    vis = np.empty(cam_idx.size, dtype=bool)
    uvc = np.empty((cam_idx.size, 2))
    B = 1 << 22
    for b0 in range(0, cam_idx.size, B):
        ci, li = cam_idx[b0:b0 + B], lm_idx[b0:b0 + B]
        uvc[b0:b0 + B], vis[b0:b0 + B] = project(R[ci], t[ci], f[ci], k1[ci], k2[ci], L[li])
        # the point lies on a building surface: cull views from behind it
        view = t[ci] - L[li]
        nrm = np.concatenate([Nrm[li], np.zeros((li.size, 1))], 1)
        vis[b0:b0 + B] &= np.einsum("ij,ij->i", view, nrm) > 0.25 * np.linalg.norm(view, axis=1)
    cam_idx, lm_idx, uvc = cam_idx[vis], lm_idx[vis], uvc[vis]
    sc = _finish("tourism", rng, R, t, f, k1, k2, L, cam_idx, lm_idx, outlier_frac, loss, scale, iters, seed,
                 uv_clean=uvc)
    sc.min_cam_degree_target = min_cam_degree
    return sc


# ----------------------------------------------------------------------------
# batch of small independent scenes (serving-style workload)
# ----------------------------------------------------------------------------

def small_scene(seed, n_cams, n_lms, track_mean=4.0, radius=10.0, half=2.0, outlier_frac=0.03, loss="huber",
                scale=1.0, iters=100):
    """A circle-of-cameras scene (as ``circle``) whose landmarks have geometric track lengths
    (mean ``track_mean``, at least 2): landmark j is seen by a window of consecutive cameras
    starting at a random one. Every landmark of the 4 m cube projects inside the image of
    every camera on the 10 m circle, so no visibility test is needed."""
    rng = np.random.default_rng(seed)
    ang = 2 * np.pi * np.arange(n_cams) / n_cams
    t = np.stack([radius * np.cos(ang), radius * np.sin(ang), np.zeros(n_cams)], 1)
    R = look_at(t, np.zeros_like(t))
    f, k1, k2 = _intrinsics(rng, n_cams)
    L = rng.uniform(-half, half, size=(n_lms, 3))
    tl = np.minimum(np.maximum(2, rng.geometric(1.0 / track_mean, n_lms)), n_cams)
    first = rng.integers(0, n_cams, n_lms)
    rep = np.repeat(np.arange(n_lms), tl)
    k = np.arange(rep.size) - np.repeat(np.cumsum(tl) - tl, tl)
    cam_idx = (first[rep] + k) % n_cams
    return _finish("small", rng, R, t, f, k1, k2, L, cam_idx, rep, outlier_frac, loss, scale, iters, seed)


def batch_scenes(n_scenes=512, seed=4, cams=(5, 200), lms=(100, 20_000), track_mean=4.0):
    """``n_scenes`` independent small scenes with log-uniform camera and landmark counts."""
    rng = np.random.default_rng(seed)
    mc = np.exp(rng.uniform(np.log(cams[0]), np.log(cams[1]), n_scenes)).round().astype(int)
    nl = np.exp(rng.uniform(np.log(lms[0]), np.log(lms[1]), n_scenes)).round().astype(int)
    seeds = rng.integers(0, 2 ** 31, n_scenes)
    return [small_scene(int(sd), int(m), int(n), track_mean) for sd, m, n in zip(seeds, mc, nl)]


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def make_scene(workload: str, scale: float = 1.0, seed: int | None = None, **kw) -> Scene:
    """Build a named workload; ``scale`` shrinks camera/landmark counts for tests."""
    if workload == "circle":
        return circle_scene(seed=0 if seed is None else seed, **kw)
    if workload == "street":
        return street_scene(seed=1 if seed is None else seed, n_cams=max(20, int(round(1000 * scale))),
                            n_lms=max(200, int(round(200_000 * scale))),
                            path_blocks=max(2, int(round(30 * scale))), **kw)
    if workload == "tourism":
        n_sites = max(1, int(round(100 * min(1.0, scale * 10))))
        return tourism_scene(seed=2 if seed is None else seed, n_cams=max(60, int(round(10_000 * scale))),
                             n_lms=max(2000, int(round(4_000_000 * scale))), n_sites=n_sites, **kw)
    raise ValueError(f"unknown workload {workload!r}")
