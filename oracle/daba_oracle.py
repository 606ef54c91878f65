"""FP64 CPU oracle for DABA (Decentralized and Accelerated Bundle Adjustment).

TEST INFRASTRUCTURE ONLY. This module is a plain, slow, FP64 restatement of the
paper's definitions and of Algorithm 1. Only the test suite, the package's
``smoke()`` check and the benchmark's CPU-baseline leg may import it; the CUDA
library never calls it and shares no code with it.

Every quantity is evaluated per observation by direct summation, in the order
and notation of the paper:

* Sec. 3   -- undistorted ray p_ij (Eq. ray), scale lambda_ij (Eq. lambdaij),
              reprojection error e_ij (Eq. error).
* Sec. 2   -- penalty F_ij = rho(|e_ij|^2)/2 (Eq. Fij), objective F (Eq. Fobj),
              robust losses satisfying Assumption 1 (App. B).
* Sec. 4   -- majorizer P_ij + Q_ij of Proposition 1 (Eqs. P, Q, a, w, gamma, g)
              and the block surrogate E^alpha (Eq. Ealpha).
* Sec. 5   -- Nesterov scalars (Eq. nesterov_scalar), extrapolation
              (Eq. nesterov_x), ProjRot3D (Eq. proj_rot3d), restart metrics
              (Eqs. DEalpha, Fainit, Fak, lFak, Eak).
* Sec. 6   -- Algorithm 1 (DABA) and its unaccelerated ablation DUBA (Sec. 7.2).

Readings where the paper is silent:

* Blocks: every camera and every landmark is its own block, so every
  reprojection pair is inter-block (E' is empty) and E^alpha of a camera is
  xi/2 |c - c_z|^2 + sum_j P_ij(c|z), of a landmark xi/2 |l - l_z|^2 + sum_i
  Q_ij(l|z); |c - c_z|^2 = |R - R_z|_F^2 + |t - t_z|^2 + |d - d_z|^2.
* Units: pixels are divided by s_norm (default: median focal length); with
  boundary coefficients k1, k2 on the normalised radius |u|/f the intrinsics
  are d = (f/s, k1 s/f, k2 s^3/f^3), loss scales c/s, and F_px = s^2 F.
* Subproblem solvers (the paper's LM details are not given): landmarks are
  solved in closed form; cameras by n_alt block-exact alternations of an
  R-step (ProjRot3D of a 3x3 matrix) and a (t, d)-step (6x6 normal equations).
* Nesterov s^k is global (Algorithm 1 never resets it); the restart test uses
  strict '>' (no restart on equality).

Method variant (not Algorithm 1 as printed; Options.restart = "global"): one
restart test for the whole problem on the sums of the block metrics,
sum_alpha E^alpha(k+1) > sum_alpha Fbar^alpha(k), which a single device can
evaluate because it holds every block; when it fires every block takes its MM
update (Eq. update_mm). Since the recursions of Eqs. Fak, lFak and Eak are
linear, the sums are the same metrics for one block made of everything, so the
convergence argument of App. C.3 applies unchanged. With
Options.momentum_reset the Nesterov scalar restarts too: after an iteration
whose global test fired, s^(k+1) = 1, so gamma^(k+1) = 0.

Method variant (Options.cam_solver = "lm"): each camera subproblem takes one
successful Levenberg-Marquardt step (Sec. 7.1 reports one successful inner LM
step). Its parameterisation, Gauss-Newton model and damping schedule are
readings (the paper gives none); the model is pinned against the surrogate's
derivatives, but parity with the paper's own LM implementation is unpinned.
"""
from __future__ import annotations

import dataclasses

import numpy as np

LOSSES = ("trivial", "huber", "cauchy", "welsch")


# ----------------------------------------------------------------------------
# robust loss (Sec. 2, Assumption 1)
# ----------------------------------------------------------------------------

def rho(loss: str, c: float, s: np.ndarray):
    """rho(s) and rho'(s) of a robust loss at s = |e|^2 (Assumption 1, App. B).

    trivial: rho(s) = s.  Huber (scale c): s for s <= c^2, else 2 c sqrt(s) - c^2.
    Cauchy: c^2 log(1 + s/c^2).  Welsch: c^2 (1 - exp(-s/c^2)).
    """
    s = np.asarray(s, dtype=np.float64)
    if loss == "trivial":
        return s.copy(), np.ones_like(s)
    if loss == "huber":
        big = s > c * c
        rs = np.sqrt(np.where(big, s, 1.0))
        return np.where(big, 2.0 * c * rs - c * c, s), np.where(big, c / rs, 1.0)
    if loss == "cauchy":
        return c * c * np.log1p(s / (c * c)), 1.0 / (1.0 + s / (c * c))
    if loss == "welsch":
        ex = np.exp(-s / (c * c))
        return c * c * (1.0 - ex), ex
    raise ValueError(loss)


# ----------------------------------------------------------------------------
# parameterisation (boundary <-> paper variables)
# ----------------------------------------------------------------------------

def so3_exp(w: np.ndarray) -> np.ndarray:
    """Rotation matrix of an axis-angle vector (Rodrigues)."""
    w = np.asarray(w, dtype=np.float64).reshape(-1, 3)
    th = np.linalg.norm(w, axis=1)
    out = np.empty((w.shape[0], 3, 3))
    for n in range(w.shape[0]):
        K = np.array([[0.0, -w[n, 2], w[n, 1]], [w[n, 2], 0.0, -w[n, 0]], [-w[n, 1], w[n, 0], 0.0]])
        if th[n] < 1e-8:
            a, b = 1.0 - th[n] ** 2 / 6.0, 0.5 - th[n] ** 2 / 24.0
        else:
            a, b = np.sin(th[n]) / th[n], (1.0 - np.cos(th[n])) / th[n] ** 2
        out[n] = np.eye(3) + a * K + b * (K @ K)
    return out


def so3_log(R: np.ndarray) -> np.ndarray:
    """Axis-angle vector of rotation matrices (principal branch, angle in [0, pi]).

    theta = atan2(|v|, (tr R - 1)/2) with v = vee(R - R^T)/2 = sin(theta) a; for
    theta above 2pi/3 the axis a is read from the symmetric part (1 - cos) a a^T.
    """
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3, 3)
    out = np.empty((R.shape[0], 3))
    for n in range(R.shape[0]):
        A = R[n]
        c = (np.trace(A) - 1.0) / 2.0
        v = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]]) / 2.0
        sn = np.linalg.norm(v)
        th = np.arctan2(sn, c)
        if c > -0.5:
            out[n] = v * (th / sn if sn > 1e-300 else 1.0)
        else:
            B = (A + A.T) / 2.0 - c * np.eye(3)
            k = int(np.argmax(np.diag(B)))
            a = B[:, k] / np.linalg.norm(B[:, k])
            if a @ v < 0:
                a = -a
            out[n] = a * th
    return out


def median_focal(cams: np.ndarray) -> float:
    f = np.sort(np.asarray(cams, dtype=np.float64)[:, 6])
    m = f.shape[0]
    return float(f[m // 2]) if m % 2 else float(0.5 * (f[m // 2 - 1] + f[m // 2]))


def to_internal(cams, lms, s_norm):
    """Boundary (axis-angle, centre, f, k1, k2) -> (R, t, d) in units of s_norm pixels."""
    cams = np.asarray(cams, dtype=np.float64)
    R = so3_exp(cams[:, 0:3])
    t = cams[:, 3:6].copy()
    f, k1, k2 = cams[:, 6], cams[:, 7], cams[:, 8]
    d = np.stack([f / s_norm, k1 * s_norm / f, k2 * s_norm ** 3 / f ** 3], 1)
    return R, t, d, np.asarray(lms, dtype=np.float64).copy()


def to_boundary(R, t, d, l, s_norm):
    f = d[:, 0] * s_norm
    k1 = d[:, 1] * f / s_norm
    k2 = d[:, 2] * f ** 3 / s_norm ** 3
    cams = np.concatenate([so3_log(R), t, f[:, None], k1[:, None], k2[:, None]], 1)
    return cams, l.copy()


# ----------------------------------------------------------------------------
# Sec. 3: the reprojection error
# ----------------------------------------------------------------------------

def ray(u, d):
    """Undistorted ray p = [u; d1 + d2 |u|^2 + d3 |u|^4] (Eq. ray)."""
    s = u[:, 0] ** 2 + u[:, 1] ** 2
    return np.stack([u[:, 0], u[:, 1], d[:, 0] + d[:, 1] * s + d[:, 2] * s * s], 1)


def lam(R, t, l, p):
    """lambda = (l - t)^T R p / |l - t|^2 (Eq. lambdaij)."""
    q = l - t
    Rp = np.einsum("nab,nb->na", R, p)
    return np.einsum("na,na->n", q, Rp) / np.einsum("na,na->n", q, q)


def reproj_error(R, t, l, p):
    """e = (I - R^T (l - t)(l - t)^T R / |l - t|^2) p (Eq. error)."""
    v = np.einsum("nba,nb->na", R, l - t)          # R^T (l - t)
    return p - v * (np.einsum("na,na->n", v, p) / np.einsum("na,na->n", v, v))[:, None]


def F_obs(loss, c, R, t, d, l, u):
    """F_ij = rho(|e_ij|^2) / 2 (Eq. Fij) for every observation row."""
    e = reproj_error(R, t, l, ray(u, d))
    r, _ = rho(loss, c, np.einsum("na,na->n", e, e))
    return 0.5 * r


def objective(loss, c, R, t, d, l, cam_idx, lm_idx, u):
    """F(x) = sum over reprojection pairs of F_ij (Eq. Fobj)."""
    return float(np.sum(F_obs(loss, c, R[cam_idx], t[cam_idx], d[cam_idx], l[lm_idx], u)))


# ----------------------------------------------------------------------------
# Sec. 4: majorization (Proposition 1) and the block surrogate (Eq. Ealpha)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Majorizer:
    """Per-observation quantities of Proposition 1 at a conditioning iterate."""
    w: np.ndarray      # Eq. w
    a: np.ndarray      # Eq. a
    lam: np.ndarray    # Eq. gamma (lambda_ij^(k))
    g: np.ndarray      # Eq. g


def majorizer(loss, c, R, t, d, l, u) -> Majorizer:
    p = ray(u, d)
    lm = lam(R, t, l, p)
    e = reproj_error(R, t, l, p)
    r = np.einsum("na,na->n", e, e)
    rv, w = rho(loss, c, r)
    a = 0.5 * rv - 0.5 * w * r
    Rp = np.einsum("nab,nb->na", R, p)
    g = 0.5 * Rp + 0.5 * lm[:, None] * t + 0.5 * lm[:, None] * l
    return Majorizer(w=w, a=a, lam=lm, g=g)


def P_obs(mj: Majorizer, R, t, d, u):
    """P_ij(c_i | x^k) = w |R p + lambda t - g|^2 + a/2 (Eq. P)."""
    res = np.einsum("nab,nb->na", R, ray(u, d)) + mj.lam[:, None] * t - mj.g
    return mj.w * np.einsum("na,na->n", res, res) + 0.5 * mj.a


def Q_obs(mj: Majorizer, l):
    """Q_ij(l_j | x^k) = w |lambda l - g|^2 + a/2 (Eq. Q)."""
    res = mj.lam[:, None] * l - mj.g
    return mj.w * np.einsum("na,na->n", res, res) + 0.5 * mj.a


def segsum(idx, vals, n):
    """Sum of per-observation values into their blocks (index order)."""
    vals = np.asarray(vals, dtype=np.float64)
    if vals.ndim == 1:
        return np.bincount(idx, weights=vals, minlength=n)
    flat = vals.reshape(vals.shape[0], -1)
    out = np.stack([np.bincount(idx, weights=flat[:, k], minlength=n) for k in range(flat.shape[1])], 1)
    return out.reshape((n,) + vals.shape[1:])


def cam_sqdist(R, t, d, Rz, tz, dz):
    return (np.sum((R - Rz) ** 2, axis=(1, 2)) + np.sum((t - tz) ** 2, axis=1) + np.sum((d - dz) ** 2, axis=1))


def E_cam(xi, mj, R, t, d, Rz, tz, dz, cam_idx, u, M):
    """E^alpha(c | z) of every camera block (Eq. Ealpha with E' empty)."""
    P = P_obs(mj, R[cam_idx], t[cam_idx], d[cam_idx], u)
    return 0.5 * xi * cam_sqdist(R, t, d, Rz, tz, dz) + segsum(cam_idx, P, M)


def E_lm(xi, mj, l, lz, lm_idx, N):
    """E^alpha(l | z) of every landmark block (Eq. Ealpha with E' empty)."""
    Q = Q_obs(mj, l[lm_idx])
    return 0.5 * xi * np.sum((l - lz) ** 2, axis=1) + segsum(lm_idx, Q, N)


# ----------------------------------------------------------------------------
# Sec. 5: rotation projection, Nesterov scalars, extrapolation
# ----------------------------------------------------------------------------

def proj_rot3d(Mx: np.ndarray) -> np.ndarray:
    """argmin_{R in SO(3)} |R - M|^2 = U diag(1, 1, det(U V^T)) V^T (Eq. proj_rot3d)."""
    U, _, Vt = np.linalg.svd(Mx)
    sgn = np.sign(np.linalg.det(U @ Vt))
    sgn = np.where(sgn == 0, 1.0, sgn)
    D = np.zeros(Mx.shape[:-2] + (3, 3))
    D[..., 0, 0] = 1.0
    D[..., 1, 1] = 1.0
    D[..., 2, 2] = sgn
    return U @ D @ Vt


def nesterov(s: float):
    """s^(k+1) = (sqrt(4 s^2 + 1) + 1)/2 and gamma^(k) = (s^(k) - 1)/s^(k+1) (Eq. nesterov_scalar)."""
    s_next = (np.sqrt(4.0 * s * s + 1.0) + 1.0) / 2.0
    return s_next, (s - 1.0) / s_next


def extrapolate(R, t, d, l, Rp, tp, dp, lp, gamma):
    """Extrapolated iterate of Eq. nesterov_x (R through ProjRot3D)."""
    return (proj_rot3d(R + gamma * (R - Rp)), t + gamma * (t - tp), d + gamma * (d - dp), l + gamma * (l - lp))


# ----------------------------------------------------------------------------
# subproblem solvers (exact block minimizers of E^alpha(. | z))
# ----------------------------------------------------------------------------

def solve_landmarks(xi, mj, lz, lm_idx, N):
    """argmin_l xi/2 |l - l_z|^2 + sum_i w |lambda l - g|^2 (closed form of the Eq. Q sum)."""
    num = 2.0 * segsum(lm_idx, (mj.w * mj.lam)[:, None] * mj.g, N) + xi * lz
    den = 2.0 * segsum(lm_idx, mj.w * mj.lam ** 2, N) + xi
    return num / den[:, None]


def solve_cameras(xi, mj, Rz, tz, dz, cam_idx, u, M, n_alt):
    """Block-exact alternation on E^alpha(c | z) of every camera, started at c_z.

    R-step: with (t, d) fixed, sum_j w |R p_j + lambda_j t - g_j|^2 + xi/2 |R - R_z|^2
    is affine in R (|R p| = |p|), so its minimiser is ProjRot3D(K) with
    K = sum_j 2 w_j (g_j - lambda_j t) p_j^T + xi R_z.
    (t, d)-step: with R fixed, R p(d) + lambda t - g = A y + b with y = (t, d),
    A = [lambda I_3 | (R e_3) phi^T], phi = (1, s, s^2), b = R[:, :2] u - g, whose
    normal equations (2 sum w A^T A + xi I) y = -2 sum w A^T b + xi y_z are solved.
    """
    R, t, d = Rz.copy(), tz.copy(), dz.copy()
    s = u[:, 0] ** 2 + u[:, 1] ** 2
    phi = np.stack([np.ones_like(s), s, s * s], 1)
    wl = mj.w
    for _ in range(n_alt):
        p = ray(u, d[cam_idx])
        v = 2.0 * wl[:, None] * (mj.g - mj.lam[:, None] * t[cam_idx])
        K = segsum(cam_idx, v[:, :, None] * p[:, None, :], M) + xi * Rz
        R = proj_rot3d(K)
        Ri = R[cam_idx]
        A = np.zeros((u.shape[0], 3, 6))
        A[:, 0, 0] = A[:, 1, 1] = A[:, 2, 2] = mj.lam
        A[:, :, 3:6] = Ri[:, :, 2][:, :, None] * phi[:, None, :]
        b = np.einsum("nab,nb->na", Ri[:, :, 0:2], u) - mj.g
        Nm = 2.0 * segsum(cam_idx, wl[:, None, None] * np.einsum("nai,naj->nij", A, A), M) + xi * np.eye(6)
        rhs = -2.0 * segsum(cam_idx, wl[:, None] * np.einsum("nai,na->ni", A, b), M) \
            + xi * np.concatenate([tz, dz], 1)
        y = np.linalg.solve(Nm, rhs[:, :, None])[:, :, 0]
        t, d = y[:, 0:3], y[:, 3:6]
    return R, t, d


def skew(v):
    """[v]x, the cross-product matrix (v [..., 3] -> [..., 3, 3])."""
    z = np.zeros(v.shape[:-1])
    return np.stack([np.stack([z, -v[..., 2], v[..., 1]], -1), np.stack([v[..., 2], z, -v[..., 0]], -1),
                     np.stack([-v[..., 1], v[..., 0], z], -1)], -2)


LM_MU0 = 1e-3      # initial damping of the camera LM step (relative to diag of the model Hessian)
LM_TRIES = 8       # damping increases (x10) before the step is given up


def lm_model(xi, mj, Rz, tz, dz, cam_idx, u, M):
    """Gauss-Newton model of E^alpha(. | z) of every camera at c_z in theta = (phi, tau, delta)
    (see solve_cameras_lm): Hessian A (M, 9, 9), gradient b (M, 9), and per observation the
    residual r(0) and ray p(d_z)."""
    s = u[:, 0] ** 2 + u[:, 1] ** 2
    phi_u = np.stack([np.ones_like(s), s, s * s], 1)
    p0 = ray(u, dz[cam_idx])
    Rzi = Rz[cam_idx]
    r0 = np.einsum("nab,nb->na", Rzi, p0) + mj.lam[:, None] * tz[cam_idx] - mj.g
    J = np.zeros((u.shape[0], 3, 9))
    J[:, :, 0:3] = -np.einsum("nab,nbc->nac", Rzi, skew(p0))
    J[:, 0, 3] = J[:, 1, 4] = J[:, 2, 5] = mj.lam
    J[:, :, 6:9] = Rzi[:, :, 2][:, :, None] * phi_u[:, None, :]
    w = mj.w
    A = 2.0 * segsum(cam_idx, w[:, None, None] * np.einsum("nai,naj->nij", J, J), M)
    A += xi * np.diag([2.0, 2.0, 2.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0])[None]
    b = 2.0 * segsum(cam_idx, w[:, None] * np.einsum("nai,na->ni", J, r0), M)
    return A, b, r0, p0


def solve_cameras_lm(xi, mj, Rz, tz, dz, cam_idx, u, M):
    """One successful Levenberg-Marquardt step on E^alpha(c | z) of every camera, from c_z
    (the subproblem solver the paper reports for DABA: one successful inner LM step).

    Parameters theta = (phi, tau, delta): R = R_z Exp(phi), t = t_z + tau, d = d_z + delta.
    Per observation the residual of Eq. P is r = R p(d) + lambda t - g with Jacobian at theta = 0
    J = [-R_z [p_z]x, lambda I, (R_z e3) (1, s, s^2)]. Gauss-Newton model of the block surrogate:
    Hessian A = 2 sum w J^T J + xi diag(2 I, I, I) (the proximal term xi/2 |R - R_z|^2 to second
    order is xi |phi|^2), gradient b = 2 sum w J^T r(0). The step solves (A + mu diag A) theta = -b;
    it is taken if the surrogate decreases, E(c | z) < E(c_z | z), else mu grows tenfold; after
    LM_TRIES failures the camera stays at c_z. The decrease is evaluated from the residual
    differences r(c) - r(0), so that no O(F) values cancel."""
    A, b, r0, p0 = lm_model(xi, mj, Rz, tz, dz, cam_idx, u, M)
    w = mj.w
    R, t, d = Rz.copy(), tz.copy(), dz.copy()
    for i in range(M):
        obs = np.flatnonzero(cam_idx == i)
        mu = LM_MU0
        for _ in range(LM_TRIES):
            Ad = A[i] + mu * np.diag(np.diag(A[i]))
            th = np.linalg.solve(Ad, -b[i])
            Rc = Rz[i] @ so3_exp(th[0:3])[0]
            tc, dc = tz[i] + th[3:6], dz[i] + th[6:9]
            dr = (np.einsum("ab,nb->na", Rc, ray(u[obs], np.broadcast_to(dc, (obs.size, 3))))
                  - np.einsum("ab,nb->na", Rz[i], p0[obs]) + mj.lam[obs, None] * (tc - tz[i]))
            dE = np.sum(w[obs] * np.einsum("na,na->n", dr, dr + 2.0 * r0[obs])) \
                + 0.5 * xi * (np.sum((Rc - Rz[i]) ** 2) + np.sum((tc - tz[i]) ** 2) + np.sum((dc - dz[i]) ** 2))
            if dE < 0.0:
                R[i], t[i], d[i] = Rc, tc, dc
                break
            mu *= 10.0
    return R, t, d


# ----------------------------------------------------------------------------
# Algorithm 1
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Options:
    loss: str = "huber"
    loss_scale_px: float = 1.0
    xi: float = 1e-10
    eta: float = 0.5
    accelerated: bool = True
    cam_alternations: int = 2
    pixel_scale: float = 0.0     # 0: median focal length
    restart: str = "block"       # "block": Algorithm 1; "global": one test on the summed block metrics
    momentum_reset: bool = False  # with restart="global": s <- 1 after a restart
    cam_solver: str = "scam"     # "scam": block-exact alternations; "lm": one successful LM step


@dataclasses.dataclass
class State:
    """Iterate x^k, x^(k-1) and the per-block restart metrics of Eqs. Fak, lFak, Eak."""
    R: np.ndarray
    t: np.ndarray
    d: np.ndarray
    l: np.ndarray
    Rp: np.ndarray
    tp: np.ndarray
    dp: np.ndarray
    lp: np.ndarray
    s: float                 # Nesterov s^(k)
    k: int
    E_cam: np.ndarray        # E^alpha(k) of camera blocks
    E_lm: np.ndarray
    Fbar_cam: np.ndarray     # Fbar^alpha(k-1)
    Fbar_lm: np.ndarray


@dataclasses.dataclass
class Problem:
    cam_idx: np.ndarray
    lm_idx: np.ndarray
    u: np.ndarray            # pixels / s_norm
    M: int
    N: int
    s_norm: float
    loss: str
    c: float                 # loss scale / s_norm
    opts: Options


def make_problem(cams, lms, cam_idx, lm_idx, uv, opts: Options):
    s_norm = opts.pixel_scale if opts.pixel_scale > 0 else median_focal(cams)
    prob = Problem(cam_idx=np.asarray(cam_idx, dtype=np.int64), lm_idx=np.asarray(lm_idx, dtype=np.int64),
                   u=np.asarray(uv, dtype=np.float64) / s_norm, M=int(np.asarray(cams).shape[0]),
                   N=int(np.asarray(lms).shape[0]), s_norm=float(s_norm), loss=opts.loss,
                   c=opts.loss_scale_px / s_norm, opts=opts)
    R, t, d, l = to_internal(cams, lms, s_norm)
    return prob, R, t, d, l


def init_state(prob: Problem, R, t, d, l) -> State:
    """x^(-1) = x^(0), s^(0) = 1 and Eq. Fainit: F^alpha(-1) = E^alpha(x^alpha(-1) | x^(-1))."""
    ci, li, u = prob.cam_idx, prob.lm_idx, prob.u
    mj = majorizer(prob.loss, prob.c, R[ci], t[ci], d[ci], l[li], u)
    Fc = E_cam(prob.opts.xi, mj, R, t, d, R, t, d, ci, u, prob.M)
    Fl = E_lm(prob.opts.xi, mj, l, l, li, prob.N)
    return State(R=R.copy(), t=t.copy(), d=d.copy(), l=l.copy(), Rp=R.copy(), tp=t.copy(), dp=d.copy(),
                 lp=l.copy(), s=1.0, k=0, E_cam=Fc.copy(), E_lm=Fl.copy(), Fbar_cam=Fc.copy(),
                 Fbar_lm=Fl.copy())


@dataclasses.dataclass
class StepInfo:
    F: float                 # F(x^k)
    F_cam: np.ndarray        # F^alpha(k)
    F_lm: np.ndarray
    Fbar_cam: np.ndarray     # Fbar^alpha(k)
    Fbar_lm: np.ndarray
    Enext_cam: np.ndarray    # E^alpha(k+1) after the restart test
    Enext_lm: np.ndarray
    Etest_cam: np.ndarray    # E^alpha(k+1) of the accelerated update (the tested value)
    Etest_lm: np.ndarray
    restart_cam: np.ndarray  # restart decisions (Algorithm 1, adaptive restart)
    restart_lm: np.ndarray
    gamma: float


def step(prob: Problem, st: State):
    """One iteration k of Algorithm 1 with singleton blocks; returns (x^(k+1) state, info)."""
    o = prob.opts
    xi, eta = o.xi, o.eta
    ci, li, u, M, N = prob.cam_idx, prob.lm_idx, prob.u, prob.M, prob.N
    # Nesterov's acceleration (Eq. nesterov_scalar, Eq. nesterov_x)
    s_next, gamma = nesterov(st.s)
    Rb, tb, db, lb = extrapolate(st.R, st.t, st.d, st.l, st.Rp, st.tp, st.dp, st.lp, gamma)
    # majorization at x^k, at the extrapolated iterate and at x^(k-1) (Prop. 1)
    mj_k = majorizer(prob.loss, prob.c, st.R[ci], st.t[ci], st.d[ci], st.l[li], u)
    mj_b = majorizer(prob.loss, prob.c, Rb[ci], tb[ci], db[ci], lb[li], u)
    mj_p = majorizer(prob.loss, prob.c, st.Rp[ci], st.tp[ci], st.dp[ci], st.lp[li], u)
    Fij = F_obs(prob.loss, prob.c, st.R[ci], st.t[ci], st.d[ci], st.l[li], u)
    # Eq. DEalpha at x^k conditioned on x^(k-1); the surrogate gap is shared by both blocks
    gap = Fij - P_obs(mj_p, st.R[ci], st.t[ci], st.d[ci], u) - Q_obs(mj_p, st.l[li])
    dE_cam = -0.5 * xi * cam_sqdist(st.R, st.t, st.d, st.Rp, st.tp, st.dp) + 0.5 * segsum(ci, gap, M)
    dE_lm = -0.5 * xi * np.sum((st.l - st.lp) ** 2, axis=1) + 0.5 * segsum(li, gap, N)
    # Eq. Fak and Eq. lFak
    F_cam = st.E_cam + dE_cam
    F_lm = st.E_lm + dE_lm
    Fbar_cam = (1.0 - eta) * st.Fbar_cam + eta * F_cam
    Fbar_lm = (1.0 - eta) * st.Fbar_lm + eta * F_lm
    # minimization: accelerated (Eq. update_amm) or plain MM (Eq. update_mm)
    cams_solve = (lambda mj, Rz, tz, dz: solve_cameras_lm(xi, mj, Rz, tz, dz, ci, u, M)) if o.cam_solver == "lm" \
        else (lambda mj, Rz, tz, dz: solve_cameras(xi, mj, Rz, tz, dz, ci, u, M, o.cam_alternations))
    Rm, tm, dm = cams_solve(mj_k, st.R, st.t, st.d)
    lm_mm = solve_landmarks(xi, mj_k, st.l, li, N)
    E0_cam = E_cam(xi, mj_k, st.R, st.t, st.d, st.R, st.t, st.d, ci, u, M)   # E^alpha(x^k | x^k)
    E0_lm = E_lm(xi, mj_k, st.l, st.l, li, N)
    Emm_cam = E_cam(xi, mj_k, Rm, tm, dm, st.R, st.t, st.d, ci, u, M) + F_cam - E0_cam
    Emm_lm = E_lm(xi, mj_k, lm_mm, st.l, li, N) + F_lm - E0_lm
    if o.accelerated:
        Ra, ta, da = cams_solve(mj_b, Rb, tb, db)
        la = solve_landmarks(xi, mj_b, lb, li, N)
        # Eq. Eak for the accelerated update, then the adaptive restart test
        Ea_cam = E_cam(xi, mj_k, Ra, ta, da, st.R, st.t, st.d, ci, u, M) + F_cam - E0_cam
        Ea_lm = E_lm(xi, mj_k, la, st.l, li, N) + F_lm - E0_lm
        if o.restart == "global":
            # the test of Algorithm 1 for the single block made of every camera and landmark
            fire = bool(np.sum(Ea_cam) + np.sum(Ea_lm) > np.sum(Fbar_cam) + np.sum(Fbar_lm))
            rs_cam = np.full(M, fire)
            rs_lm = np.full(N, fire)
            if fire and o.momentum_reset:
                s_next = 1.0
        else:
            rs_cam = Ea_cam > Fbar_cam
            rs_lm = Ea_lm > Fbar_lm
    else:
        Ra, ta, da, la = Rm, tm, dm, lm_mm
        Ea_cam, Ea_lm = Emm_cam, Emm_lm
        rs_cam = np.ones(M, dtype=bool)
        rs_lm = np.ones(N, dtype=bool)
    Rn = np.where(rs_cam[:, None, None], Rm, Ra)
    tn = np.where(rs_cam[:, None], tm, ta)
    dn = np.where(rs_cam[:, None], dm, da)
    ln = np.where(rs_lm[:, None], lm_mm, la)
    En_cam = np.where(rs_cam, Emm_cam, Ea_cam)
    En_lm = np.where(rs_lm, Emm_lm, Ea_lm)
    new = State(R=Rn, t=tn, d=dn, l=ln, Rp=st.R, tp=st.t, dp=st.d, lp=st.l, s=s_next, k=st.k + 1,
                E_cam=En_cam, E_lm=En_lm, Fbar_cam=Fbar_cam, Fbar_lm=Fbar_lm)
    info = StepInfo(F=float(np.sum(Fij)), F_cam=F_cam, F_lm=F_lm, Fbar_cam=Fbar_cam, Fbar_lm=Fbar_lm,
                    Enext_cam=En_cam, Enext_lm=En_lm, Etest_cam=Ea_cam, Etest_lm=Ea_lm,
                    restart_cam=rs_cam if o.accelerated else np.zeros(M, dtype=bool),
                    restart_lm=rs_lm if o.accelerated else np.zeros(N, dtype=bool), gamma=gamma)
    return new, info


@dataclasses.dataclass
class RunResult:
    trace_px2: np.ndarray            # F(x^k) for k = 0..iters, in pixel^2
    restarts: np.ndarray             # restarted blocks per iteration
    state: State
    infos: list
    prob: Problem


def daba(cams, lms, cam_idx, lm_idx, uv, opts: Options, iters: int, keep_infos: int = 0) -> RunResult:
    """Run Algorithm 1 (DABA, or DUBA with opts.accelerated=False) for `iters` iterations."""
    prob, R, t, d, l = make_problem(cams, lms, cam_idx, lm_idx, uv, opts)
    st = init_state(prob, R, t, d, l)
    trace, restarts, infos = [], [], []
    for _ in range(iters):
        st, info = step(prob, st)
        trace.append(info.F)
        restarts.append(int(info.restart_cam.sum() + info.restart_lm.sum()))
        if len(infos) < keep_infos:
            infos.append(info)
    trace.append(objective(prob.loss, prob.c, st.R, st.t, st.d, st.l, prob.cam_idx, prob.lm_idx, prob.u))
    return RunResult(trace_px2=np.asarray(trace) * prob.s_norm ** 2, restarts=np.asarray(restarts),
                     state=st, infos=infos, prob=prob)


def boundary_state(res: RunResult):
    """Final iterate in boundary parameters (cams (M, 9), lms (N, 3))."""
    st = res.state
    return to_boundary(st.R, st.t, st.d, st.l, res.prob.s_norm)


# ----------------------------------------------------------------------------
# Euclidean gradients of F_ij (App. D, Eq. DFij, with the d-selector acting on e)
# ----------------------------------------------------------------------------

def grad_F_obs(loss, c, R, t, d, l, u):
    """Per-observation Euclidean gradients of F_ij w.r.t. t_i, l_j, d_i and R_i.

    F_ij = rho(|e|^2)/2 with e = (I - n n^T) p, n = R^T(l - t)/|l - t|:
      grad_t = w lambda R e,  grad_l = -w lambda R e                  (Eq. DFij)
      grad_d = w (e_3 . e) phi with phi = (1, s, s^2)                 (Eq. DFij, selector on e)
      grad_R = -w lambda (l - t) e^T  (one ambient extension; its tangent part
               R skew(R^T G) agrees with every other extension, Eq. proj_grad).
    """
    p = ray(u, d)
    lm = lam(R, t, l, p)
    e = reproj_error(R, t, l, p)
    r = np.einsum("na,na->n", e, e)
    _, w = rho(loss, c, r)
    Re = np.einsum("nab,nb->na", R, e)
    gt = (w * lm)[:, None] * Re
    gl = -gt
    s = u[:, 0] ** 2 + u[:, 1] ** 2
    phi = np.stack([np.ones_like(s), s, s * s], 1)
    gd = (w * e[:, 2])[:, None] * phi
    gR = -(w * lm)[:, None, None] * (l - t)[:, :, None] * e[:, None, :]
    return gt, gl, gd, gR


def grad_F_obs_u(loss, c, R, t, d, l, u):
    """Per-observation gradient of F_ij w.r.t. the pixel u (internal units).

    p = (u_1, u_2, d_1 + d_2 s + d_3 s^2) (Eq. ray) and, lambda being the minimiser of
    |p - lambda R^T (l - t)|^2 (Eq. lambdaij), dF/dp = w e (camera frame), so
      dF/du_a = w (e_a + e_3 * 2 u_a (d_2 + 2 d_3 s)).
    """
    p = ray(u, d)
    e = reproj_error(R, t, l, p)
    r = np.einsum("na,na->n", e, e)
    _, w = rho(loss, c, r)
    s = u[:, 0] ** 2 + u[:, 1] ** 2
    dpz = 2.0 * (d[:, 1] + 2.0 * d[:, 2] * s)
    return w[:, None] * (e[:, 0:2] + (e[:, 2] * dpz)[:, None] * u)


def so3_right_jacobian(w):
    """J_r(w) with Exp(w + dw) = Exp(w) Exp(J_r(w) dw) + O(dw^2):
    J_r = I - (1 - cos th)/th^2 [w]x + (th - sin th)/th^3 [w]x^2 (series below 1e-6)."""
    w = np.asarray(w, dtype=np.float64)
    th = np.linalg.norm(w, axis=-1)[..., None, None]
    K = np.zeros(w.shape[:-1] + (3, 3))
    K[..., 0, 1], K[..., 0, 2], K[..., 1, 2] = -w[..., 2], w[..., 1], -w[..., 0]
    K[..., 1, 0], K[..., 2, 0], K[..., 2, 1] = w[..., 2], -w[..., 1], w[..., 0]
    small = th < 1e-6
    ths = np.where(small, 1.0, th)
    a = np.where(small, 0.5 - th ** 2 / 24.0, (1.0 - np.cos(ths)) / ths ** 2)
    b = np.where(small, 1.0 / 6.0 - th ** 2 / 120.0, (ths - np.sin(ths)) / ths ** 3)
    return np.eye(3) - a * K + b * (K @ K)


def grad_objective_boundary(cams, lms, cam_idx, lm_idx, uv, opts: Options):
    """F(x) in pixel^2 (Eq. Fobj) and its gradient w.r.t. the boundary parameters: cameras
    [w, t, f, k1, k2] (M x 9), landmarks (N x 3) and observed pixels (nnz x 2).

    Per observation the Euclidean gradients of Eq. DFij (grad_F_obs) and of the pixel
    (grad_F_obs_u) are summed per camera and landmark, then carried to the boundary:
    rotation through F(R Exp(phi)) (tangent gradient vee(R^T G - G^T R)) and the right
    Jacobian of Exp; intrinsics through d = (f/s, k1 s/f, k2 s^3/f^3); pixels through
    u' = u/s. F_px = s^2 F' with s the internal unit, which leaves F_px independent of s.
    """
    prob, R, t, d, l = make_problem(cams, lms, cam_idx, lm_idx, uv, opts)
    ci, li, u, s = prob.cam_idx, prob.lm_idx, prob.u, prob.s_norm
    Ri, ti, di, lj = R[ci], t[ci], d[ci], l[li]
    F = float(np.sum(F_obs(prob.loss, prob.c, Ri, ti, di, lj, u))) * s * s
    gt, gl, gd, gR = grad_F_obs(prob.loss, prob.c, Ri, ti, di, lj, u)
    gu = grad_F_obs_u(prob.loss, prob.c, Ri, ti, di, lj, u)
    M, N = prob.M, prob.N
    G = segsum(ci, gR.reshape(-1, 9), M).reshape(M, 3, 3)
    Gt = segsum(ci, gt, M)
    Gd = segsum(ci, gd, M)
    Gl = segsum(li, gl, N)
    RtG = np.einsum("nba,nbc->nac", R, G)
    S = RtG - np.transpose(RtG, (0, 2, 1))
    gphi = np.stack([S[:, 2, 1], S[:, 0, 2], S[:, 1, 0]], 1)
    cams = np.asarray(cams, dtype=np.float64)
    Jr = so3_right_jacobian(cams[:, 0:3])
    gw = np.einsum("nba,nb->na", Jr, gphi)
    f, k1, k2 = cams[:, 6], cams[:, 7], cams[:, 8]
    gf = Gd[:, 0] / s - Gd[:, 1] * k1 * s / f ** 2 - 3.0 * Gd[:, 2] * k2 * s ** 3 / f ** 4
    gk1 = Gd[:, 1] * s / f
    gk2 = Gd[:, 2] * s ** 3 / f ** 3
    g_cams = np.concatenate([gw, Gt, gf[:, None], gk1[:, None], gk2[:, None]], 1) * s * s
    return F, g_cams, Gl * s * s, gu * s
