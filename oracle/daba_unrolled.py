"""Gradient of the state after K iterations of Algorithm 1 (FP64, CPU): test infrastructure.

TEST INFRASTRUCTURE ONLY, like daba_oracle.py. The update of one iteration, written out again
with plain PyTorch CPU float64 operations so that autograd differentiates it. It follows the
numpy oracle step by step: Eqs. nesterov_scalar and nesterov_x for the extrapolation, the
majorizer of Proposition 1 (w, lambda, g), the closed-form landmark solve, S-CAM (or, with
cam_solver = "lm", one successful LM step) for the cameras and ProjRot3D (Eq. proj_rot3d, as the
polar factor). The adaptive-restart decisions are
taken from a run of the numpy oracle and held fixed: they are piecewise constant in the
inputs, so they carry no gradient. The internal unit s (pixels) is held fixed as well: the
iteration depends on it only through xi, which is given in internal units.

unrolled_state(...) returns the boundary state after K iterations as torch tensors that
depend on the initial boundary state (cams, lms) and the pixels uv.
"""
from __future__ import annotations

import numpy as np
import torch

from oracle import daba_oracle as O

F64 = torch.float64


def _segsum(idx, vals, n):
    out = torch.zeros((n,) + tuple(vals.shape[1:]), dtype=F64)
    return out.index_add(0, idx, vals)


def _rho_w(loss, c, s):
    """rho'(s) of the losses of daba_oracle.rho (only w enters the update)."""
    if loss == "trivial":
        return torch.ones_like(s)
    if loss == "huber":
        big = s > c * c
        return torch.where(big, c / torch.sqrt(torch.where(big, s, torch.ones_like(s))), torch.ones_like(s))
    if loss == "cauchy":
        return 1.0 / (1.0 + s / (c * c))
    if loss == "welsch":
        return torch.exp(-s / (c * c))
    raise ValueError(loss)


def _ray(u, d):
    s = u[:, 0] ** 2 + u[:, 1] ** 2
    return torch.stack([u[:, 0], u[:, 1], d[:, 0] + d[:, 1] * s + d[:, 2] * s * s], 1)


def _majorizer(loss, c, R, t, d, l, u):
    """w, lambda and g of Proposition 1 (Eqs. w, gamma, g) at a conditioning iterate."""
    p = _ray(u, d)
    q = l - t
    Rp = torch.einsum("nab,nb->na", R, p)
    lam = (q * Rp).sum(1) / (q * q).sum(1)
    E = Rp - lam[:, None] * q                      # R e (world frame)
    w = _rho_w(loss, c, (E * E).sum(1))
    g = 0.5 * Rp + 0.5 * lam[:, None] * t + 0.5 * lam[:, None] * l
    return w, lam, g


def _proj_rot3d(K):
    """ProjRot3D for det K > 0 (every K of the iteration here): the orthogonal polar factor,
    by Newton's iteration X <- (z X + X^{-T} / z) / 2 (Frobenius scaling z for the first steps,
    held constant under differentiation) run to convergence. Its limit is the SVD answer of
    Eq. proj_rot3d, and unlike the SVD its derivative stays defined when K is a rotation
    (equal singular values), as at the first extrapolation."""
    X = K
    for it in range(40):
        Xi = torch.linalg.inv(X).transpose(-1, -2)
        if it < 8:
            z = torch.sqrt(torch.linalg.matrix_norm(Xi) / torch.linalg.matrix_norm(X)).detach()[..., None, None]
            X = 0.5 * (z * X + Xi / z)
        else:
            X = 0.5 * (X + Xi)
    return X


def _solve_landmarks(xi, w, lam, g, lz, li, N):
    num = 2.0 * _segsum(li, (w * lam)[:, None] * g, N) + xi * lz
    den = 2.0 * _segsum(li, w * lam ** 2, N) + xi
    return num / den[:, None]


def _solve_cameras(xi, w, lam, g, Rz, tz, dz, ci, u, M, n_alt):
    R, t, d = Rz, tz, dz
    s = u[:, 0] ** 2 + u[:, 1] ** 2
    phi = torch.stack([torch.ones_like(s), s, s * s], 1)
    for _ in range(n_alt):
        p = _ray(u, d[ci])
        v = 2.0 * w[:, None] * (g - lam[:, None] * t[ci])
        K = _segsum(ci, v[:, :, None] * p[:, None, :], M) + xi * Rz
        R = _proj_rot3d(K)
        Ri = R[ci]
        n = u.shape[0]
        A = torch.zeros((n, 3, 6), dtype=F64)
        eye = torch.eye(3, dtype=F64)
        A = A + torch.cat([lam[:, None, None] * eye[None], Ri[:, :, 2][:, :, None] * phi[:, None, :]], 2)
        b = torch.einsum("nab,nb->na", Ri[:, :, 0:2], u) - g
        Nm = 2.0 * _segsum(ci, w[:, None, None] * torch.einsum("nai,naj->nij", A, A), M) + xi * torch.eye(6, dtype=F64)
        rhs = -2.0 * _segsum(ci, w[:, None] * torch.einsum("nai,na->ni", A, b), M) + xi * torch.cat([tz, dz], 1)
        y = torch.linalg.solve(Nm, rhs[:, :, None])[:, :, 0]
        t, d = y[:, 0:3], y[:, 3:6]
    return R, t, d


def _skew(p):
    z = torch.zeros_like(p[:, 0])
    return torch.stack([torch.stack([z, -p[:, 2], p[:, 1]], 1), torch.stack([p[:, 2], z, -p[:, 0]], 1),
                        torch.stack([-p[:, 1], p[:, 0], z], 1)], 1)


def _solve_cameras_lm(xi, w, lam, g, Rz, tz, dz, ci, u, M):
    """One successful LM step per camera, as daba_oracle.solve_cameras_lm: the Gauss-Newton model
    (A, b) from the per-observation Jacobians at c_z, theta = -(A + mu diag A)^-1 b for mu = 1e-3,
    1e-2, ..., the first trial that lowers the block surrogate taken (else the camera stays at c_z).
    Which trial is taken is decided without gradient (piecewise constant); the taken theta is
    differentiated through A, b and Exp."""
    s = u[:, 0] ** 2 + u[:, 1] ** 2
    phi_u = torch.stack([torch.ones_like(s), s, s * s], 1)
    p0 = _ray(u, dz[ci])
    Rzi = Rz[ci]
    r0 = torch.einsum("nab,nb->na", Rzi, p0) + lam[:, None] * tz[ci] - g
    eye = torch.eye(3, dtype=F64).expand(u.shape[0], 3, 3)
    J = torch.cat([-torch.einsum("nab,nbc->nac", Rzi, _skew(p0)), lam[:, None, None] * eye,
                   Rzi[:, :, 2][:, :, None] * phi_u[:, None, :]], 2)
    A = 2.0 * _segsum(ci, w[:, None, None] * torch.einsum("nai,naj->nij", J, J), M)
    A = A + xi * torch.diag(torch.tensor([2.0, 2.0, 2.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0], dtype=F64))[None]
    b = 2.0 * _segsum(ci, w[:, None] * torch.einsum("nai,na->ni", J, r0), M)
    theta = torch.zeros((M, 9), dtype=F64)
    done = torch.zeros(M, dtype=torch.bool)
    mu = O.LM_MU0
    for _ in range(O.LM_TRIES):
        Ad = A + mu * torch.diag_embed(torch.diagonal(A, dim1=1, dim2=2))
        th = torch.linalg.solve(Ad, -b[:, :, None])[:, :, 0]
        with torch.no_grad():   # the surrogate decrease decides the trial (as the numpy oracle)
            Rc = Rz @ _exp(th[:, 0:3])
            tc, dc = tz + th[:, 3:6], dz + th[:, 6:9]
            dr = (torch.einsum("nab,nb->na", Rc[ci], _ray(u, dc[ci])) - torch.einsum("nab,nb->na", Rzi, p0)
                  + lam[:, None] * (tc - tz)[ci])
            dE = _segsum(ci, w * (dr * (dr + 2.0 * r0)).sum(1), M) + 0.5 * xi * (
                ((Rc - Rz) ** 2).sum((1, 2)) + ((tc - tz) ** 2).sum(1) + ((dc - dz) ** 2).sum(1))
            take = (~done) & (dE < 0.0)
        theta = torch.where(take[:, None], th, theta)
        done = done | take
        mu *= 10.0
    return Rz @ _exp(theta[:, 0:3]), tz + theta[:, 3:6], dz + theta[:, 6:9]


def _exp(w):
    th = torch.sqrt((w * w).sum(-1) + 1e-300)[..., None, None]
    K = torch.zeros(w.shape[:-1] + (3, 3), dtype=F64)
    K = K + torch.stack([torch.stack([torch.zeros_like(w[..., 0]), -w[..., 2], w[..., 1]], -1),
                         torch.stack([w[..., 2], torch.zeros_like(w[..., 0]), -w[..., 0]], -1),
                         torch.stack([-w[..., 1], w[..., 0], torch.zeros_like(w[..., 0])], -1)], -2)
    a = torch.sin(th) / th
    b = (1.0 - torch.cos(th)) / (th * th)
    return torch.eye(3, dtype=F64) + a * K + b * (K @ K)


def _log(R):
    c = ((R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]) - 1.0) / 2.0
    v = torch.stack([R[:, 2, 1] - R[:, 1, 2], R[:, 0, 2] - R[:, 2, 0], R[:, 1, 0] - R[:, 0, 1]], 1) / 2.0
    sn = torch.sqrt((v * v).sum(1))
    th = torch.atan2(sn, c)
    return v * (th / sn)[:, None]


def unrolled_state(cams, lms, uv, cam_idx, lm_idx, opts: O.Options, K: int, restart_cam, restart_lm, s_norm):
    """Boundary state (cams M x 9, lms N x 3) after K iterations from x^0 = x^(-1) = (cams, lms),
    as torch tensors; restart_cam[k], restart_lm[k] are the decisions of iteration k."""
    ci = torch.as_tensor(np.asarray(cam_idx, np.int64))
    li = torch.as_tensor(np.asarray(lm_idx, np.int64))
    M, N = cams.shape[0], lms.shape[0]
    sn = float(s_norm)
    u = uv / sn
    c = opts.loss_scale_px / sn
    xi = opts.xi
    R = _exp(cams[:, 0:3])
    t = cams[:, 3:6]
    f = cams[:, 6]
    d = torch.stack([f / sn, cams[:, 7] * sn / f, cams[:, 8] * sn ** 3 / f ** 3], 1)
    l = lms
    Rp, tp, dp, lp = R, t, d, l
    s = 1.0

    def cameras(w, lam, g, Rz, tz, dz):
        if opts.cam_solver == "lm":
            return _solve_cameras_lm(xi, w, lam, g, Rz, tz, dz, ci, u, M)
        return _solve_cameras(xi, w, lam, g, Rz, tz, dz, ci, u, M, opts.cam_alternations)

    for k in range(K):
        s, gamma = O.nesterov(s)
        w, lam, g = _majorizer(opts.loss, c, R[ci], t[ci], d[ci], l[li], u)
        Rm, tm, dm = cameras(w, lam, g, R, t, d)
        lmm = _solve_landmarks(xi, w, lam, g, l, li, N)
        if opts.accelerated:
            Rb = _proj_rot3d(R + gamma * (R - Rp))
            tb, db, lb = t + gamma * (t - tp), d + gamma * (d - dp), l + gamma * (l - lp)
            wb, lamb, gb = _majorizer(opts.loss, c, Rb[ci], tb[ci], db[ci], lb[li], u)
            Ra, ta, da = cameras(wb, lamb, gb, Rb, tb, db)
            la = _solve_landmarks(xi, wb, lamb, gb, lb, li, N)
            rc = torch.as_tensor(np.asarray(restart_cam[k], bool))
            rl = torch.as_tensor(np.asarray(restart_lm[k], bool))
            Rn = torch.where(rc[:, None, None], Rm, Ra)
            tn = torch.where(rc[:, None], tm, ta)
            dn = torch.where(rc[:, None], dm, da)
            ln = torch.where(rl[:, None], lmm, la)
            if opts.momentum_reset and opts.restart == "global" and bool(np.all(restart_cam[k])):
                s = 1.0   # the Nesterov scalar restarts with a global restart (the momentum reset)
        else:
            Rn, tn, dn, ln = Rm, tm, dm, lmm
        Rp, tp, dp, lp = R, t, d, l
        R, t, d, l = Rn, tn, dn, ln
    f = d[:, 0] * sn
    out_c = torch.cat([_log(R), t, f[:, None], (d[:, 1] * f / sn)[:, None], (d[:, 2] * f ** 3 / sn ** 3)[:, None]], 1)
    return out_c, l


def unrolled_grad(cams, lms, cam_idx, lm_idx, uv, opts: O.Options, K: int, g_cams, g_lms):
    """Gradient of <g_cams, cams_K> + <g_lms, lms_K> w.r.t. (cams, lms, uv) and the final state;
    the restart decisions come from the numpy oracle's run of the same K iterations."""
    res = O.daba(cams, lms, cam_idx, lm_idx, uv, opts, K, keep_infos=K)
    s_norm = res.prob.s_norm
    rc = [inf.restart_cam for inf in res.infos]
    rl = [inf.restart_lm for inf in res.infos]
    tc = torch.tensor(np.asarray(cams, np.float64), requires_grad=True)
    tl = torch.tensor(np.asarray(lms, np.float64), requires_grad=True)
    tu = torch.tensor(np.asarray(uv, np.float64), requires_grad=True)
    oc, ol = unrolled_state(tc, tl, tu, cam_idx, lm_idx, opts, K, rc, rl, s_norm)
    loss = (oc * torch.as_tensor(g_cams)).sum() + (ol * torch.as_tensor(g_lms)).sum()
    gc, gl, gu = torch.autograd.grad(loss, (tc, tl, tu))
    return gc.numpy(), gl.numpy(), gu.numpy(), oc.detach().numpy(), ol.detach().numpy(), res
