"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-derived
closed forms (tests/golden), invariants of the method (Props. 1-2, Lemma 1,
Eq. FklFk0), an independent second method (ProjRot3D by Horn's quaternion
eigenvector instead of the SVD), finite differences, or brute force.
"""
import json
import os

import numpy as np
import pytest

from oracle import daba_oracle as O
from tests.conftest import cached_scene

GOLD = os.path.join(os.path.dirname(__file__), "golden", "closed_form_cases.json")


def _rand_rot(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z], -1)], -2)


def _rand_obs(rng, n):
    """Random camera/landmark/pixel rows in normalised units with the point in front."""
    R = _rand_rot(rng, n)
    t = rng.normal(scale=3.0, size=(n, 3))
    d = np.stack([rng.uniform(0.8, 1.2, n), rng.normal(0, 0.05, n), rng.normal(0, 0.01, n)], 1)
    u = rng.uniform(-0.6, 0.6, size=(n, 2))
    p = O.ray(u, d)
    depth = rng.uniform(2.0, 20.0, n)
    dirc = p / np.linalg.norm(p, axis=1, keepdims=True)
    noise = rng.normal(scale=0.02, size=(n, 3))
    l = t + np.einsum("nab,nb->na", R, dirc * depth[:, None] + noise * depth[:, None])
    return R, t, d, l, u


# ----------------------------------------------------------------------------
# Sec. 3 closed forms
# ----------------------------------------------------------------------------

def test_golden_reprojection_cases():
    g = json.load(open(GOLD))
    for c in g["cases"]:
        R = np.array(c["R"], float)[None]
        t = np.array(c["t"], float)[None]
        d = np.array(c["d"], float)[None]
        l = np.array(c["l"], float)[None]
        u = np.array(c["u"], float)[None]
        p = O.ray(u, d)
        np.testing.assert_allclose(p[0], c["p"], atol=1e-15)
        np.testing.assert_allclose(O.lam(R, t, l, p)[0], c["lambda"], atol=1e-15)
        e = O.reproj_error(R, t, l, p)[0]
        np.testing.assert_allclose(e, c["e"], atol=1e-15)
        np.testing.assert_allclose(e @ e, c["r"], atol=1e-15)


def test_golden_losses():
    g = json.load(open(GOLD))["loss_cases"]
    for c in g["cases"]:
        r, dr = O.rho(c["loss"], c["c"], np.array([c["s"]]))
        assert r[0] == pytest.approx(c["rho"], rel=1e-15, abs=1e-15)
        assert dr[0] == pytest.approx(c["drho"], rel=1e-15)


def test_error_geometry():
    """e is p projected on the plane normal to R^T(l - t): e . R^T q = 0, |e| = |p| sin(theta),
    and lambda minimises |p - lambda R^T q|^2 (Eq. error_opt)."""
    rng = np.random.default_rng(1)
    R, t, d, l, u = _rand_obs(rng, 500)
    p = O.ray(u, d)
    v = np.einsum("nba,nb->na", R, l - t)
    e = O.reproj_error(R, t, l, p)
    assert np.max(np.abs(np.einsum("na,na->n", e, v)) / np.linalg.norm(v, axis=1)) < 1e-14
    cos = np.einsum("na,na->n", p, v) / (np.linalg.norm(p, axis=1) * np.linalg.norm(v, axis=1))
    np.testing.assert_allclose(np.linalg.norm(e, axis=1), np.linalg.norm(p, axis=1) * np.sqrt(1 - cos ** 2),
                               rtol=1e-9, atol=1e-14)
    lam = O.lam(R, t, l, p)
    base = np.sum(e * e, axis=1)
    for dl in (1e-4, -1e-4, 1e-2, -0.3):
        alt = p - (lam + dl)[:, None] * v
        assert np.all(np.sum(alt * alt, axis=1) >= base)


def test_zero_error_at_noise_free_truth():
    """Eq. err0: noise-free observations generated by the division model give e = 0 at the truth."""
    sc = cached_scene("circle", noise_free=True)
    opts = O.Options(loss="trivial")
    prob, R, t, d, l = O.make_problem(sc.cams_gt, sc.lms_gt, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    F = O.objective("trivial", prob.c, R, t, d, l, prob.cam_idx, prob.lm_idx, prob.u) * prob.s_norm ** 2
    assert F < 1e-16 * sc.nnz
    prob0, R0, t0, d0, l0 = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    assert O.objective("trivial", prob0.c, R0, t0, d0, l0, prob0.cam_idx, prob0.lm_idx, prob0.u) > 1e-3


def test_similarity_invariance():
    """F depends only on the direction of l - t in each camera frame (Eq. error): a rigid
    motion plus a global scale of the whole scene leaves it unchanged."""
    sc = cached_scene("circle")
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px)
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    F0 = O.objective(prob.loss, prob.c, R, t, d, l, prob.cam_idx, prob.lm_idx, prob.u)
    rng = np.random.default_rng(3)
    Q = _rand_rot(rng, 1)[0]
    b = rng.normal(size=3) * 10
    sig = 3.7
    F1 = O.objective(prob.loss, prob.c, Q @ R, sig * t @ Q.T + b, d, sig * l @ Q.T + b,
                     prob.cam_idx, prob.lm_idx, prob.u)
    assert F1 == pytest.approx(F0, rel=1e-12)


def test_unit_reparameterisation():
    """The internal units of s_norm pixels are an exact reparameterisation: F in pixels^2 does not
    depend on the chosen scale (k1, k2 on |u|/f map to d = (f/s, k1 s/f, k2 s^3/f^3))."""
    sc = cached_scene("circle")
    vals = []
    for s in (1.0, 123.0, 650.0):
        opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, pixel_scale=s)
        prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
        vals.append(O.objective(prob.loss, prob.c, R, t, d, l, prob.cam_idx, prob.lm_idx, prob.u) * s * s)
    np.testing.assert_allclose(vals, vals[0], rtol=1e-12)


def test_boundary_roundtrip():
    sc = cached_scene("circle")
    s = O.median_focal(sc.cams)
    R, t, d, l = O.to_internal(sc.cams, sc.lms, s)
    cams, lms = O.to_boundary(R, t, d, l, s)
    np.testing.assert_allclose(cams, sc.cams, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(lms, sc.lms)
    w = np.array([[np.pi - 1e-7, 0.0, 0.0], [0.0, 1e-9, 0.0], [0.3, -2.0, 1.0]])
    w[2] *= (np.pi - 1e-3) / np.linalg.norm(w[2])
    np.testing.assert_allclose(O.so3_log(O.so3_exp(w)), w, atol=1e-8)


# ----------------------------------------------------------------------------
# Assumption 1 (robust losses)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("loss", O.LOSSES)
def test_loss_assumption1(loss):
    c = 0.7
    s = np.concatenate([[0.0], np.geomspace(1e-8, 50.0, 400)])
    r, dr = O.rho(loss, c, s)
    assert r[0] == 0.0 and dr[0] == 1.0                       # (a), (d) at 0
    assert np.all(r >= 0) and np.all(dr >= 0) and np.all(dr <= 1)  # (a), (d)
    h = 1e-6 * np.maximum(s, 1e-3)
    fd = (O.rho(loss, c, s + h)[0] - O.rho(loss, c, np.maximum(s - h, 0))[0]) / (s + h - np.maximum(s - h, 0))
    np.testing.assert_allclose(fd[1:], dr[1:], rtol=2e-5, atol=1e-9)   # (b): rho' is the derivative
    X, Y = np.meshgrid(s, s)
    rx = O.rho(loss, c, X)[0]
    ry, dry = O.rho(loss, c, Y)
    assert np.all(rx <= ry + dry * (X - Y) + 1e-12 * (1 + np.abs(X)))  # (c) concavity (tangent bound)


@pytest.mark.parametrize("loss", ["huber", "cauchy", "welsch"])
def test_loss_scale_homogeneity(loss):
    """rho_c(s^2 x) = s^2 rho_{c/s}(x): the pixel rescaling is exact for the scaled losses."""
    x = np.geomspace(1e-6, 10, 50)
    for sc in (0.01, 3.0, 700.0):
        np.testing.assert_allclose(O.rho(loss, 1.5, sc * sc * x)[0], sc * sc * O.rho(loss, 1.5 / sc, x)[0],
                                   rtol=1e-12)


# ----------------------------------------------------------------------------
# Proposition 1 and 2 (majorization)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("loss", O.LOSSES)
def test_majorizer_prop1(loss):
    rng = np.random.default_rng(7)
    R, t, d, l, u = _rand_obs(rng, 2000)
    c = 0.02
    mj = O.majorizer(loss, c, R, t, d, l, u)
    F = O.F_obs(loss, c, R, t, d, l, u)
    P = O.P_obs(mj, R, t, d, u)
    Q = O.Q_obs(mj, l)
    np.testing.assert_allclose(P + Q, F, rtol=1e-11, atol=1e-18)       # equality at x^k
    np.testing.assert_allclose(P, Q, rtol=1e-10, atol=1e-18)           # P = Q = F/2 at x^k
    # Eq. approx0: |R p + lambda t - g| = |lambda l - g| = |e|/2 at x^k
    p = O.ray(u, d)
    e = O.reproj_error(R, t, l, p)
    r1 = np.einsum("nab,nb->na", R, p) + mj.lam[:, None] * t - mj.g
    r2 = mj.lam[:, None] * l - mj.g
    np.testing.assert_allclose(np.linalg.norm(r1, axis=1), 0.5 * np.linalg.norm(e, axis=1), rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(r2, axis=1), 0.5 * np.linalg.norm(e, axis=1), rtol=1e-9, atol=1e-14)
    # inequality at random points, near and far
    for scale in (1e-4, 1e-2, 0.3):
        dR = O.so3_exp(rng.normal(scale=scale, size=(2000, 3)))
        R2, t2 = R @ dR, t + rng.normal(scale=scale, size=t.shape)
        d2 = d + rng.normal(scale=scale * 0.1, size=d.shape)
        l2 = l + rng.normal(scale=scale * 10, size=l.shape)
        F2 = O.F_obs(loss, c, R2, t2, d2, l2, u)
        bound = O.P_obs(mj, R2, t2, d2, u) + O.Q_obs(mj, l2)
        assert np.all(F2 <= bound * (1 + 1e-12) + 1e-18)


def test_surrogate_prop2(circle):
    """F(x) <= E(x | x^k) = sum_alpha E^alpha with equality at x^k (Prop. 2)."""
    sc = circle
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px)
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    ci, li = prob.cam_idx, prob.lm_idx
    mj = O.majorizer(prob.loss, prob.c, R[ci], t[ci], d[ci], l[li], prob.u)
    E = lambda R2, t2, d2, l2: (O.E_cam(opts.xi, mj, R2, t2, d2, R, t, d, ci, prob.u, prob.M).sum()
                                + O.E_lm(opts.xi, mj, l2, l, li, prob.N).sum())
    F = lambda R2, t2, d2, l2: O.objective(prob.loss, prob.c, R2, t2, d2, l2, ci, li, prob.u)
    assert E(R, t, d, l) == pytest.approx(F(R, t, d, l), rel=1e-12)
    rng = np.random.default_rng(11)
    for scale in (1e-5, 1e-3, 1e-1):
        R2 = R @ O.so3_exp(rng.normal(scale=scale, size=(prob.M, 3)))
        t2 = t + rng.normal(scale=scale, size=t.shape)
        d2 = d + rng.normal(scale=scale * 0.01, size=d.shape)
        l2 = l + rng.normal(scale=scale, size=l.shape)
        assert F(R2, t2, d2, l2) <= E(R2, t2, d2, l2) * (1 + 1e-13)


# ----------------------------------------------------------------------------
# gradients (App. C.3, D.4): finite differences and F/E gradient equality
# ----------------------------------------------------------------------------

def _tangent_fd(f, R, t, d, l, h=1e-6):
    """Central differences of a scalar function along the tangent directions of each variable."""
    out = {}
    n = R.shape[0]
    gR = np.zeros((n, 3))
    for a in range(3):
        w = np.zeros((n, 3))
        w[:, a] = h
        gR[:, a] = (f(R @ O.so3_exp(w), t, d, l) - f(R @ O.so3_exp(-w), t, d, l)) / (2 * h)
    out["R"] = gR
    for name, X in (("t", t), ("d", d), ("l", l)):
        G = np.zeros_like(X)
        for a in range(X.shape[1]):
            dX = np.zeros_like(X)
            dX[:, a] = h
            args = {"t": t, "d": d, "l": l}
            args[name] = X + dX
            fp = f(R, args["t"], args["d"], args["l"])
            args[name] = X - dX
            fm = f(R, args["t"], args["d"], args["l"])
            G[:, a] = (fp - fm) / (2 * h)
        out[name] = G
    return out


@pytest.mark.parametrize("loss", ["trivial", "huber", "cauchy"])
def test_gradient_fd(loss):
    """Eq. DFij (with the d-selector acting on e) against FP64 central differences."""
    rng = np.random.default_rng(5)
    R, t, d, l, u = _rand_obs(rng, 300)
    c = 0.01
    f = lambda R2, t2, d2, l2: O.F_obs(loss, c, R2, t2, d2, l2, u)
    fd = _tangent_fd(f, R, t, d, l)
    gt, gl, gd, gR = O.grad_F_obs(loss, c, R, t, d, l, u)
    scale = np.abs(gt).max()
    np.testing.assert_allclose(fd["t"], gt, atol=1e-7 * scale, rtol=1e-5)
    np.testing.assert_allclose(fd["l"], gl, atol=1e-7 * scale, rtol=1e-5)
    np.testing.assert_allclose(fd["d"], gd, atol=1e-7 * np.abs(gd).max(), rtol=1e-5)
    # tangent component of the ambient R gradient: d/dw F(R Exp(w)) = vee(skew(R^T G)) * 2 ... as a vector
    RtG = np.einsum("nba,nbc->nac", R, gR)
    S = RtG - np.transpose(RtG, (0, 2, 1))
    vee = np.stack([S[:, 2, 1], S[:, 0, 2], S[:, 1, 0]], 1)
    np.testing.assert_allclose(fd["R"], vee, atol=1e-7 * np.abs(vee).max(), rtol=1e-5)


def test_gradient_F_equals_gradient_E_at_xk():
    """Riemannian gradients of F and of E(. | x^k) agree at x^k (Eq. gradFij)."""
    rng = np.random.default_rng(9)
    R, t, d, l, u = _rand_obs(rng, 200)
    c = 0.01
    mj = O.majorizer("huber", c, R, t, d, l, u)
    fF = lambda R2, t2, d2, l2: O.F_obs("huber", c, R2, t2, d2, l2, u)
    fE = lambda R2, t2, d2, l2: O.P_obs(mj, R2, t2, d2, u) + O.Q_obs(mj, l2)
    a = _tangent_fd(fF, R, t, d, l)
    b = _tangent_fd(fE, R, t, d, l)
    for k in a:
        sc = max(np.abs(a[k]).max(), 1e-12)
        np.testing.assert_allclose(a[k], b[k], atol=2e-7 * sc)


# ----------------------------------------------------------------------------
# ProjRot3D (Eq. proj_rot3d) against an independent method
# ----------------------------------------------------------------------------

def _horn(Mx):
    """Independent second method: the maximiser of <R, M> over SO(3) is R(q) for the dominant
    eigenvector q of the 4x4 symmetric matrix N(M) with q^T N q = <R(q), M>."""
    out = []
    for K in Mx:
        N = np.array([
            [K[0, 0] + K[1, 1] + K[2, 2], K[2, 1] - K[1, 2], K[0, 2] - K[2, 0], K[1, 0] - K[0, 1]],
            [K[2, 1] - K[1, 2], K[0, 0] - K[1, 1] - K[2, 2], K[0, 1] + K[1, 0], K[0, 2] + K[2, 0]],
            [K[0, 2] - K[2, 0], K[0, 1] + K[1, 0], -K[0, 0] + K[1, 1] - K[2, 2], K[1, 2] + K[2, 1]],
            [K[1, 0] - K[0, 1], K[0, 2] + K[2, 0], K[1, 2] + K[2, 1], -K[0, 0] - K[1, 1] + K[2, 2]]])
        wv, V = np.linalg.eigh(N)
        w, x, y, z = V[:, -1]
        out.append([[w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y)],
                    [2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x)],
                    [2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z]])
    return np.array(out)


def test_proj_rot3d():
    rng = np.random.default_rng(2)
    Mx = rng.normal(size=(300, 3, 3))
    Mx[:100] *= -1.0    # many with det < 0
    R = O.proj_rot3d(Mx)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-12)
    np.testing.assert_allclose(np.einsum("nab,nac->nbc", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-12)
    np.testing.assert_allclose(R, _horn(Mx), atol=1e-9)
    Q = _rand_rot(rng, 50)
    np.testing.assert_allclose(O.proj_rot3d(Q), Q, atol=1e-13)            # idempotent on SO(3)
    A = rng.normal(size=(50, 3, 3))
    S = np.einsum("nab,ncb->nac", A, A) + 0.1 * np.eye(3)
    np.testing.assert_allclose(O.proj_rot3d(Q @ S), Q, atol=1e-10)        # polar factor of R S
    # brute force: no nearby rotation is closer to M
    for K, Rk in zip(Mx[:20], R[:20]):
        base = np.sum((Rk - K) ** 2)
        for _ in range(50):
            R2 = Rk @ O.so3_exp(rng.normal(scale=0.05, size=(1, 3)))[0]
            assert np.sum((R2 - K) ** 2) >= base - 1e-12


def test_nesterov_scalars():
    """s^0 = 1, gamma^0 = 0, gamma in [0, 1) and Eq. gamma_bnd gamma <= (s-1)/s."""
    s = 1.0
    s_next, g = O.nesterov(s)
    assert g == 0.0 and s_next == pytest.approx((np.sqrt(5.0) + 1) / 2, rel=1e-15)
    for k in range(2000):
        s_next, g = O.nesterov(s)
        assert 0.0 <= g < 1.0
        assert g <= (s - 1) / s + 1e-15
        assert s_next > s
        s = s_next
    assert s == pytest.approx(2001 / 2, rel=5e-3)    # s^k ~ (k + 1)/2 asymptotically


def _axis_rot(axis, phi):
    """Rotation by angle phi about the unit axis (Rodrigues' formula, written out here)."""
    K = np.array([[0.0, -axis[2], axis[1]], [axis[2], 0.0, -axis[0]], [-axis[1], axis[0], 0.0]])
    return np.eye(3) + np.sin(phi) * K + (1.0 - np.cos(phi)) * (K @ K)


def test_extrapolate_closed_form():
    """Eq. nesterov_x on a one-parameter subgroup. With R^(k-1) = R^k Exp(-theta a) (unit axis a),
    R^k + gamma (R^k - R^(k-1)) = R^k A with A = I + gamma (I - Exp(-theta a)), a polynomial in
    [a]x that fixes a and acts on the plane normal to a as (1 + gamma (1 - cos theta)) I
    + gamma sin theta J (J the quarter turn): a positive multiple of the rotation by
    phi = atan2(gamma sin theta, 1 + gamma (1 - cos theta)). Its projection onto SO(3) is
    therefore R^k Exp(phi a), exactly. t, d and l extrapolate affinely in gamma, and gamma = 0
    returns x^k."""
    rng = np.random.default_rng(12)
    Rk = _rand_rot(rng, 40)
    axes = rng.normal(size=(40, 3))
    axes /= np.linalg.norm(axes, axis=1, keepdims=True)
    theta = rng.uniform(0.0, 2.5, 40)
    gamma = rng.uniform(0.0, 0.99, 40)
    Rp = np.stack([Rk[n] @ _axis_rot(axes[n], -theta[n]) for n in range(40)])
    t, tp = rng.normal(size=(40, 3)), rng.normal(size=(40, 3))
    d, dp = rng.normal(size=(40, 3)), rng.normal(size=(40, 3))
    l, lp = rng.normal(size=(40, 3)), rng.normal(size=(40, 3))
    for n in range(40):
        g = gamma[n]
        Rb, tb, db, lb = O.extrapolate(Rk[n:n + 1], t[n:n + 1], d[n:n + 1], l[n:n + 1], Rp[n:n + 1], tp[n:n + 1],
                                       dp[n:n + 1], lp[n:n + 1], g)
        phi = np.arctan2(g * np.sin(theta[n]), 1.0 + g * (1.0 - np.cos(theta[n])))
        np.testing.assert_allclose(Rb[0], Rk[n] @ _axis_rot(axes[n], phi), atol=1e-12)
        np.testing.assert_allclose(tb[0], (1 + g) * t[n] - g * tp[n], atol=1e-13)
        np.testing.assert_allclose(db[0], (1 + g) * d[n] - g * dp[n], atol=1e-13)
        np.testing.assert_allclose(lb[0], (1 + g) * l[n] - g * lp[n], atol=1e-13)
    Rb, tb, db, lb = O.extrapolate(Rk, t, d, l, Rp, tp, dp, lp, 0.0)
    np.testing.assert_allclose(Rb, Rk, atol=1e-13)
    assert np.array_equal(tb, t) and np.array_equal(db, d) and np.array_equal(lb, l)
    # a wrong sign (x^(k-1) - x^k) would turn the other way: phi has the sign of gamma theta
    assert np.all(np.arctan2(gamma * np.sin(theta), 1.0 + gamma * (1.0 - np.cos(theta))) >= 0)


# ----------------------------------------------------------------------------
# subproblem solvers
# ----------------------------------------------------------------------------

def _small_problem(seed=0, loss="huber"):
    sc = cached_scene("circle")
    opts = O.Options(loss=loss, loss_scale_px=sc.loss_scale_px, xi=1e-6)
    return (sc,) + O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)


def test_landmark_solve_optimal():
    sc, prob, R, t, d, l = _small_problem()
    ci, li = prob.cam_idx, prob.lm_idx
    mj = O.majorizer(prob.loss, prob.c, R[ci], t[ci], d[ci], l[li], prob.u)
    xi = prob.opts.xi
    lz = l + 0.01
    ls = O.solve_landmarks(xi, mj, lz, li, prob.N)
    # zero gradient: xi (l - l_z) + 2 sum w lambda (lambda l - g) = 0
    res = (mj.lam[:, None] * ls[li] - mj.g) * (mj.w * mj.lam)[:, None]
    grad = xi * (ls - lz) + 2 * O.segsum(li, res, prob.N)
    assert np.abs(grad).max() < 1e-12
    E0 = O.E_lm(xi, mj, ls, lz, li, prob.N)
    rng = np.random.default_rng(0)
    for _ in range(5):
        E1 = O.E_lm(xi, mj, ls + rng.normal(scale=1e-4, size=ls.shape), lz, li, prob.N)
        assert np.all(E1 >= E0)


def test_camera_solve_steps():
    """Each S-CAM sub-step is an exact block minimiser: E never increases, the R-step satisfies
    the SO(3) optimality condition R^T K symmetric, and random perturbations do not improve it."""
    sc, prob, R, t, d, l = _small_problem()
    ci, li = prob.cam_idx, prob.lm_idx
    xi = prob.opts.xi
    rng = np.random.default_rng(4)
    Rz = R @ O.so3_exp(rng.normal(scale=0.01, size=(prob.M, 3)))
    tz = t + rng.normal(scale=0.05, size=t.shape)
    dz = d.copy()
    mj = O.majorizer(prob.loss, prob.c, Rz[ci], tz[ci], dz[ci], l[li], prob.u)
    prev = O.E_cam(xi, mj, Rz, tz, dz, Rz, tz, dz, ci, prob.u, prob.M)
    for n_alt in (1, 2, 3, 5):
        R2, t2, d2 = O.solve_cameras(xi, mj, Rz, tz, dz, ci, prob.u, prob.M, n_alt)
        E2 = O.E_cam(xi, mj, R2, t2, d2, Rz, tz, dz, ci, prob.u, prob.M)
        assert np.all(E2 <= prev + 1e-12 * np.abs(prev))
        prev = E2
    # the final (t, d)-step is exact: random (t, d) perturbations never lower E
    for _ in range(5):
        tp = t2 + rng.normal(scale=1e-5, size=t2.shape)
        dp = d2 + rng.normal(scale=1e-7, size=d2.shape)
        assert np.all(O.E_cam(xi, mj, R2, tp, dp, Rz, tz, dz, ci, prob.u, prob.M) >= prev - 1e-15 * np.abs(prev))
    # one more R-step from the final (t, d): R^T K symmetric at its solution
    p = O.ray(prob.u, d2[ci])
    v = 2.0 * mj.w[:, None] * (mj.g - mj.lam[:, None] * t2[ci])
    K = O.segsum(ci, v[:, :, None] * p[:, None, :], prob.M) + xi * Rz
    Rr = O.proj_rot3d(K)
    A = np.einsum("nba,nbc->nac", Rr, K)
    assert np.abs(A - np.transpose(A, (0, 2, 1))).max() < 1e-9 * np.abs(A).max()
    Er = O.E_cam(xi, mj, Rr, t2, d2, Rz, tz, dz, ci, prob.u, prob.M)
    for _ in range(5):
        Rq = Rr @ O.so3_exp(rng.normal(scale=1e-4, size=(prob.M, 3)))
        assert np.all(O.E_cam(xi, mj, Rq, t2, d2, Rz, tz, dz, ci, prob.u, prob.M) >= Er - 1e-15 * np.abs(Er))


def test_camera_solve_brute_force_tiny():
    """On a camera with three observations, the converged alternation matches a brute-force
    minimisation of E^alpha over (R, t, d) (scipy's general optimiser, independent of S-CAM)."""
    from scipy.optimize import minimize
    rng = np.random.default_rng(12)
    R, t, d, l, u = _rand_obs(rng, 5)
    R = np.repeat(R[:1], 5, 0)
    t = np.repeat(t[:1], 5, 0)
    d = np.repeat(d[:1], 5, 0)
    mj = O.majorizer("trivial", 1.0, R, t, d, l, u)
    ci = np.zeros(5, dtype=np.int64)
    xi = 1e-3
    Rz, tz, dz = R[:1], t[:1], d[:1]

    def Ef(x):
        Rx = Rz @ O.so3_exp(x[None, 0:3])
        return O.E_cam(xi, mj, Rx, x[None, 3:6], x[None, 6:9], Rz, tz, dz, ci, u, 1)[0]

    x0 = np.concatenate([np.zeros(3), tz[0], dz[0]])
    bf = minimize(Ef, x0, method="BFGS", options={"gtol": 1e-12, "maxiter": 5000})
    R2, t2, d2 = O.solve_cameras(xi, mj, Rz, tz, dz, ci, u, 1, 200)
    E2 = O.E_cam(xi, mj, R2, t2, d2, Rz, tz, dz, ci, u, 1)[0]
    assert E2 <= bf.fun * (1 + 1e-6) + 1e-14


def _lm_energy(xi, mj, Rz, tz, dz, ci, u, M, i, th):
    """E^alpha(c | z) of camera i at R = R_z Exp(phi), t = t_z + tau, d = d_z + delta (every other
    camera at its conditioning point)."""
    R, t, d = Rz.copy(), tz.copy(), dz.copy()
    R[i] = Rz[i] @ O.so3_exp(th[0:3])[0]
    t[i] = tz[i] + th[3:6]
    d[i] = dz[i] + th[6:9]
    return O.E_cam(xi, mj, R, t, d, Rz, tz, dz, ci, u, M)[i]


@pytest.mark.parametrize("noise_free", [False, True])
def test_lm_model_matches_surrogate_derivatives(noise_free):
    """The camera LM model: its gradient is the surrogate's gradient in (phi, tau, delta) by central
    differences; at a zero-residual point (noise-free truth, r(0) = 0) its Gauss-Newton Hessian is
    the exact Hessian (second differences)."""
    sc = cached_scene("circle", noise_free=noise_free)
    opts = O.Options(loss="huber", loss_scale_px=2.0, xi=1e-3)
    cams = sc.cams_gt if noise_free else sc.cams
    lms = sc.lms_gt if noise_free else sc.lms
    prob, R, t, d, l = O.make_problem(cams, lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    ci, li, u = prob.cam_idx, prob.lm_idx, prob.u
    mj = O.majorizer(prob.loss, prob.c, R[ci], t[ci], d[ci], l[li], u)
    A, b, r0, _ = O.lm_model(opts.xi, mj, R, t, d, ci, u, prob.M)
    scale = np.array([1e-3] * 3 + [1e-3] * 3 + [1e-3, 1e-3, 1e-3])
    for i in (0, 7):
        E = lambda th: _lm_energy(opts.xi, mj, R, t, d, ci, u, prob.M, i, th)
        g = np.array([(E(h * e) - E(-h * e)) / (2 * h) for e, h in zip(np.eye(9), scale * 1e-2)])
        if not noise_free:
            np.testing.assert_allclose(b[i], g, rtol=1e-5, atol=1e-7 * np.abs(b[i]).max())
            continue
        assert np.abs(r0).max() < 1e-9
        H = np.zeros((9, 9))
        for a in range(9):
            for c in range(9):
                ea, ec = np.eye(9)[a] * scale[a], np.eye(9)[c] * scale[c]
                H[a, c] = (E(ea + ec) - E(ea - ec) - E(-ea + ec) + E(-ea - ec)) / (4 * scale[a] * scale[c])
        np.testing.assert_allclose(A[i], H, rtol=1e-4, atol=1e-6 * np.abs(A[i]).max())


def test_lm_step_decreases_surrogate(circle):
    """One successful LM step lowers E^alpha(. | z) of every camera with a nonzero gradient."""
    sc = circle
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px)
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    ci, li, u = prob.cam_idx, prob.lm_idx, prob.u
    mj = O.majorizer(prob.loss, prob.c, R[ci], t[ci], d[ci], l[li], u)
    E0 = O.E_cam(opts.xi, mj, R, t, d, R, t, d, ci, u, prob.M)
    Rl, tl, dl = O.solve_cameras_lm(opts.xi, mj, R, t, d, ci, u, prob.M)
    El = O.E_cam(opts.xi, mj, Rl, tl, dl, R, t, d, ci, u, prob.M)
    assert np.all(El < E0)


# ----------------------------------------------------------------------------
# Algorithm 1: Lemma 1, Eq. FklFk0, DUBA monotonicity, convergence, fixed point
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("eta,solver", [(0.1, "scam"), (0.5, "scam"), (1.0, "scam"), (0.5, "lm")])
def test_algorithm1_invariants(circle, eta, solver):
    """Lemma 1a-c, Eq. FakplFk1 and Eq. FklFk0 every iteration, for both camera solvers (any
    solver that does not increase E^alpha(. | z) from c_z keeps them)."""
    sc = circle
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, eta=eta, xi=1e-8, cam_solver=solver)
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    st = O.init_state(prob, R, t, d, l)
    Fbar_global = O.objective(prob.loss, prob.c, R, t, d, l, prob.cam_idx, prob.lm_idx, prob.u)
    nrs = 0
    for k in range(25):
        prev = st
        st, info = O.step(prob, prev)
        F = info.F
        # Lemma 1a, 1b, 1c
        assert info.F_cam.sum() + info.F_lm.sum() == pytest.approx(F, rel=1e-11)
        Fbar_global = (1 - eta) * Fbar_global + eta * F
        assert info.Fbar_cam.sum() + info.Fbar_lm.sum() == pytest.approx(Fbar_global, rel=1e-11)
        assert np.all(info.F_cam <= prev.E_cam + 1e-12 * np.abs(prev.E_cam))
        assert np.all(info.F_lm <= prev.E_lm + 1e-12 * np.abs(prev.E_lm))
        # Eq. FakplFk1: E^alpha(k+1) <= Fbar^alpha(k)
        assert np.all(info.Enext_cam <= info.Fbar_cam + 1e-12 * np.abs(info.Fbar_cam))
        assert np.all(info.Enext_lm <= info.Fbar_lm + 1e-12 * np.abs(info.Fbar_lm))
        # Eq. FklFk0: F(x^(k+1)) - Fbar^(k) <= -xi/2 |x^(k+1) - x^k|^2
        Fn = O.objective(prob.loss, prob.c, st.R, st.t, st.d, st.l, prob.cam_idx, prob.lm_idx, prob.u)
        dx2 = O.cam_sqdist(st.R, st.t, st.d, prev.R, prev.t, prev.d).sum() + np.sum((st.l - prev.l) ** 2)
        assert Fn - Fbar_global <= -0.5 * opts.xi * dx2 + 1e-12 * Fbar_global
        nrs += int(info.restart_cam.sum() + info.restart_lm.sum())
        if k == 0:
            assert info.gamma == 0.0 and nrs == 0
    if eta >= 0.5:
        assert nrs > 0   # the adaptive restart is exercised on this scene


@pytest.mark.parametrize("eta,reset", [(0.5, False), (1.0, False), (0.5, True)])
def test_global_restart_invariants(circle, eta, reset):
    """Global restart variant: Lemma 1 and Eq. FklFk0 for the single block made of everything
    (the sums of the block metrics), all-or-nothing decisions, a monotone objective at eta = 1
    (then Fbar = F), and gamma = 0 after a restart when the momentum is reset."""
    sc = circle
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, eta=eta, xi=1e-8, restart="global",
                     momentum_reset=reset)
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    st = O.init_state(prob, R, t, d, l)
    Fbar = O.objective(prob.loss, prob.c, R, t, d, l, prob.cam_idx, prob.lm_idx, prob.u)
    fired, gammas, F_prev = [], [], None
    for k in range(40):
        prev = st
        st, info = O.step(prob, prev)
        F = info.F
        gammas.append(info.gamma)
        assert info.F_cam.sum() + info.F_lm.sum() == pytest.approx(F, rel=1e-11)
        Fbar = (1 - eta) * Fbar + eta * F
        assert info.Fbar_cam.sum() + info.Fbar_lm.sum() == pytest.approx(Fbar, rel=1e-11)
        rc, rl = info.restart_cam, info.restart_lm
        assert (rc.all() and rl.all()) or not (rc.any() or rl.any())
        fired.append(bool(rc.all()))
        # the restart test of the single block: sum E(k+1) <= sum Fbar(k)
        assert info.Enext_cam.sum() + info.Enext_lm.sum() <= Fbar + 1e-12 * abs(Fbar)
        Fn = O.objective(prob.loss, prob.c, st.R, st.t, st.d, st.l, prob.cam_idx, prob.lm_idx, prob.u)
        dx2 = O.cam_sqdist(st.R, st.t, st.d, prev.R, prev.t, prev.d).sum() + np.sum((st.l - prev.l) ** 2)
        assert Fn - Fbar <= -0.5 * opts.xi * dx2 + 1e-12 * Fbar
        if eta == 1.0:
            assert Fn <= F * (1 + 1e-12)
        F_prev = F
    assert any(fired) and not all(fired)
    for k in range(1, 40):
        if reset and fired[k - 1]:
            assert gammas[k] == 0.0
        elif k > 1 and not reset:
            assert gammas[k] > 0.0


@pytest.mark.parametrize("loss,solver", [("trivial", "scam"), ("huber", "scam"), ("cauchy", "scam"),
                                         ("welsch", "scam"), ("huber", "lm")])
def test_duba_monotone(loss, solver):
    """DUBA (always the MM update, Sec. 7.2) never increases F (Sec. 4)."""
    sc = cached_scene("circle")
    opts = O.Options(loss=loss, loss_scale_px=2.0, accelerated=False, cam_solver=solver)
    res = O.daba(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts, 15)
    assert np.all(np.diff(res.trace_px2) <= 1e-12 * res.trace_px2[:-1])
    assert res.trace_px2[-1] < 0.9 * res.trace_px2[0]


def test_daba_faster_than_duba(circle):
    sc = circle
    a = O.daba(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, O.Options(loss=sc.loss), 30)
    b = O.daba(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, O.Options(loss=sc.loss, accelerated=False), 30)
    assert a.trace_px2[-1] < b.trace_px2[-1]


def test_noise_free_converges_to_zero():
    """Noise-free observations: DABA drives the objective towards zero (Eq. err0)."""
    sc = cached_scene("circle", noise_free=True)
    opts = O.Options(loss="trivial")
    res = O.daba(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts, 150)
    assert res.trace_px2[-1] < 1e-3 * res.trace_px2[0]
    assert np.all(np.isfinite(res.trace_px2))


def test_fixed_point_at_truth():
    """At the noise-free ground truth every block's subproblem is already solved."""
    sc = cached_scene("circle", noise_free=True)
    opts = O.Options(loss="huber")
    res = O.daba(sc.cams_gt, sc.lms_gt, sc.cam_idx, sc.lm_idx, sc.uv, opts, 3)
    cams, lms = O.boundary_state(res)
    np.testing.assert_allclose(lms, sc.lms_gt, atol=1e-9)
    np.testing.assert_allclose(cams, sc.cams_gt, atol=1e-8)
    assert res.trace_px2.max() < 1e-14 * sc.nnz


@pytest.mark.parametrize("loss", ["huber", "cauchy", "trivial"])
def test_boundary_gradient_fd(loss):
    """Gradient of F (pixel^2) w.r.t. the boundary cameras [w, t, f, k1, k2], landmarks and pixels
    against FP64 central differences of the objective along random directions."""
    from paper_2305_07026_b300 import scenes
    sc = scenes.circle_scene(seed=11, n_cams=6, n_lms=40, cap=6)
    o = O.Options(loss=loss, loss_scale_px=2.0)
    F, gc, gl, gu = O.grad_objective_boundary(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, o)

    def Fx(c, l, u):
        prob, R, t, d, lm = O.make_problem(c, l, sc.cam_idx, sc.lm_idx, u, o)
        return O.objective(prob.loss, prob.c, R, t, d, lm, prob.cam_idx, prob.lm_idx, prob.u) * prob.s_norm ** 2

    assert F == pytest.approx(Fx(sc.cams, sc.lms, sc.uv), rel=1e-14)
    rng = np.random.default_rng(3)
    cscale = np.array([1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 0.5, 1e-4, 1e-6])
    for _ in range(16):
        vc = rng.normal(size=sc.cams.shape) * cscale
        vl = rng.normal(size=sc.lms.shape) * 1e-3
        vu = rng.normal(size=sc.uv.shape) * 1e-2
        h = 1e-3
        fd = (Fx(sc.cams + h * vc, sc.lms + h * vl, sc.uv + h * vu) -
              Fx(sc.cams - h * vc, sc.lms - h * vl, sc.uv - h * vu)) / (2 * h)
        an = np.sum(gc * vc) + np.sum(gl * vl) + np.sum(gu * vu)
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(F))
    # each block separately (a wrong chain rule in one part cannot hide behind the others)
    for part in range(3):
        v = [np.zeros_like(sc.cams), np.zeros_like(sc.lms), np.zeros_like(sc.uv)]
        v[part] = rng.normal(size=v[part].shape) * (cscale if part == 0 else (1e-3 if part == 1 else 1e-2))
        h = 1e-3
        fd = (Fx(sc.cams + h * v[0], sc.lms + h * v[1], sc.uv + h * v[2]) -
              Fx(sc.cams - h * v[0], sc.lms - h * v[1], sc.uv - h * v[2])) / (2 * h)
        an = np.sum(gc * v[0]) + np.sum(gl * v[1]) + np.sum(gu * v[2])
        assert an == pytest.approx(fd, rel=1e-6), part
    # each camera parameter column separately
    for k in range(9):
        v = np.zeros_like(sc.cams)
        v[:, k] = rng.normal(size=sc.M) * cscale[k]
        h = 1e-3
        fd = (Fx(sc.cams + h * v, sc.lms, sc.uv) - Fx(sc.cams - h * v, sc.lms, sc.uv)) / (2 * h)
        assert np.sum(gc * v) == pytest.approx(fd, rel=1e-5, abs=1e-12 * abs(F)), k


@pytest.mark.parametrize("loss,accel,K,solver", [("huber", True, 6, "scam"), ("cauchy", True, 12, "scam"),
                                                 ("trivial", False, 8, "scam"), ("huber", True, 6, "lm"),
                                                 ("cauchy", False, 5, "lm"), ("huber", True, 15, "scam-reset"),
                                                 ("trivial", True, 14, "lm-reset")])
def test_unrolled_gradient_fd(loss, accel, K, solver):
    """Gradient of a linear functional of the state after K iterations (autograd through the
    PyTorch restatement of the update, restart decisions and, with the LM camera solver, the
    taken damping trials fixed) against FP64 central differences of the numpy oracle's
    K-iteration map along random directions."""
    from oracle import daba_unrolled as U
    from paper_2305_07026_b300 import scenes
    sc = scenes.circle_scene(seed=11, n_cams=6, n_lms=40, cap=6)
    kw = {}
    if solver.endswith("-reset"):   # global restart with the momentum reset: one restart fires within K
        solver = solver[:-6]
        kw = dict(restart="global", momentum_reset=True)
    o = O.Options(loss=loss, loss_scale_px=2.0, accelerated=accel, pixel_scale=650.0, cam_solver=solver, **kw)
    rng = np.random.default_rng(4)
    g_c, g_l = rng.normal(size=sc.cams.shape), rng.normal(size=sc.lms.shape)
    gc, gl, gu, oc, ol, res = U.unrolled_grad(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, o, K, g_c, g_l)
    if kw:
        assert any(np.all(i.restart_cam) for i in res.infos[:K - 1])
    cams_o, lms_o = O.boundary_state(res)
    np.testing.assert_allclose(oc, cams_o, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(ol, lms_o, rtol=1e-9, atol=1e-9)

    def J(c, l, u):
        r = O.daba(c, l, sc.cam_idx, sc.lm_idx, u, o, K)
        cc, ll = O.boundary_state(r)
        return float(np.sum(cc * g_c) + np.sum(ll * g_l))

    cscale = np.array([1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 0.5, 1e-4, 1e-6])
    for part in range(3):
        v = [np.zeros_like(sc.cams), np.zeros_like(sc.lms), np.zeros_like(sc.uv)]
        v[part] = rng.normal(size=v[part].shape) * (cscale if part == 0 else (1e-3 if part == 1 else 1e-2))
        # steps above the rounding noise of J and below the curvature of each part
        h = (1e-3, 1e-2, 1e-2)[part]
        fd = (J(sc.cams + h * v[0], sc.lms + h * v[1], sc.uv + h * v[2]) -
              J(sc.cams - h * v[0], sc.lms - h * v[1], sc.uv - h * v[2])) / (2 * h)
        an = np.sum(gc * v[0]) + np.sum(gl * v[1]) + np.sum(gu * v[2])
        assert an == pytest.approx(fd, rel=1e-5, abs=1e-9), part
