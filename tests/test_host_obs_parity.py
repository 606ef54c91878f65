"""Parity of the per-observation evaluation on the CPU: the library's eval_obs (FP64, the code
nvcc compiles for the camera pass) built for the host with g++ and fed the same seeded inputs as
the oracle's Eqs. ray, lambdaij, error, the losses of Assumption 1, the extrapolation of
Eq. nesterov_x and the majorizer of Proposition 1 (Eqs. P, Q). Compared per observation:
lambda, R e, |e|^2, rho, w at x^k; lambda, Rbar ebar, w at the extrapolated iterate; and the
surrogate gap F_ij(x^k) - P_ij(c^k | x^(k-1)) - Q_ij(l^k | x^(k-1)). No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import daba_oracle as O
from tests.test_host_device_math import FLAGS, HOST

LOSSES = {"trivial": 0, "huber": 1, "cauchy": 2, "welsch": 3}


@pytest.fixture(scope="module")
def obs_eval(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("obs_eval") / "obs_eval")
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, "obs_eval.cpp"), "-o", exe], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    return exe


def _inputs(seed, n, c):
    """Cameras, their previous iterate and landmarks in front of them along the observed rays,
    displaced so that |e|^2 falls on both sides of the loss scale c^2 (internal units)."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(-1.0, 1.0, (n, 3))
    R = O.so3_exp(w)
    t = rng.uniform(-1.0, 1.0, (n, 3))
    d = np.stack([1.0 + 0.1 * rng.uniform(-1, 1, n), 0.1 * rng.uniform(-1, 1, n), 0.05 * rng.uniform(-1, 1, n)], 1)
    u = rng.uniform(-0.5, 0.5, (n, 2))
    lam_t = rng.uniform(2.0, 6.0, n)
    spread = np.where(np.arange(n) % 2 == 0, 0.05, 0.005) * c / 0.02
    l = t + np.einsum("nab,nb->na", R, O.ray(u, d)) / lam_t[:, None] + spread[:, None] * rng.uniform(-1, 1, (n, 3))
    Rp = O.so3_exp(w + 0.02 * rng.uniform(-1, 1, (n, 3)))
    tp = t + 0.01 * rng.uniform(-1, 1, (n, 3))
    dp = d + np.array([1e-3, 1e-3, 1e-4]) * rng.uniform(-1, 1, (n, 3))
    lp = l + 0.01 * rng.uniform(-1, 1, (n, 3))
    gamma = rng.uniform(0.0, 0.9, n)
    return R, t, d, Rp, tp, dp, l, lp, u, gamma


@pytest.mark.parametrize("loss", sorted(LOSSES))
def test_eval_obs_matches_oracle(obs_eval, loss):
    n, c = 400, 0.02
    R, t, d, Rp, tp, dp, l, lp, u, gamma = _inputs(11 + LOSSES[loss], n, c)
    ext = [O.extrapolate(R[i:i + 1], t[i:i + 1], d[i:i + 1], l[i:i + 1], Rp[i:i + 1], tp[i:i + 1], dp[i:i + 1],
                         lp[i:i + 1], float(gamma[i])) for i in range(n)]
    Rb, tb, db, lb = (np.concatenate([x[k] for x in ext]) for k in range(4))
    rows = np.concatenate([R.reshape(n, 9), t, d, Rp.reshape(n, 9), tp, dp, Rb.reshape(n, 9), l, lp, u,
                           gamma[:, None]], 1)
    stdin = f"{LOSSES[loss]} {c!r} {n}\n" + "\n".join(" ".join(repr(float(x)) for x in row) for row in rows) + "\n"
    run = subprocess.run([obs_eval], input=stdin, capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stderr[-2000:]
    dev = np.array([[float(x) for x in line.split()] for line in run.stdout.splitlines()])
    assert dev.shape == (n, 13)

    # x^k
    p = O.ray(u, d)
    lam = O.lam(R, t, l, p)
    e = O.reproj_error(R, t, l, p)
    r = np.einsum("na,na->n", e, e)
    rho, w = O.rho(loss, c, r)
    Re = np.einsum("nab,nb->na", R, e)
    # extrapolated iterate (Eq. nesterov_x, the rotation through ProjRot3D)
    pb = O.ray(u, db)
    lamb = O.lam(Rb, tb, lb, pb)
    eb = O.reproj_error(Rb, tb, lb, pb)
    _, wb = O.rho(loss, c, np.einsum("na,na->n", eb, eb))
    Reb = np.einsum("nab,nb->na", Rb, eb)
    # surrogate gap with the majorizer built at x^(k-1)
    mj = O.majorizer(loss, c, Rp, tp, dp, lp, u)
    P, Q = O.P_obs(mj, R, t, d, u), O.Q_obs(mj, l)
    gap = 0.5 * rho - P - Q

    close = dict(rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(dev[:, 0], lam, **close)
    np.testing.assert_allclose(dev[:, 1:4], Re, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(dev[:, 4], r, rtol=1e-9, atol=1e-16)
    np.testing.assert_allclose(dev[:, 5], rho, rtol=1e-9, atol=1e-16)
    np.testing.assert_allclose(dev[:, 6], w, **close)
    np.testing.assert_allclose(dev[:, 7], lamb, **close)
    np.testing.assert_allclose(dev[:, 8:11], Reb, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(dev[:, 11], wb, **close)
    # the oracle forms the gap as a difference of O(P + Q) values; the library without cancellation
    np.testing.assert_allclose(dev[:, 12], gap, rtol=0, atol=1e-12 * max(1.0, float(np.max(P + Q))))
    assert np.all(dev[:, 12] <= 1e-12)   # Proposition 1: P + Q majorizes F
