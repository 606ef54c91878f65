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


def _run(obs_eval, bits, loss, seed, n, c):
    """The driver's 13 values per observation and the oracle's counterparts on the same inputs."""
    R, t, d, Rp, tp, dp, l, lp, u, gamma = _inputs(seed, n, c)
    ext = [O.extrapolate(R[i:i + 1], t[i:i + 1], d[i:i + 1], l[i:i + 1], Rp[i:i + 1], tp[i:i + 1], dp[i:i + 1],
                         lp[i:i + 1], float(gamma[i])) for i in range(n)]
    Rb, tb, db, lb = (np.concatenate([x[k] for x in ext]) for k in range(4))
    rows = np.concatenate([R.reshape(n, 9), t, d, Rp.reshape(n, 9), tp, dp, Rb.reshape(n, 9), l, lp, u,
                           gamma[:, None]], 1)
    stdin = (f"{bits} {LOSSES[loss]} {c!r} {n}\n"
             + "\n".join(" ".join(repr(float(x)) for x in row) for row in rows) + "\n")
    run = subprocess.run([obs_eval], input=stdin, capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stderr[-2000:]
    dev = np.array([[float(x) for x in line.split()] for line in run.stdout.splitlines()])
    assert dev.shape == (n, 13)
    ora = {}
    # x^k
    p = O.ray(u, d)
    ora["p_norm"] = np.linalg.norm(p, axis=1)
    ora["lam"] = O.lam(R, t, l, p)
    e = O.reproj_error(R, t, l, p)
    ora["r"] = np.einsum("na,na->n", e, e)
    ora["rho"], ora["w"] = O.rho(loss, c, ora["r"])
    ora["Re"] = np.einsum("nab,nb->na", R, e)
    # extrapolated iterate (Eq. nesterov_x, the rotation through ProjRot3D)
    pb = O.ray(u, db)
    ora["pb_norm"] = np.linalg.norm(pb, axis=1)
    ora["lamb"] = O.lam(Rb, tb, lb, pb)
    eb = O.reproj_error(Rb, tb, lb, pb)
    _, ora["wb"] = O.rho(loss, c, np.einsum("na,na->n", eb, eb))
    ora["Reb"] = np.einsum("nab,nb->na", Rb, eb)
    # surrogate gap with the majorizer built at x^(k-1)
    mj = O.majorizer(loss, c, Rp, tp, dp, lp, u)
    ora["PQ"] = O.P_obs(mj, R, t, d, u) + O.Q_obs(mj, l)
    ora["gap"] = 0.5 * ora["rho"] - ora["PQ"]
    return dev, ora


@pytest.mark.parametrize("loss", sorted(LOSSES))
def test_eval_obs_matches_oracle(obs_eval, loss):
    """FP64: the same quantities to rounding."""
    dev, ora = _run(obs_eval, 64, loss, 11 + LOSSES[loss], 400, 0.02)
    close = dict(rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(dev[:, 0], ora["lam"], **close)
    np.testing.assert_allclose(dev[:, 1:4], ora["Re"], rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(dev[:, 4], ora["r"], rtol=1e-9, atol=1e-16)
    np.testing.assert_allclose(dev[:, 5], ora["rho"], rtol=1e-9, atol=1e-16)
    np.testing.assert_allclose(dev[:, 6], ora["w"], **close)
    np.testing.assert_allclose(dev[:, 7], ora["lamb"], **close)
    np.testing.assert_allclose(dev[:, 8:11], ora["Reb"], rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(dev[:, 11], ora["wb"], **close)
    # the oracle forms the gap as a difference of O(P + Q) values; the library without cancellation
    np.testing.assert_allclose(dev[:, 12], ora["gap"], rtol=0, atol=1e-12 * max(1.0, float(np.max(ora["PQ"]))))
    assert np.all(dev[:, 12] <= 1e-12)   # Proposition 1: P + Q majorizes F


# FP32 error bounds of the MIXED pass (ten times what the host build of the same code shows on
# 2,000 observations per loss; the GPU's approximate division and reciprocal square root add a few
# ulp): lambda relative; R e, Rbar ebar relative to the ray length |p| (e is a small difference of
# O(|p|) vectors); r = |e|^2 and rho relative to |p| |e|; the weights relative (absolute below
# 1e-6); the gap relative to P + Q, the size of the terms it is the difference of
FP32_BOUNDS = {"lam": 5e-6, "Re": 4e-6, "r": 6e-6, "w": 2e-3, "gap": 3e-4}


@pytest.mark.parametrize("loss", sorted(LOSSES))
def test_eval_obs_fp32_error(obs_eval, loss):
    dev, ora = _run(obs_eval, 32, loss, 31 + LOSSES[loss], 2000, 0.02)
    e_norm = np.sqrt(ora["r"])
    err = {
        "lam": max(np.max(np.abs(dev[:, 0] / ora["lam"] - 1)), np.max(np.abs(dev[:, 7] / ora["lamb"] - 1))),
        "Re": max(np.max(np.linalg.norm(dev[:, 1:4] - ora["Re"], axis=1) / ora["p_norm"]),
                  np.max(np.linalg.norm(dev[:, 8:11] - ora["Reb"], axis=1) / ora["pb_norm"])),
        "r": max(np.max(np.abs(dev[:, 4] - ora["r"]) / (ora["p_norm"] * e_norm)),
                 np.max(np.abs(dev[:, 5] - ora["rho"]) / (ora["p_norm"] * e_norm))),
        # weights below 1e-6 (Welsch far out, down to FP32 underflow) are compared absolutely
        "w": max(np.max(np.abs(dev[:, 6] - ora["w"]) / np.maximum(ora["w"], 1e-6)),
                 np.max(np.abs(dev[:, 11] - ora["wb"]) / np.maximum(ora["wb"], 1e-6))),
        "gap": np.max(np.abs(dev[:, 12] - ora["gap"]) / ora["PQ"]),
    }
    for k, bound in FP32_BOUNDS.items():
        assert err[k] <= bound, f"{loss} {k}: {err[k]:.2e} > {bound:.0e}"
