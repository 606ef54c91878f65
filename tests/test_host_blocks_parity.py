"""Parity of the coarse-block solve's per-pair math on the CPU: the library's blk_intra_jac,
blk_F and sym3_inv (the code nvcc compiles into the block solve, k_blk_solve) built for the host
with g++ and fed seeded inputs. For an intra-block pair (camera and landmark in one block, whose
exact F_ij stays in Eq. Ealpha) the solve's Gauss-Newton model needs R e (Eqs. lambdaij, error)
and its Jacobians with respect to the camera step (R Exp(phi), t + tau, d + delta) and the
landmark step (l + epsilon). Checked here:
  * R e and F_ij = rho(|e|^2)/2 against the oracle's Eq. error and Eq. Fij, per loss;
  * the Jacobians against central differences of the library's own residual (a pin that does
    not go through the oracle) and against the block oracle's intra_residual_jacobian;
  * the packed 3 x 3 inverse of a landmark's damped block against numpy.
No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import daba_blocks as B
from oracle import daba_oracle as O
from tests.test_host_device_math import FLAGS, HOST

LOSSES = {"trivial": 0, "huber": 1, "cauchy": 2, "welsch": 3}


@pytest.fixture(scope="module")
def blk_pair(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("blk_pair") / "blk_pair")
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, "blk_pair.cpp"), "-o", exe], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    return exe


def _call(exe, stdin, width):
    run = subprocess.run([exe], input=stdin, capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stderr[-2000:]
    out = np.array([[float(x) for x in line.split()] for line in run.stdout.splitlines()])
    assert out.shape[1] == width
    return out


def _pairs(exe, loss, c, R, t, d, l, u):
    """The driver's R e (n, 3), Jc (n, 3, 9), Jl (n, 3, 3) and F (n) on these pairs."""
    n = R.shape[0]
    rows = np.concatenate([R.reshape(n, 9), t, d, l, u], 1)
    stdin = (f"pair {LOSSES[loss]} {c!r} {n}\n"
             + "\n".join(" ".join(repr(float(x)) for x in row) for row in rows) + "\n")
    out = _call(exe, stdin, 3 + 27 + 9 + 1)
    return out[:, 0:3], out[:, 3:30].reshape(n, 3, 9), out[:, 30:39].reshape(n, 3, 3), out[:, 39]


def _inputs(seed, n, c):
    """Cameras with landmarks near their observed rays (|e|^2 on both sides of c^2, internal units)."""
    rng = np.random.default_rng(seed)
    R = O.so3_exp(rng.uniform(-1.0, 1.0, (n, 3)))
    t = rng.uniform(-1.0, 1.0, (n, 3))
    d = np.stack([1.0 + 0.1 * rng.uniform(-1, 1, n), 0.1 * rng.uniform(-1, 1, n), 0.05 * rng.uniform(-1, 1, n)], 1)
    u = rng.uniform(-0.5, 0.5, (n, 2))
    lam_t = rng.uniform(2.0, 6.0, n)
    spread = np.where(np.arange(n) % 2 == 0, 0.05, 0.005) * c / 0.02
    l = t + np.einsum("nab,nb->na", R, O.ray(u, d)) / lam_t[:, None] + spread[:, None] * rng.uniform(-1, 1, (n, 3))
    return R, t, d, l, u


@pytest.mark.parametrize("loss", list(LOSSES))
def test_intra_pair_residual_and_F_match_oracle(blk_pair, loss):
    """R e and F_ij of the block solve equal the oracle's Eq. error (rotated into the world
    frame) and Eq. Fij on 300 seeded pairs per loss."""
    c = 0.02
    R, t, d, l, u = _inputs(11 + LOSSES[loss], 300, c)
    f, _, _, F = _pairs(blk_pair, loss, c, R, t, d, l, u)
    Re = np.einsum("nab,nb->na", R, O.reproj_error(R, t, l, O.ray(u, d)))
    np.testing.assert_allclose(f, Re, rtol=0, atol=1e-13)
    Fo = O.F_obs(loss, c, R, t, d, l, u)
    np.testing.assert_allclose(F, Fo, rtol=1e-12, atol=1e-20)
    # both sides of the loss scale are exercised
    r = np.einsum("na,na->n", Re, Re)
    assert (r > c * c).any() and (r < c * c).any()


def test_intra_pair_jacobian_central_differences(blk_pair):
    """The Jacobians of R e with respect to (phi, tau, delta) and epsilon equal central
    differences of the library's own residual at R Exp(+-h e_k), t +- h e_k, d +- h e_k,
    l +- h e_k (h = 1e-6), relative to the largest entry of each pair's Jacobian."""
    n, h = 120, 1e-6
    R, t, d, l, u = _inputs(5, n, 0.02)
    _, Jc, Jl, _ = _pairs(blk_pair, "trivial", 1.0, R, t, d, l, u)
    J = np.concatenate([Jc, Jl], 2)   # (n, 3, 12)
    # all 24 perturbed copies of every pair in one call
    Rs, ts, ds, ls = [], [], [], []
    for k in range(12):
        for sgn in (1.0, -1.0):
            e = np.zeros(3)
            e[k % 3] = sgn * h
            Rk, tk, dk, lk = R, t, d, l
            if k < 3:
                Rk = np.einsum("nab,bc->nac", R, O.so3_exp(e[None])[0])
            elif k < 6:
                tk = t + e
            elif k < 9:
                dk = d + e
            else:
                lk = l + e
            Rs.append(Rk), ts.append(tk), ds.append(dk), ls.append(lk)
    fp, _, _, _ = _pairs(blk_pair, "trivial", 1.0, np.concatenate(Rs), np.concatenate(ts), np.concatenate(ds),
                         np.concatenate(ls), np.tile(u, (24, 1)))
    fp = fp.reshape(12, 2, n, 3)
    fd = np.transpose((fp[:, 0] - fp[:, 1]) / (2 * h), (1, 2, 0))   # (n, 3, 12)
    scale = np.abs(fd).max(axis=(1, 2))
    err = np.abs(J - fd).max(axis=(1, 2)) / scale
    assert err.max() < 1e-7, err.max()


def test_intra_pair_jacobian_matches_block_oracle(blk_pair):
    """The same Jacobians against the block oracle's intra_residual_jacobian (the model its LM
    step builds), to rounding."""
    R, t, d, l, u = _inputs(23, 200, 0.02)
    f, Jc, Jl, _ = _pairs(blk_pair, "huber", 0.02, R, t, d, l, u)
    fo, Jo = B.intra_residual_jacobian(R, t, d, l, u)
    np.testing.assert_allclose(f, fo, rtol=0, atol=1e-13)
    scale = np.abs(Jo).max(axis=(1, 2))[:, None, None]
    np.testing.assert_allclose(np.concatenate([Jc, Jl], 2) / scale, Jo / scale, rtol=0, atol=1e-12)


def test_sym3_inverse(blk_pair):
    """A landmark's damped 3 x 3 block (packed xx, yx, yy, zx, zy, zz) inverted by the block
    solve equals numpy's inverse, for well- and poorly-conditioned (up to 1e6) SPD matrices."""
    rng = np.random.default_rng(3)
    mats = []
    for i in range(200):
        A = rng.normal(size=(3, 3))
        ev = 10.0 ** rng.uniform(-3, 3, 3) if i % 2 else rng.uniform(0.5, 2.0, 3)
        Q, _ = np.linalg.qr(A)
        mats.append(Q @ np.diag(ev) @ Q.T)
    mats = np.array(mats)
    packed = mats[:, [0, 1, 1, 2, 2, 2], [0, 0, 1, 0, 1, 2]]
    stdin = f"sym3 {len(mats)}\n" + "\n".join(" ".join(repr(float(x)) for x in row) for row in packed) + "\n"
    inv = _call(blk_pair, stdin, 6)
    ref = np.linalg.inv(mats)[:, [0, 1, 1, 2, 2, 2], [0, 0, 1, 0, 1, 2]]
    cond = np.linalg.cond(mats)
    err = np.abs(inv - ref).max(axis=1) / np.abs(ref).max(axis=1)
    # the cofactor formula and LU each carry an error of a small multiple of cond * 2^-52
    assert (err < 2e-13 * cond).all(), (err / cond).max()
    assert err[cond < 10].max() < 1e-14
