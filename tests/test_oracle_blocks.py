"""Pins of the coarse-block oracle (oracle/daba_blocks.py: Algorithm 1 with blocks of many
cameras and landmarks, Eq. Ealpha with E' not empty) against what the paper and the mathematics
fix: the Jacobian of the intra-pair residual against central differences, Proposition 2 for
multi-element blocks (the block surrogates majorize F and touch it at the conditioning iterate),
the Gauss-Newton model's gradient against central differences of the surrogate, the LM step
never raising a block's surrogate, Lemma 1 and Eq. FklFk0 every iteration, the unaccelerated
iteration's monotone objective, the noise-free scene, and the ground truth as a fixed point."""
import numpy as np
import pytest

from oracle import daba_blocks as B
from oracle import daba_oracle as O


def _scene():
    from paper_2305_07026_b300 import scenes
    return scenes.circle_scene(n_lms=240)


def _problem(sc, n_blocks, **kw):
    opts = O.Options(**{"loss": sc.loss, "loss_scale_px": sc.loss_scale_px, **kw})
    prob, R, t, d, l = O.make_problem(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts)
    part = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, n_blocks)
    return prob, part, R, t, d, l


def _perturb(rng, R, t, d, l, scale):
    Rx = np.einsum("nab,nbc->nac", R, O.so3_exp(rng.normal(scale=scale, size=(R.shape[0], 3))))
    return (Rx, t + rng.normal(scale=scale, size=t.shape), d + rng.normal(scale=scale * 1e-2, size=d.shape),
            l + rng.normal(scale=scale, size=l.shape))


def test_partition_has_intra_and_inter_pairs():
    sc = _scene()
    prob, part, *_ = _problem(sc, 4)
    isin = B.intra(part, prob.cam_idx, prob.lm_idx)
    assert part.S == 4 and 0.1 < isin.mean() < 0.9
    # every observed landmark sits in the block of one of its observing cameras
    owner_seen = np.zeros(sc.N, bool)
    np.logical_or.at(owner_seen, prob.lm_idx, isin)
    assert owner_seen[np.unique(prob.lm_idx)].all()


def test_intra_jacobian_central_differences():
    rng = np.random.default_rng(3)
    sc = _scene()
    prob, part, R, t, d, l = _problem(sc, 4)
    ci, li, u = prob.cam_idx[:60], prob.lm_idx[:60], prob.u[:60]
    f0, J = B.intra_residual_jacobian(R[ci], t[ci], d[ci], l[li], u)
    h = 1e-6
    for k in range(12):
        e = np.zeros(12)
        e[k] = h
        out = []
        for sgn in (1.0, -1.0):
            th = sgn * e
            Rx = np.einsum("nab,nbc->nac", R[ci], O.so3_exp(np.broadcast_to(th[0:3], (ci.size, 3))))
            fx, _ = B.intra_residual_jacobian(Rx, t[ci] + th[3:6], d[ci] + th[6:9], l[li] + th[9:12], u)
            out.append(fx)
        fd = (out[0] - out[1]) / (2 * h)
        # the differences of O(1) rays leave about 1e-16 / h = 1e-10 of rounding in the quotient
        np.testing.assert_allclose(J[:, :, k], fd, rtol=1e-6, atol=1e-9)
    # R e has the length of e (Eq. error)
    e = O.reproj_error(R[ci], t[ci], l[li], O.ray(u, d[ci]))
    np.testing.assert_allclose(np.linalg.norm(f0, axis=1), np.linalg.norm(e, axis=1), rtol=1e-12)


@pytest.mark.parametrize("loss", ["huber", "cauchy", "trivial"])
def test_block_surrogates_majorize(loss):
    """Proposition 2: sum_alpha E^alpha(x | z) >= F(x) with equality at x = z."""
    rng = np.random.default_rng(5)
    sc = _scene()
    prob, part, R, t, d, l = _problem(sc, 4, loss=loss)
    isin = B.intra(part, prob.cam_idx, prob.lm_idx)
    ci, li = prob.cam_idx, prob.lm_idx
    Ez = B.E_blocks_at(prob, part, isin, R, t, d, l)
    F = O.objective(prob.loss, prob.c, R, t, d, l, ci, li, prob.u)
    assert Ez.sum() == pytest.approx(F, rel=1e-13)
    mj = O.majorizer(prob.loss, prob.c, R[ci], t[ci], d[ci], l[li], prob.u)
    for scale in (1e-4, 1e-3, 1e-2, 5e-2):
        Rx, tx, dx, lx = _perturb(rng, R, t, d, l, scale)
        Ex = Ez + B.dE_blocks(prob, part, isin, mj, Rx, tx, dx, lx, R, t, d, l)
        Fx = O.objective(prob.loss, prob.c, Rx, tx, dx, lx, ci, li, prob.u)
        assert Ex.sum() >= Fx - 1e-12 * Fx
    # the surrogate of the single block made of everything is F itself plus the proximal term
    one = B.make_partition(np.zeros(sc.M, int), np.zeros(sc.N, int))
    Rx, tx, dx, lx = _perturb(rng, R, t, d, l, 1e-2)
    E1 = B.dE_blocks(prob, one, B.intra(one, ci, li), mj, Rx, tx, dx, lx, R, t, d, l)[0] + F
    prox = 0.5 * prob.opts.xi * (O.cam_sqdist(Rx, tx, dx, R, t, d).sum() + np.sum((lx - l) ** 2))
    assert E1 == pytest.approx(O.objective(prob.loss, prob.c, Rx, tx, dx, lx, ci, li, prob.u) + prox, rel=1e-12)


@pytest.mark.parametrize("loss", ["huber", "cauchy"])
def test_block_model_gradient(loss):
    """The Gauss-Newton model's gradient g is the gradient of E^alpha(. | z) at z: central
    differences of the surrogate along random parameter directions of a block."""
    rng = np.random.default_rng(9)
    sc = _scene()
    prob, part, R, t, d, l = _problem(sc, 4, loss=loss, xi=1e-4)
    ci, li = prob.cam_idx, prob.lm_idx
    isin = B.intra(part, ci, li)
    mj = O.majorizer(prob.loss, prob.c, R[ci], t[ci], d[ci], l[li], prob.u)
    for alpha in (0, 3):
        H, g, cams, lms = B.block_model(prob, part, isin, mj, R, t, d, l, alpha)
        nc = cams.size
        assert np.all(np.linalg.eigvalsh(H.toarray()) > 0)   # the damped system is solvable
        for _ in range(3):
            v = rng.normal(size=g.size)
            h = 1e-6
            vals = []
            for sgn in (1.0, -1.0):
                th = sgn * h * v
                Rx, tx, dx, lx = R.copy(), t.copy(), d.copy(), l.copy()
                for k, i in enumerate(cams):
                    Rx[i] = R[i] @ O.so3_exp(th[9 * k:9 * k + 3][None])[0]
                    tx[i] = t[i] + th[9 * k + 3:9 * k + 6]
                    dx[i] = d[i] + th[9 * k + 6:9 * k + 9]
                for k, j in enumerate(lms):
                    lx[j] = l[j] + th[9 * nc + 3 * k:9 * nc + 3 * k + 3]
                vals.append(B.dE_blocks(prob, part, isin, mj, Rx, tx, dx, lx, R, t, d, l)[alpha])
            fd = (vals[0] - vals[1]) / (2 * h)
            assert g @ v == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(g).sum())


def test_lm_step_never_raises_a_block_surrogate():
    rng = np.random.default_rng(2)
    sc = _scene()
    prob, part, R, t, d, l = _problem(sc, 4)
    ci, li = prob.cam_idx, prob.lm_idx
    isin = B.intra(part, ci, li)
    Rz, tz, dz, lz = _perturb(rng, R, t, d, l, 1e-2)
    mj = O.majorizer(prob.loss, prob.c, Rz[ci], tz[ci], dz[ci], lz[li], prob.u)
    Rn, tn, dn, ln, taken = B.solve_blocks_lm(prob, part, isin, mj, Rz, tz, dz, lz)
    dE = B.dE_blocks(prob, part, isin, mj, Rn, tn, dn, ln, Rz, tz, dz, lz)
    assert np.all(dE <= 0.0) and taken == part.S and np.all(dE < 0.0)


@pytest.mark.parametrize("n_blocks,eta,restart", [(4, 0.5, "block"), (2, 1.0, "block"), (20, 0.5, "block"),
                                                   (4, 0.5, "global"), (20, 1.0, "global"), (4, 0.5, "reset")])
def test_algorithm1_invariants_with_blocks(n_blocks, eta, restart):
    """Lemma 1a-c, Eq. FakplFk1 and Eq. FklFk0 every iteration with multi-element blocks; with the
    global restart Lemma 1c holds for the sums over the blocks (the test of Algorithm 1 for the one
    block made of all), every block restarts together, and a restart fires within 15 iterations."""
    sc = _scene()
    kw = {"block": {}, "global": {"restart": "global"}, "reset": {"restart": "global", "momentum_reset": True}}[restart]
    prob, part, R, t, d, l = _problem(sc, n_blocks, eta=eta, xi=1e-8, **kw)
    st = B.init_state(prob, part, R, t, d, l)
    Fbar_global = O.objective(prob.loss, prob.c, R, t, d, l, prob.cam_idx, prob.lm_idx, prob.u)
    nrs = 0
    for k in range(15):
        prev = st
        st, info = B.step(prob, part, prev)
        F = info.F
        assert info.F_blk.sum() == pytest.approx(F, rel=1e-11)
        Fbar_global = (1 - eta) * Fbar_global + eta * F
        assert info.Fbar_blk.sum() == pytest.approx(Fbar_global, rel=1e-11)
        assert np.all(info.F_blk <= prev.E + 1e-12 * np.abs(prev.E))
        if restart == "block":
            assert np.all(st.E <= info.Fbar_blk + 1e-12 * np.abs(info.Fbar_blk))
        else:
            assert st.E.sum() <= info.Fbar_blk.sum() * (1 + 1e-12)
            assert info.restart.all() or not info.restart.any()
            if restart == "reset" and info.restart.any():
                assert st.s == 1.0
        Fn = O.objective(prob.loss, prob.c, st.R, st.t, st.d, st.l, prob.cam_idx, prob.lm_idx, prob.u)
        dx2 = O.cam_sqdist(st.R, st.t, st.d, prev.R, prev.t, prev.d).sum() + np.sum((st.l - prev.l) ** 2)
        assert Fn - Fbar_global <= -0.5 * prob.opts.xi * dx2 + 1e-12 * Fbar_global
        nrs += int(info.restart.sum())
        if k == 0:
            assert info.gamma == 0.0 and nrs == 0
    assert st.Fbar.sum() < 0.9 * O.objective(prob.loss, prob.c, R, t, d, l, prob.cam_idx, prob.lm_idx, prob.u)
    if restart != "block":
        assert nrs > 0


@pytest.mark.parametrize("n_blocks", [1, 4])
def test_duba_with_blocks_is_monotone(n_blocks):
    sc = _scene()
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px, accelerated=False)
    part = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, n_blocks)
    res = B.daba(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, part, opts, 12)
    assert np.all(np.diff(res.trace_px2) <= 1e-12 * res.trace_px2[:-1])
    assert res.trace_px2[-1] < res.trace_px2[0]


def test_noise_free_and_truth_with_blocks():
    from paper_2305_07026_b300 import scenes
    sc = scenes.circle_scene(n_lms=240, noise_free=True)
    part = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, 4)
    res = B.daba(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, part, O.Options(loss="trivial"), 40)
    assert res.trace_px2[-1] < 1e-3 * res.trace_px2[0]
    res = B.daba(sc.cams_gt, sc.lms_gt, sc.cam_idx, sc.lm_idx, sc.uv, part, O.Options(loss="huber"), 2)
    cams, lms = B.boundary_state(res)
    np.testing.assert_allclose(lms, sc.lms_gt, atol=1e-9)
    np.testing.assert_allclose(cams, sc.cams_gt, atol=1e-8)


def test_coarse_blocks_beat_singletons_per_iteration():
    """The paper notes that fewer, larger blocks give tighter surrogates (Sec. 7): after the
    same iterations the objective with 4 blocks is below the singleton partition's."""
    sc = _scene()
    opts = O.Options(loss=sc.loss, loss_scale_px=sc.loss_scale_px)
    part = B.camera_group_partition(sc.M, sc.cam_idx, sc.lm_idx, sc.N, 4)
    coarse = B.daba(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, part, opts, 10)
    single = O.daba(sc.cams, sc.lms, sc.cam_idx, sc.lm_idx, sc.uv, opts, 10)
    assert coarse.trace_px2[-1] < single.trace_px2[-1]


def test_block_decrease_restricted_to_the_block():
    """The LM acceptance test's per-block decrease (dE_block: the block's own cameras, landmarks
    and pairs) equals that block's entry of the decrease of every block at once."""
    rng = np.random.default_rng(5)
    sc = _scene()
    prob, part, R, t, d, l = _problem(sc, 4)
    ci, li = prob.cam_idx, prob.lm_idx
    isin = B.intra(part, ci, li)
    Rz, tz, dz, lz = _perturb(rng, R, t, d, l, 1e-2)
    mj = O.majorizer(prob.loss, prob.c, Rz[ci], tz[ci], dz[ci], lz[li], prob.u)
    all_blocks = B.dE_blocks(prob, part, isin, mj, R, t, d, l, Rz, tz, dz, lz)
    for alpha in range(part.S):
        one = B.dE_block(prob, part, isin, mj, R, t, d, l, Rz, tz, dz, lz, alpha)
        assert one == pytest.approx(all_blocks[alpha], rel=1e-13, abs=1e-16)
