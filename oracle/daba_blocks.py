"""FP64 oracle of Algorithm 1 (arXiv 2305.07026) with coarse blocks: test infrastructure only.

Only tests/ and bench.py's CPU legs import this module; the library never does.

A partition assigns every camera and every landmark to one of S blocks (the paper's devices,
Sec. 4). Reprojection pairs whose camera and landmark share a block form E' and keep their exact
F_ij in that block's surrogate; the other pairs (E'') are split by the majorizer of
Proposition 1 into P_ij (the camera's block) and Q_ij (the landmark's block), Eq. Ealpha:

    E^alpha(x^alpha | z) = xi/2 |x^alpha - z^alpha|^2 + sum_{E' in alpha} F_ij
                           + sum_{E'', i in alpha} P_ij(c_i | z) + sum_{E'', j in alpha} Q_ij(l_j | z).

Restart metrics per block (Eqs. DEalpha, Fainit, Fak, lFak, Eak): the surrogate gap of Eq. DEalpha
runs over the pairs of E'' that touch the block, each block taking half of it.

Subproblem solver (the paper reports one successful inner Levenberg-Marquardt step per
subproblem, Sec. 7.1, without its details; this is the reading): parameters per camera
theta_c = (phi, tau, delta) with R = R_z Exp(phi), t = t_z + tau, d = d_z + delta, per landmark
epsilon with l = l_z + epsilon. The Gauss-Newton model at theta = 0 is built from residuals:
  * an intra pair: sqrt(w) R e with w = rho'(|e|^2) at z (the reweighted Gauss-Newton model of
    F_ij = rho(|e|^2)/2, whose gradient w J^T R e is exact at z); R e = (I - q q^T/|q|^2) R p,
    q = l - t, so |R e| = |e| (Eq. error);
  * an inter pair's P_ij: sqrt(2 w_z) (R p(d) + lambda_z t - g_z) (Eq. P);
  * an inter pair's Q_ij: sqrt(2 w_z) (lambda_z l - g_z) (Eq. Q);
  * the proximal term: xi/2 |R_z Exp(phi) - R_z|^2 to second order is xi |phi|^2, so the model
    Hessian takes 2 xi on phi and xi on tau, delta, epsilon.
The step solves (H + mu diag H) theta = -g over all parameters of the block (mu = 1e-3, raised
tenfold up to 8 times); it is taken if E^alpha decreases, else the block stays at its start. The
decrease is evaluated term by term (residual differences for P and Q), so that no O(F) values
cancel. Start point and proximal centre are the conditioning iterate (x_bar^k for the accelerated
update, x^k for the MM update).

Global restart (Options.restart = "global"): one restart test on the sums over all blocks, every
block taking the MM update when it fires; with Options.momentum_reset the Nesterov scalar restarts
too (s <- 1), as in the singleton oracle.

Parity unpinned: the paper's own LM details (damping, parameterisation) are not given.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import daba_oracle as O

LM_MU0 = O.LM_MU0
LM_TRIES = O.LM_TRIES


@dataclasses.dataclass
class Partition:
    cam_block: np.ndarray   # (M,) block of every camera, 0 .. S-1
    lm_block: np.ndarray    # (N,) block of every landmark
    S: int


def make_partition(cam_block, lm_block) -> Partition:
    cb = np.asarray(cam_block, dtype=np.int64)
    lb = np.asarray(lm_block, dtype=np.int64)
    return Partition(cam_block=cb, lm_block=lb, S=int(max(cb.max(initial=-1), lb.max(initial=-1)) + 1))


def camera_group_partition(M, cam_idx, lm_idx, N, n_blocks):
    """Contiguous groups of cameras; every landmark joins the block of its lowest-index observing
    camera (a landmark seen by no camera joins block 0)."""
    cam_block = (np.arange(M) * n_blocks) // M
    first_cam = np.full(N, M, dtype=np.int64)
    np.minimum.at(first_cam, lm_idx, cam_idx)
    lm_block = np.where(first_cam < M, cam_block[np.minimum(first_cam, M - 1)], 0)
    return make_partition(cam_block, lm_block)


def intra(part: Partition, cam_idx, lm_idx):
    """Mask of the pairs in E' (camera and landmark in the same block)."""
    return part.cam_block[cam_idx] == part.lm_block[lm_idx]


# ----------------------------------------------------------------------------
# per-observation Jacobian of R e for the intra pairs
# ----------------------------------------------------------------------------

def intra_residual_jacobian(R, t, d, l, u):
    """R e (n, 3) and its Jacobian (n, 3, 12) w.r.t. (phi, tau, delta, epsilon) at theta = 0.

    With v = R p(d) and q = l - t, R e = v - lambda q = (I - q q^T/|q|^2) v (Eqs. lambdaij, error).
    d(R e)/dv = I - q q^T/|q|^2; d(R e)/dq = -lambda I - q (v - 2 lambda q)^T / |q|^2;
    dv/dphi = -R [p]x (R Exp(phi) p); dv/ddelta = (R e3) (1, s, s^2); dq/dtau = -I; dq/depsilon = I."""
    p = O.ray(u, d)
    v = np.einsum("nab,nb->na", R, p)
    q = l - t
    qq = np.einsum("na,na->n", q, q)
    lm = np.einsum("na,na->n", q, v) / qq
    f = v - lm[:, None] * q
    Pi = np.eye(3)[None] - q[:, :, None] * q[:, None, :] / qq[:, None, None]
    Dq = -lm[:, None, None] * np.eye(3)[None] - q[:, :, None] * (v - 2.0 * lm[:, None] * q)[:, None, :] / qq[:, None, None]
    s = u[:, 0] ** 2 + u[:, 1] ** 2
    phi_u = np.stack([np.ones_like(s), s, s * s], 1)
    J = np.zeros((u.shape[0], 3, 12))
    J[:, :, 0:3] = np.einsum("nab,nbc->nac", Pi, -np.einsum("nab,nbc->nac", R, O.skew(p)))
    J[:, :, 3:6] = -Dq
    J[:, :, 6:9] = np.einsum("nab,nb->na", Pi, R[:, :, 2])[:, :, None] * phi_u[:, None, :]
    J[:, :, 9:12] = Dq
    return f, J


# ----------------------------------------------------------------------------
# block surrogate differences
# ----------------------------------------------------------------------------

def dE_blocks(prob, part, isin, mj, Rx, tx, dx, lx, Rz, tz, dz, lz):
    """E^alpha(x | z) - E^alpha(z | z) of every block (S,), term by term: the proximal term, the
    exact F_ij of the intra pairs, and P_ij, Q_ij of the inter pairs from residual differences."""
    ci, li, u, M, N = prob.cam_idx, prob.lm_idx, prob.u, prob.M, prob.N
    xi = prob.opts.xi
    out = 0.5 * xi * (O.segsum(part.cam_block, O.cam_sqdist(Rx, tx, dx, Rz, tz, dz), part.S)
                      + O.segsum(part.lm_block, np.sum((lx - lz) ** 2, axis=1), part.S))
    ii = np.flatnonzero(isin)
    if ii.size:
        Fx = O.F_obs(prob.loss, prob.c, Rx[ci[ii]], tx[ci[ii]], dx[ci[ii]], lx[li[ii]], u[ii])
        Fz = O.F_obs(prob.loss, prob.c, Rz[ci[ii]], tz[ci[ii]], dz[ci[ii]], lz[li[ii]], u[ii])
        out += O.segsum(part.cam_block[ci[ii]], Fx - Fz, part.S)
    oo = np.flatnonzero(~isin)
    if oo.size:
        c, lj = ci[oo], li[oo]
        w, lam, g = mj.w[oo], mj.lam[oo], mj.g[oo]
        rP0 = np.einsum("nab,nb->na", Rz[c], O.ray(u[oo], dz[c])) + lam[:, None] * tz[c] - g
        drP = np.einsum("nab,nb->na", Rx[c], O.ray(u[oo], dx[c])) + lam[:, None] * tx[c] - g - rP0
        out += O.segsum(part.cam_block[c], w * np.einsum("na,na->n", drP, drP + 2.0 * rP0), part.S)
        rQ0 = lam[:, None] * lz[lj] - g
        drQ = lam[:, None] * (lx[lj] - lz[lj])
        out += O.segsum(part.lm_block[lj], w * np.einsum("na,na->n", drQ, drQ + 2.0 * rQ0), part.S)
    return out


def E_blocks_at(prob, part, isin, R, t, d, l):
    """E^alpha(x | x) of every block: sum of F_ij over its intra pairs plus half of F_ij over the
    inter pairs that touch it (P_ij = Q_ij = F_ij / 2 at the conditioning iterate, Eq. approx0)."""
    ci, li = prob.cam_idx, prob.lm_idx
    F = O.F_obs(prob.loss, prob.c, R[ci], t[ci], d[ci], l[li], prob.u)
    return (O.segsum(part.cam_block[ci], np.where(isin, F, 0.5 * F), part.S)
            + O.segsum(part.lm_block[li], np.where(isin, 0.0, 0.5 * F), part.S))


# ----------------------------------------------------------------------------
# one successful LM step per block
# ----------------------------------------------------------------------------

def block_params(part, alpha):
    cams = np.flatnonzero(part.cam_block == alpha)
    lms = np.flatnonzero(part.lm_block == alpha)
    return cams, lms


def block_model(prob, part, isin, mj, Rz, tz, dz, lz, alpha):
    """Gauss-Newton model (H, g) of E^alpha(. | z) at z over the block's parameters, ordered
    [9 per camera (ascending index) | 3 per landmark (ascending index)]; H is a sparse matrix
    (scipy CSC) whose entries are the sums of the per-term blocks below."""
    ci, li, u = prob.cam_idx, prob.lm_idx, prob.u
    xi = prob.opts.xi
    cams, lms = block_params(part, alpha)
    nc, nl = cams.size, lms.size
    n = 9 * nc + 3 * nl
    cpos = np.full(part.cam_block.size, -1)
    cpos[cams] = np.arange(nc)
    lpos = np.full(part.lm_block.size, -1)
    lpos[lms] = np.arange(nl)
    rows, cols, vals = [], [], []
    g = np.zeros(n)

    def add(idx, blocks):   # idx (m, k) parameter indices, blocks (m, k, k) Hessian terms
        rows.append(np.broadcast_to(idx[:, :, None], blocks.shape).ravel())
        cols.append(np.broadcast_to(idx[:, None, :], blocks.shape).ravel())
        vals.append(blocks.ravel())

    # proximal term: 2 xi on phi, xi on tau, delta and epsilon
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(np.concatenate([np.tile(np.r_[np.full(3, 2.0 * xi), np.full(6, xi)], nc), np.full(3 * nl, xi)]))
    r9, r3 = np.arange(9), np.arange(3)
    # intra pairs: reweighted Gauss-Newton on R e
    ii = np.flatnonzero(isin & (part.cam_block[ci] == alpha))
    if ii.size:
        f, J = intra_residual_jacobian(Rz[ci[ii]], tz[ci[ii]], dz[ci[ii]], lz[li[ii]], u[ii])
        r = np.einsum("na,na->n", f, f)
        _, w = O.rho(prob.loss, prob.c, r)
        idx = np.concatenate([9 * cpos[ci[ii]][:, None] + r9, 9 * nc + 3 * lpos[li[ii]][:, None] + r3], 1)
        add(idx, w[:, None, None] * np.einsum("nai,naj->nij", J, J))
        np.add.at(g, idx, w[:, None] * np.einsum("nai,na->ni", J, f))
    # inter pairs, camera side: P_ij residual R p(d) + lambda t - g (as in the camera LM model)
    oc = np.flatnonzero(~isin & (part.cam_block[ci] == alpha))
    if oc.size:
        c = ci[oc]
        s = u[oc, 0] ** 2 + u[oc, 1] ** 2
        phi_u = np.stack([np.ones_like(s), s, s * s], 1)
        p0 = O.ray(u[oc], dz[c])
        r0 = np.einsum("nab,nb->na", Rz[c], p0) + mj.lam[oc, None] * tz[c] - mj.g[oc]
        JP = np.zeros((oc.size, 3, 9))
        JP[:, :, 0:3] = -np.einsum("nab,nbc->nac", Rz[c], O.skew(p0))
        JP[:, 0, 3] = JP[:, 1, 4] = JP[:, 2, 5] = mj.lam[oc]
        JP[:, :, 6:9] = Rz[c][:, :, 2][:, :, None] * phi_u[:, None, :]
        idx = 9 * cpos[c][:, None] + r9
        w2 = 2.0 * mj.w[oc]
        add(idx, w2[:, None, None] * np.einsum("nai,naj->nij", JP, JP))
        np.add.at(g, idx, w2[:, None] * np.einsum("nai,na->ni", JP, r0))
    # inter pairs, landmark side: Q_ij residual lambda l - g
    ol = np.flatnonzero(~isin & (part.lm_block[li] == alpha))
    if ol.size:
        w, lam = mj.w[ol], mj.lam[ol]
        idx = 9 * nc + 3 * lpos[li[ol]][:, None] + r3
        rows.append(idx.ravel())
        cols.append(idx.ravel())
        vals.append(np.repeat(2.0 * w * lam * lam, 3))
        np.add.at(g, idx, (2.0 * w * lam)[:, None] * (lam[:, None] * lz[li[ol]] - mj.g[ol]))
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsc()
    return H, g, cams, lms


def dE_block(prob, part, isin, mj, Rx, tx, dx, lx, Rz, tz, dz, lz, alpha):
    """E^alpha(x | z) - E^alpha(z | z) of block alpha alone: dE_blocks restricted to the terms of
    the block (the same sums, over the block's own cameras, landmarks and pairs, in order)."""
    ci, li = prob.cam_idx, prob.lm_idx
    cm, lm = part.cam_block == alpha, part.lm_block == alpha
    ob = np.flatnonzero(cm[ci] | lm[li])
    sub = O.Problem(**{**prob.__dict__, "cam_idx": ci[ob], "lm_idx": li[ob], "u": prob.u[ob]})
    one = Partition(cam_block=np.where(cm, 0, 1), lm_block=np.where(lm, 0, 1), S=2)
    mjo = O.Majorizer(**{k: v[ob] for k, v in mj.__dict__.items()})
    return dE_blocks(sub, one, isin[ob], mjo, Rx, tx, dx, lx, Rz, tz, dz, lz)[0]


def solve_blocks_lm(prob, part, isin, mj, Rz, tz, dz, lz):
    """One successful LM step per block on E^alpha(. | z) from z (module docstring); returns the
    new (R, t, d, l) of every camera and landmark and the accepted step count."""
    R, t, d, l = Rz.copy(), tz.copy(), dz.copy(), lz.copy()
    taken = 0
    for alpha in range(part.S):
        H, g, cams, lms = block_model(prob, part, isin, mj, Rz, tz, dz, lz, alpha)
        if g.size == 0:
            continue
        nc = cams.size
        D = sp.diags(H.diagonal())
        mu = LM_MU0
        for _ in range(LM_TRIES):
            th = spla.spsolve((H + mu * D).tocsc(), -g)
            Rc, tc, dc, lc = R.copy(), t.copy(), d.copy(), l.copy()
            for k, i in enumerate(cams):
                Rc[i] = Rz[i] @ O.so3_exp(th[9 * k:9 * k + 3][None])[0]
                tc[i] = tz[i] + th[9 * k + 3:9 * k + 6]
                dc[i] = dz[i] + th[9 * k + 6:9 * k + 9]
            for k, j in enumerate(lms):
                lc[j] = lz[j] + th[9 * nc + 3 * k:9 * nc + 3 * k + 3]
            dE = dE_block(prob, part, isin, mj, Rc, tc, dc, lc, Rz, tz, dz, lz, alpha)
            if dE < 0.0:
                R[cams], t[cams], d[cams], l[lms] = Rc[cams], tc[cams], dc[cams], lc[lms]
                taken += 1
                break
            mu *= 10.0
    return R, t, d, l, taken


# ----------------------------------------------------------------------------
# Algorithm 1 with blocks
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class BlockState:
    R: np.ndarray
    t: np.ndarray
    d: np.ndarray
    l: np.ndarray
    Rp: np.ndarray
    tp: np.ndarray
    dp: np.ndarray
    lp: np.ndarray
    s: float
    k: int
    E: np.ndarray      # E^alpha(k) per block
    Fbar: np.ndarray   # Fbar^alpha(k-1)


@dataclasses.dataclass
class BlockStepInfo:
    F: float
    F_blk: np.ndarray
    Fbar_blk: np.ndarray
    Etest: np.ndarray
    restart: np.ndarray
    gamma: float


def init_state(prob, part, R, t, d, l) -> BlockState:
    """x^(-1) = x^(0), s^(0) = 1, F^alpha(-1) = Fbar^alpha(-1) = E^alpha(0) = E^alpha(x^0 | x^0)
    (Eq. Fainit)."""
    isin = intra(part, prob.cam_idx, prob.lm_idx)
    E0 = E_blocks_at(prob, part, isin, R, t, d, l)
    return BlockState(R=R.copy(), t=t.copy(), d=d.copy(), l=l.copy(), Rp=R.copy(), tp=t.copy(), dp=d.copy(),
                      lp=l.copy(), s=1.0, k=0, E=E0.copy(), Fbar=E0.copy())


def step(prob, part, st: BlockState):
    """One iteration k of Algorithm 1 with the blocks of `part`."""
    o = prob.opts
    xi, eta = o.xi, o.eta
    ci, li, u = prob.cam_idx, prob.lm_idx, prob.u
    isin = intra(part, ci, li)
    s_next, gamma = O.nesterov(st.s)
    Rb, tb, db, lb = O.extrapolate(st.R, st.t, st.d, st.l, st.Rp, st.tp, st.dp, st.lp, gamma)
    mj_k = O.majorizer(prob.loss, prob.c, st.R[ci], st.t[ci], st.d[ci], st.l[li], u)
    mj_b = O.majorizer(prob.loss, prob.c, Rb[ci], tb[ci], db[ci], lb[li], u)
    mj_p = O.majorizer(prob.loss, prob.c, st.Rp[ci], st.tp[ci], st.dp[ci], st.lp[li], u)
    Fij = O.F_obs(prob.loss, prob.c, st.R[ci], st.t[ci], st.d[ci], st.l[li], u)
    # Eq. DEalpha: the proximal displacement and half the surrogate gap of every inter pair that
    # touches the block
    gap = np.where(isin, 0.0, Fij - O.P_obs(mj_p, st.R[ci], st.t[ci], st.d[ci], u) - O.Q_obs(mj_p, st.l[li]))
    disp = (O.segsum(part.cam_block, O.cam_sqdist(st.R, st.t, st.d, st.Rp, st.tp, st.dp), part.S)
            + O.segsum(part.lm_block, np.sum((st.l - st.lp) ** 2, axis=1), part.S))
    dE = -0.5 * xi * disp + 0.5 * (O.segsum(part.cam_block[ci], gap, part.S) + O.segsum(part.lm_block[li], gap, part.S))
    F_blk = st.E + dE                                   # Eq. Fak
    Fbar = (1.0 - eta) * st.Fbar + eta * F_blk          # Eq. lFak
    Rm, tm, dm, lm_, _ = solve_blocks_lm(prob, part, isin, mj_k, st.R, st.t, st.d, st.l)
    Emm = F_blk + dE_blocks(prob, part, isin, mj_k, Rm, tm, dm, lm_, st.R, st.t, st.d, st.l)   # Eq. Eak
    if o.accelerated:
        Ra, ta, da, la, _ = solve_blocks_lm(prob, part, isin, mj_b, Rb, tb, db, lb)
        Ea = F_blk + dE_blocks(prob, part, isin, mj_k, Ra, ta, da, la, st.R, st.t, st.d, st.l)
        if o.restart == "global":
            # the test of Algorithm 1 for the one block made of all blocks; with the momentum
            # reset the Nesterov scalar restarts with it
            fire = bool(np.sum(Ea) > np.sum(Fbar))
            rs = np.full(part.S, fire)
            if fire and o.momentum_reset:
                s_next = 1.0
        else:
            rs = Ea > Fbar
    else:
        Ra, ta, da, la, Ea = Rm, tm, dm, lm_, Emm
        rs = np.ones(part.S, dtype=bool)
    rc, rl = rs[part.cam_block], rs[part.lm_block]
    new = BlockState(R=np.where(rc[:, None, None], Rm, Ra), t=np.where(rc[:, None], tm, ta),
                     d=np.where(rc[:, None], dm, da), l=np.where(rl[:, None], lm_, la), Rp=st.R, tp=st.t, dp=st.d,
                     lp=st.l, s=s_next, k=st.k + 1, E=np.where(rs, Emm, Ea), Fbar=Fbar)
    info = BlockStepInfo(F=float(np.sum(Fij)), F_blk=F_blk, Fbar_blk=Fbar, Etest=Ea,
                         restart=rs if o.accelerated else np.zeros(part.S, dtype=bool), gamma=gamma)
    return new, info


@dataclasses.dataclass
class BlockRunResult:
    trace_px2: np.ndarray
    restarts: np.ndarray
    state: BlockState
    infos: list
    prob: O.Problem


def daba(cams, lms, cam_idx, lm_idx, uv, part: Partition, opts: O.Options, iters: int, keep_infos: int = 0):
    """Algorithm 1 with the blocks of `part` for `iters` iterations (DUBA with opts.accelerated=False)."""
    prob, R, t, d, l = O.make_problem(cams, lms, cam_idx, lm_idx, uv, opts)
    st = init_state(prob, part, R, t, d, l)
    trace, restarts, infos = [], [], []
    for _ in range(iters):
        st, info = step(prob, part, st)
        trace.append(info.F)
        restarts.append(int(info.restart.sum()))
        if len(infos) < keep_infos:
            infos.append(info)
    trace.append(O.objective(prob.loss, prob.c, st.R, st.t, st.d, st.l, prob.cam_idx, prob.lm_idx, prob.u))
    return BlockRunResult(trace_px2=np.asarray(trace) * prob.s_norm ** 2, restarts=np.asarray(restarts), state=st,
                          infos=infos, prob=prob)


def boundary_state(res: BlockRunResult):
    st = res.state
    return O.to_boundary(st.R, st.t, st.d, st.l, res.prob.s_norm)
