// daba_blocks.cuh -- Algorithm 1 with coarse blocks (Eq. Ealpha with E' not empty), FP64.
//
// A block holds at most one camera and any set of landmarks. Pairs whose camera and landmark
// share a block (E') keep their exact F_ij in the block surrogate; the others are split by the
// majorizer of Proposition 1. Per iteration:
//   1. the camera pass in block mode (k_cpass_blk): as k_cpass, but an intra pair adds to no
//      statistics, gap or landmark record; it adds F_ij to the camera's F sums;
//   2. the landmark pass in sum mode: every landmark's sums of its inter records (a, b at x̄^k
//      and at x^k, F_ij and the surrogate gap);
//   3. k_blk_solve, one warp per block: the restart metrics (Eqs. DEalpha, Fak, lFak), one
//      successful Levenberg-Marquardt step on E^alpha(. | x̄^k) from x̄^k, the restart test
//      (Eq. Eak) and, where it fires, the LM step on E^alpha(. | x^k) from x^k.
// LM step: parameters (phi, tau, delta) of the camera (R = R_z Exp(phi), t = t_z + tau,
// d = d_z + delta) and epsilon of each landmark (l = l_z + epsilon). Gauss-Newton model: the
// camera's inter pairs and proximal term from its statistics (cam_lm_model); each landmark's
// inter pairs 2 a I and 2 b, proximal xi I; each intra pair the reweighted Gauss-Newton terms of
// R e = (I - q q^T/|q|^2) R p with w = rho'(|e|^2) at z. The damped system (H + mu diag H) is
// solved through the 9 x 9 Schur complement of the camera (each landmark's 3 x 3 block
// eliminated); the step is taken if E^alpha decreases (surrogate differences term by term),
// otherwise mu grows tenfold, at most LM_TRIES times.
#pragma once

#include "daba_kernels.cuh"

namespace daba {

// landmark sums written by the landmark pass in sum mode (per internal landmark)
enum { LS_AB = 0, LS_BB = 1, LS_AK = 4, LS_BK = 5, LS_F = 8, LS_G = 9, LS_N = 10 };
// per owned landmark scratch of the block solve
enum { BS_C = 0, BS_G = 6, BS_B = 9, BS_FZ = 36, BS_L = 37, BS_N = 40 };

struct BlkArgs {
  int S;
  const int *blk_cam, *blk_lm_ptr, *blk_lms, *blk_obs;   // block camera (-1: none); owned landmarks; their intra pair (-1: none)
  const int* c_lm;
  const double2* c_u;
  const int* cam_chunk_ptr;
  const double* part;
  const double* lm_sums;   // LS_N per internal landmark
  double *cam_x, *cam_dx, *cam_Rbar, *cam_Fsum;
  uint8_t* cam_rs;
  const V4<double>* lmrec;   // landmark state of iteration k
  V4<double>* lmrec_out;     // of iteration k + 1
  double *blk_E, *blk_Fbar, *blk_F;
  uint8_t* blk_rs;
  double* scr;     // BS_N per internal landmark
  V4<double>* pack_next;
  LossC<double> L;
};

// R e = (I - q q^T/|q|^2) R p and its Jacobian: Jc (3 x 9: phi, tau, delta) and Jl (3 x 3)
__device__ inline void blk_intra_jac(const CamT<double>& c, const double* l, double u0, double u1, double* f,
                                     double Jc[3][9], double Jl[3][3]) {
  const double s = u0 * u0 + u1 * u1;
  const double p[3] = {u0, u1, c.d[0] + c.d[1] * s + c.d[2] * s * s};
  double v[3], q[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    v[r] = c.R[3 * r] * p[0] + c.R[3 * r + 1] * p[1] + c.R[3 * r + 2] * p[2];
    q[r] = l[r] - c.t[r];
  }
  const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
  const double lam = (q[0] * v[0] + q[1] * v[1] + q[2] * v[2]) / qq;
#pragma unroll
  for (int r = 0; r < 3; ++r) f[r] = v[r] - lam * q[r];
  double Pi[3][3], Dq[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Pi[r][k] = (r == k ? 1.0 : 0.0) - q[r] * q[k] / qq;
      Dq[r][k] = (r == k ? -lam : 0.0) - q[r] * (v[k] - 2.0 * lam * q[k]) / qq;
    }
  // -R [p]x, column k: -R (e_k x p)... [p]x = [[0,-p2,p1],[p2,0,-p0],[-p1,p0,0]]
  const double px[3][3] = {{0.0, -p[2], p[1]}, {p[2], 0.0, -p[0]}, {-p[1], p[0], 0.0}};
  double Mr[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      Mr[r][k] = -(c.R[3 * r] * px[0][k] + c.R[3 * r + 1] * px[1][k] + c.R[3 * r + 2] * px[2][k]);
  double pe[3];   // Pi R e3
#pragma unroll
  for (int r = 0; r < 3; ++r) pe[r] = Pi[r][0] * c.R[2] + Pi[r][1] * c.R[5] + Pi[r][2] * c.R[8];
  const double ph[3] = {1.0, s, s * s};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Jc[r][k] = Pi[r][0] * Mr[0][k] + Pi[r][1] * Mr[1][k] + Pi[r][2] * Mr[2][k];
      Jc[r][3 + k] = -Dq[r][k];
      Jc[r][6 + k] = pe[r] * ph[k];
      Jl[r][k] = Dq[r][k];
    }
  }
}

// F_ij = rho(|e|^2) / 2 at (camera, landmark)
__device__ inline double blk_F(const CamT<double>& c, const double* l, double u0, double u1, const LossC<double>& L,
                               int loss) {
  const double s = u0 * u0 + u1 * u1;
  const double p[3] = {u0, u1, c.d[0] + c.d[1] * s + c.d[2] * s * s};
  double v[3], q[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    v[r] = c.R[3 * r] * p[0] + c.R[3 * r + 1] * p[1] + c.R[3 * r + 2] * p[2];
    q[r] = l[r] - c.t[r];
  }
  const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
  const double lam = (q[0] * v[0] + q[1] * v[1] + q[2] * v[2]) / qq;
  double r2 = 0.0;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double e = v[r] - lam * q[r];
    r2 += e * e;
  }
  double rho, w;
  switch (loss) {
    case LOSS_TRIVIAL: rho_w<LOSS_TRIVIAL, double>(L, r2, rho, w); break;
    case LOSS_HUBER: rho_w<LOSS_HUBER, double>(L, r2, rho, w); break;
    case LOSS_CAUCHY: rho_w<LOSS_CAUCHY, double>(L, r2, rho, w); break;
    default: rho_w<LOSS_WELSCH, double>(L, r2, rho, w); break;
  }
  return 0.5 * rho;
}

// sum over the warp, lane 0's result on every lane (the butterfly's lanes associate the sums in
// different orders; the block's decisions must be the same on every lane)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return __shfl_sync(0xffffffffu, v, 0);
}

// 3 x 3 symmetric (packed xx, yx, yy, zx, zy, zz) inverse
__device__ __forceinline__ void sym3_inv(const double* C, double* I) {
  const double a = C[0], b = C[1], c = C[2], d = C[3], e = C[4], f = C[5];
  const double A0 = c * f - e * e, A1 = -(b * f - e * d), A3 = b * e - c * d;
  const double det = a * A0 + b * A1 + d * A3;
  const double id = 1.0 / det;
  I[0] = A0 * id;
  I[1] = A1 * id;
  I[2] = (a * f - d * d) * id;
  I[3] = A3 * id;
  I[4] = -(a * e - b * d) * id;
  I[5] = (a * c - b * b) * id;
}
__device__ __forceinline__ void sym3_mul(const double* S, const double* x, double* y) {
  y[0] = S[0] * x[0] + S[1] * x[1] + S[3] * x[2];
  y[1] = S[1] * x[0] + S[2] * x[1] + S[4] * x[2];
  y[2] = S[3] * x[0] + S[4] * x[1] + S[5] * x[2];
}

// Landmark position of the conditioning iterate: x^k or x̄^k = l + gamma (l - l^(k-1))
__device__ __forceinline__ void blk_lpos(const V4<double>* lmrec, int j, double gamma, bool bar, double* l) {
  const V4<double> A = lmrec[2 * (size_t)j], B = lmrec[2 * (size_t)j + 1];
  l[0] = A.x + (bar ? gamma * A.w : 0.0);
  l[1] = A.y + (bar ? gamma * B.x : 0.0);
  l[2] = A.z + (bar ? gamma * B.y : 0.0);
}

// One LM step of block b (its warp) on E^alpha(. | z), z = x̄^k (bar) or x^k, from z. The
// solution's landmarks go to scratch scr + BS_L, the camera to *cs. Returns nothing; a block whose
// step is never taken stays at z.
__device__ inline void blk_lm(const BlkArgs& A, int b, int lane, bool bar, double gamma, int cam, const double* stz,
                              const CamT<double>& cz, double xi, double* scr, CamT<double>& cs, int loss) {
  const int l0 = A.blk_lm_ptr[b], l1 = A.blk_lm_ptr[b + 1];
  const int ao = bar ? LS_AB : LS_AK, bo = bar ? LS_BB : LS_BK;
  double Am[45], g[9];
  if (cam >= 0) cam_lm_model(stz, cz, xi, Am, g);
  double Ai[45], gi[9];
#pragma unroll
  for (int k = 0; k < 45; ++k) Ai[k] = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) gi[k] = 0.0;
  // ---- per landmark: its 3 x 3 block, gradient, coupling to the camera, F at z of its intra pair
  for (int e = l0 + lane; e < l1; e += 32) {
    const int j = A.blk_lms[e];
    double* s = scr + (size_t)j * BS_N;
    double lz[3];
    blk_lpos(A.lmrec, j, gamma, bar, lz);
    const double* sm = A.lm_sums + (size_t)j * LS_N;
    const double a2 = 2.0 * sm[ao];
    double C[6] = {a2 + xi, 0.0, a2 + xi, 0.0, 0.0, a2 + xi};
    double gl[3] = {2.0 * sm[bo], 2.0 * sm[bo + 1], 2.0 * sm[bo + 2]};
    double Bm[27];
#pragma unroll
    for (int k = 0; k < 27; ++k) Bm[k] = 0.0;
    double Fz = 0.0;
    const int o = A.blk_obs[e];
    if (o >= 0 && cam >= 0) {
      const double2 u = A.c_u[o];
      double f[3], Jc[3][9], Jl[3][3];
      blk_intra_jac(cz, lz, u.x, u.y, f, Jc, Jl);
      const double r = f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
      double rho, w;
      switch (loss) {
        case LOSS_TRIVIAL: rho_w<LOSS_TRIVIAL, double>(A.L, r, rho, w); break;
        case LOSS_HUBER: rho_w<LOSS_HUBER, double>(A.L, r, rho, w); break;
        case LOSS_CAUCHY: rho_w<LOSS_CAUCHY, double>(A.L, r, rho, w); break;
        default: rho_w<LOSS_WELSCH, double>(A.L, r, rho, w); break;
      }
      Fz = 0.5 * rho;
      int q = 0;
#pragma unroll
      for (int r1 = 0; r1 < 3; ++r1)
#pragma unroll
        for (int c1 = 0; c1 <= r1; ++c1, ++q) {
          double v = 0.0;
#pragma unroll
          for (int k = 0; k < 3; ++k) v += Jl[k][r1] * Jl[k][c1];
          C[q] += w * v;
        }
#pragma unroll
      for (int r1 = 0; r1 < 3; ++r1) gl[r1] += w * (Jl[0][r1] * f[0] + Jl[1][r1] * f[1] + Jl[2][r1] * f[2]);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
#pragma unroll
        for (int k = 0; k < 3; ++k) Bm[i * 3 + k] = w * (Jc[0][i] * Jl[0][k] + Jc[1][i] * Jl[1][k] + Jc[2][i] * Jl[2][k]);
        gi[i] += w * (Jc[0][i] * f[0] + Jc[1][i] * f[1] + Jc[2][i] * f[2]);
#pragma unroll
        for (int k = 0; k <= i; ++k) Ai[lt9(i, k)] += w * (Jc[0][i] * Jc[0][k] + Jc[1][i] * Jc[1][k] + Jc[2][i] * Jc[2][k]);
      }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) s[BS_C + k] = C[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) s[BS_G + k] = gl[k];
#pragma unroll
    for (int k = 0; k < 27; ++k) s[BS_B + k] = Bm[k];
    s[BS_FZ] = Fz;
#pragma unroll
    for (int k = 0; k < 3; ++k) s[BS_L + k] = lz[k];   // the landmark stays at z unless a step is taken
  }
  if (cam >= 0) {
#pragma unroll
    for (int k = 0; k < 45; ++k) Am[k] += warp_sum(Ai[k]);
#pragma unroll
    for (int k = 0; k < 9; ++k) g[k] += warp_sum(gi[k]);
  }
  cs = cz;
  double mu = LM_MU0;
  for (int tr = 0; tr < LM_TRIES; ++tr, mu *= 10.0) {
    // ---- Schur complement of the damped system onto the camera
    double Sacc[45], racc[9];
#pragma unroll
    for (int k = 0; k < 45; ++k) Sacc[k] = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) racc[k] = 0.0;
    for (int e = l0 + lane; e < l1; e += 32) {
      if (cam < 0 || A.blk_obs[e] < 0) continue;
      const double* s = scr + (size_t)A.blk_lms[e] * BS_N;
      double Cm[6], Ci[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) Cm[k] = s[BS_C + k];
      Cm[0] *= 1.0 + mu;
      Cm[2] *= 1.0 + mu;
      Cm[5] *= 1.0 + mu;
      sym3_inv(Cm, Ci);
      double BC[9][3];   // B C^-1
#pragma unroll
      for (int i = 0; i < 9; ++i) sym3_mul(Ci, s + BS_B + 3 * i, BC[i]);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
#pragma unroll
        for (int k = 0; k <= i; ++k)
          Sacc[lt9(i, k)] -= BC[i][0] * s[BS_B + 3 * k] + BC[i][1] * s[BS_B + 3 * k + 1] + BC[i][2] * s[BS_B + 3 * k + 2];
        racc[i] += BC[i][0] * s[BS_G] + BC[i][1] * s[BS_G + 1] + BC[i][2] * s[BS_G + 2];
      }
    }
    double dc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool ok = true;
    if (cam >= 0) {
      double L9[45];
#pragma unroll
      for (int k = 0; k < 45; ++k) L9[k] = warp_sum(Sacc[k]);
      double rhs[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) rhs[k] = -g[k] + warp_sum(racc[k]);
      // Cholesky of (A + mu diag A) - sum B C^-1 B^T, every lane the same
      for (int i = 0; i < 9; ++i) {
        for (int j = 0; j <= i; ++j) {
          double v = Am[lt9(i, j)] * (i == j ? 1.0 + mu : 1.0) + L9[lt9(i, j)];
          for (int k = 0; k < j; ++k) v -= L9[lt9(i, k)] * L9[lt9(j, k)];
          if (i == j) {
            if (!(v > 0.0)) ok = false;
            L9[lt9(i, i)] = sqrt(ok ? v : 1.0);
          } else {
            L9[lt9(i, j)] = v / L9[lt9(j, j)];
          }
        }
      }
      double y[9];
      for (int i = 0; i < 9; ++i) {
        double v = rhs[i];
        for (int k = 0; k < i; ++k) v -= L9[lt9(i, k)] * y[k];
        y[i] = v / L9[lt9(i, i)];
      }
      for (int i = 8; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < 9; ++k) v -= L9[lt9(k, i)] * dc[k];
        dc[i] = v / L9[lt9(i, i)];
      }
    }
    if (!ok) continue;
    // ---- candidate: the camera, then each landmark's back substitution, and E^alpha's decrease
    CamT<double> cc = cz;
    double dEc = 0.0;
    if (cam >= 0) {
      double Ex[9];
      rodrigues(dc, Ex);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          cc.R[r * 3 + k] = cz.R[r * 3 + 0] * Ex[0 * 3 + k] + cz.R[r * 3 + 1] * Ex[1 * 3 + k] + cz.R[r * 3 + 2] * Ex[2 * 3 + k];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cc.t[k] = cz.t[k] + dc[3 + k];
        cc.d[k] = cz.d[k] + dc[6 + k];
      }
      dEc = cam_phi(stz, cz, cc, xi);   // inter pairs' P and the camera's proximal term
    }
    double dEl = 0.0;
    for (int e = l0 + lane; e < l1; e += 32) {
      const int j = A.blk_lms[e];
      const double* s = scr + (size_t)j * BS_N;
      double Cm[6], Ci[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) Cm[k] = s[BS_C + k];
      Cm[0] *= 1.0 + mu;
      Cm[2] *= 1.0 + mu;
      Cm[5] *= 1.0 + mu;
      sym3_inv(Cm, Ci);
      double rr[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        rr[k] = s[BS_G + k];
#pragma unroll
        for (int i = 0; i < 9; ++i) rr[k] += s[BS_B + 3 * i + k] * dc[i];
      }
      double dl[3];
      sym3_mul(Ci, rr, dl);
      dl[0] = -dl[0], dl[1] = -dl[1], dl[2] = -dl[2];
      double lz[3];
      blk_lpos(A.lmrec, j, gamma, bar, lz);
      const double* sm = A.lm_sums + (size_t)j * LS_N;
      const double dd = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
      dEl += sm[ao] * dd + 2.0 * (dl[0] * sm[bo] + dl[1] * sm[bo + 1] + dl[2] * sm[bo + 2]) + 0.5 * xi * dd;
      const int o = A.blk_obs[e];
      if (o >= 0 && cam >= 0) {
        const double2 u = A.c_u[o];
        const double lc[3] = {lz[0] + dl[0], lz[1] + dl[1], lz[2] + dl[2]};
        dEl += blk_F(cc, lc, u.x, u.y, A.L, loss) - s[BS_FZ];
      }
    }
    const double dE = dEc + warp_sum(dEl);
    if (dE < 0.0) {   // the step is taken: landmarks to the scratch, the camera to cs
      for (int e = l0 + lane; e < l1; e += 32) {
        const int j = A.blk_lms[e];
        double* s = scr + (size_t)j * BS_N;
        double Cm[6], Ci[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) Cm[k] = s[BS_C + k];
        Cm[0] *= 1.0 + mu;
        Cm[2] *= 1.0 + mu;
        Cm[5] *= 1.0 + mu;
        sym3_inv(Cm, Ci);
        double rr[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          rr[k] = s[BS_G + k];
#pragma unroll
          for (int i = 0; i < 9; ++i) rr[k] += s[BS_B + 3 * i + k] * dc[i];
        }
        double dl[3];
        sym3_mul(Ci, rr, dl);
        s[BS_L + 0] -= dl[0];
        s[BS_L + 1] -= dl[1];
        s[BS_L + 2] -= dl[2];
      }
      cs = cc;
      return;
    }
  }
}

// E^alpha(x | x^k) - E^alpha(x^k | x^k) of block b for the solution in scratch scr (landmarks at
// BS_L) and camera cs: the camera's P terms and proximal term from its x^k statistics, each
// landmark's Q terms and proximal term from its x^k sums, and the intra pairs' F_ij differences.
__device__ inline double blk_dE_k(const BlkArgs& A, int b, int lane, int cam, const double* stk, const CamT<double>& ck,
                                  const CamT<double>& cs, double xi, const double* scr, int loss) {
  const int l0 = A.blk_lm_ptr[b], l1 = A.blk_lm_ptr[b + 1];
  double dEl = 0.0;
  for (int e = l0 + lane; e < l1; e += 32) {
    const int j = A.blk_lms[e];
    const double* s = scr + (size_t)j * BS_N;
    double lk[3];
    blk_lpos(A.lmrec, j, 0.0, false, lk);
    const double dl[3] = {s[BS_L] - lk[0], s[BS_L + 1] - lk[1], s[BS_L + 2] - lk[2]};
    const double* sm = A.lm_sums + (size_t)j * LS_N;
    const double dd = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
    dEl += sm[LS_AK] * dd + 2.0 * (dl[0] * sm[LS_BK] + dl[1] * sm[LS_BK + 1] + dl[2] * sm[LS_BK + 2]) + 0.5 * xi * dd;
    const int o = A.blk_obs[e];
    if (o >= 0 && cam >= 0) {
      const double2 u = A.c_u[o];
      dEl += blk_F(cs, s + BS_L, u.x, u.y, A.L, loss) - blk_F(ck, lk, u.x, u.y, A.L, loss);
    }
  }
  return (cam >= 0 ? cam_phi(stk, ck, cs, xi) : 0.0) + warp_sum(dEl);
}

__global__ void __launch_bounds__(128) k_blk_solve(BlkArgs A, IterParams P, int loss) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (b >= A.S) return;
  const int it = *P.it, first = *P.first;
  const double gamma = P.gam[it], xi = P.xi;
  const int cam = A.blk_cam[b];
  const int l0 = A.blk_lm_ptr[b], l1 = A.blk_lm_ptr[b + 1];
  // ---- the camera's x^k, x^(k-1) displacement, statistics and F sums
  CamT<double> ck, cb;
  double st_b[39], st_k[39];
  double Fall = 0.0, Fin = 0.0, Gc = 0.0, disp = 0.0;
  double* x = nullptr;
  double* dx = nullptr;
  if (cam >= 0) {
    x = A.cam_x + (size_t)cam * CSTRIDE;
    dx = A.cam_dx + (size_t)cam * CSTRIDE;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      ck.R[a] = x[CS_R + a];
      cb.R[a] = A.cam_Rbar[(size_t)cam * 9 + a];
      disp += dx[CS_R + a] * dx[CS_R + a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ck.t[a] = x[CS_T + a];
      ck.d[a] = x[CS_D + a];
      cb.t[a] = ck.t[a] + gamma * dx[CS_T + a];
      cb.d[a] = ck.d[a] + gamma * dx[CS_D + a];
      disp += dx[CS_T + a] * dx[CS_T + a] + dx[CS_D + a] * dx[CS_D + a];
    }
    const int c0 = A.cam_chunk_ptr[cam], c1 = A.cam_chunk_ptr[cam + 1];
    sum_stats<double, double>(A.part, c0, c1, PART_XB, st_b);
    sum_stats<double, double>(A.part, c0, c1, PART_XK, st_k);
    for (int c = c0; c < c1; ++c) {
      Fall += A.part[(size_t)c * CP_STRIDE + PART_F];
      Gc += A.part[(size_t)c * CP_STRIDE + PART_G];
      Fin += A.part[(size_t)c * CP_STRIDE + PART_FI];
    }
  }
  // ---- the landmarks' displacements, gaps and inter F sums
  double dl2 = 0.0, Gl = 0.0, Fl = 0.0;
  for (int e = l0 + lane; e < l1; e += 32) {
    const int j = A.blk_lms[e];
    const V4<double> LA = A.lmrec[2 * (size_t)j], LB = A.lmrec[2 * (size_t)j + 1];
    dl2 += LA.w * LA.w + LB.x * LB.x + LB.y * LB.y;
    Gl += A.lm_sums[(size_t)j * LS_N + LS_G];
    Fl += A.lm_sums[(size_t)j * LS_N + LS_F];
  }
  dl2 = warp_sum(dl2);
  Gl = warp_sum(Gl);
  Fl = warp_sum(Fl);
  // Eq. DEalpha, Eq. Fainit, Eq. Fak, Eq. lFak: E^alpha(x^k | x^k) = sum_E' F + (1/2) sum_E'' F
  const double E0 = Fin + 0.5 * (Fall - Fin) + 0.5 * Fl;
  const double dE = -0.5 * xi * (disp + dl2) + 0.5 * (Gc + Gl);
  const double E = first ? E0 : A.blk_E[b];
  const double Fb_prev = first ? E0 : A.blk_Fbar[b];
  const double F = E + dE;
  const double Fbar = (1.0 - P.eta) * Fb_prev + P.eta * F;
  // ---- accelerated LM step from x̄^k, then the restart test; the MM step from x^k where it fires
  CamT<double> cs = ck;
  double* scr_acc = A.scr;   // the landmark solutions of the step in use (the MM step reuses it)
  bool rs = true;
  double Enext = 0.0;
  if (P.accelerated) {
    blk_lm(A, b, lane, true, gamma, cam, st_b, cb, xi, scr_acc, cs, loss);
    const double dEa = blk_dE_k(A, b, lane, cam, st_k, ck, cs, xi, scr_acc, loss);
    Enext = F + dEa;
    rs = Enext > Fbar;   // Eq. Eak, restart test (strict)
  }
  if (rs) {
    blk_lm(A, b, lane, false, gamma, cam, st_k, ck, xi, scr_acc, cs, loss);
    Enext = F + blk_dE_k(A, b, lane, cam, st_k, ck, cs, xi, scr_acc, loss);
  }
  // ---- new state: landmarks (x^(k+1), displacement), camera, pack of k+1
  for (int e = l0 + lane; e < l1; e += 32) {
    const int j = A.blk_lms[e];
    const double* s = scr_acc + (size_t)j * BS_N;
    const V4<double> LA = A.lmrec[2 * (size_t)j];
    V4<double> nA, nB;
    nA.x = s[BS_L];
    nA.y = s[BS_L + 1];
    nA.z = s[BS_L + 2];
    nA.w = s[BS_L] - LA.x;
    nB.x = s[BS_L + 1] - LA.y;
    nB.y = s[BS_L + 2] - LA.z;
    nB.z = 0.0;
    nB.w = 0.0;
    A.lmrec_out[2 * (size_t)j] = nA;
    A.lmrec_out[2 * (size_t)j + 1] = nB;
  }
  if (lane == 0) {
    A.blk_E[b] = Enext;
    A.blk_Fbar[b] = Fbar;
    A.blk_F[b] = F;
    A.blk_rs[b] = (rs && P.accelerated) ? 1 : 0;
  }
  if (cam >= 0 && lane == 0) {
    A.cam_Fsum[cam] = Fall;
    A.cam_rs[cam] = (rs && P.accelerated) ? 1 : 0;
    CamT<double> ndx;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      ndx.R[a] = cs.R[a] - ck.R[a];
      x[CS_R + a] = cs.R[a];
      dx[CS_R + a] = ndx.R[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ndx.t[a] = cs.t[a] - ck.t[a];
      ndx.d[a] = cs.d[a] - ck.d[a];
      x[CS_T + a] = cs.t[a];
      dx[CS_T + a] = ndx.t[a];
      x[CS_D + a] = cs.d[a];
      dx[CS_D + a] = ndx.d[a];
    }
    const double gn = P.gam[it + 1];
    double K[9], Rb[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) K[a] = cs.R[a] + gn * ndx.R[a];
    extrap_rotation<double>(K, Rb);
#pragma unroll
    for (int a = 0; a < 9; ++a) A.cam_Rbar[(size_t)cam * 9 + a] = Rb[a];
    write_pack_t<double>(cs, ndx, Rb, A.pack_next + (size_t)cam * P4N);
  }
}

}  // namespace daba
