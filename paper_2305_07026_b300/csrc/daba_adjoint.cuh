// daba_adjoint.cuh -- reverse-mode derivative of K iterations of Algorithm 1 (FP64 path).
//
// One iteration maps (x^k, x^(k-1), u) to x^(k+1): the extrapolation x̄^k (Eqs. nesterov_x,
// nesterov_R), per block a conditioning point z (x̄^k for the accelerated update, x^k after a
// restart), the centred statistics of every observation at z, and the block solves
// (landmarks in closed form, cameras by S-CAM). The restart decisions are piecewise constant
// in the inputs and carry no derivative; the adjoint takes them, with the camera statistics
// and the landmark (a, b) sums, from a forward run of the same iterations.
//
// Adjoints of the camera state are ambient: 3x3 for R (only the component tangent to SO(3)
// matters downstream, since every R enters through a polar factor or the boundary), 3 for t,
// 3 for d; of a landmark 3. The adjoint of one iteration has five kernels:
//   k_adj_cams  (thread per camera)   : S-CAM run again with its intermediates, then reversed:
//                                       adjoint of the 39 statistics and of the conditioning
//                                       point from the adjoint of x^(k+1);
//   k_adj_lms   (thread per landmark) : the same for l = l_z - b / (a + xi/2): adjoint of (a, b)
//                                       and of l_z;
//   k_adj_obs   (warp per chunk)      : per observation, the statistics' adjoints pulled back to
//                                       the camera, the landmark and the pixel at x̄^k and at x^k
//                                       (w, lambda, R e as functions of them; rho'' for w);
//   k_adj_lms_sum / k_adj_cams_sum    : per-block sums of those contributions and the adjoint
//                                       of the extrapolation (polar factor for R̄).
#pragma once

#include "daba_grad.cuh"

namespace daba {

// ---- rho''(s) of the losses of rho_w (FP64)
template <int LOSS>
__device__ __forceinline__ double rho_dd(const LossC<double>& L, double s) {
  if (LOSS == LOSS_TRIVIAL) return 0.0;
  if (LOSS == LOSS_HUBER) return s > L.c2 ? -0.5 * L.c / (s * sqrt(s)) : 0.0;
  if (LOSS == LOSS_CAUCHY) {
    const double q = 1.0 / (1.0 + s * L.inv_c2);
    return -L.inv_c2 * q * q;
  }
  return -L.inv_c2 * exp(-s * L.inv_c2);   // Welsch
}

// Adjoint of the polar factor R of K (det K > 0): with S = R^T K (symmetric positive definite),
// dR = R [w]x where (tr(S) I - S) w = vee(R^T dK - dK^T R); for an ambient adjoint Rb of R,
// <Rb, dR> = <K̄, dK> with K̄ = R [h]x, h = (tr(S) I - S)^-1 vee(R^T Rb - Rb^T R).
__device__ inline void polar_vjp(const double* K, const double* R, const double* Rb, double* Kb) {
  double S[9], A[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      S[r * 3 + c] = R[0 * 3 + r] * K[0 * 3 + c] + R[1 * 3 + r] * K[1 * 3 + c] + R[2 * 3 + r] * K[2 * 3 + c];
      A[r * 3 + c] = R[0 * 3 + r] * Rb[0 * 3 + c] + R[1 * 3 + r] * Rb[1 * 3 + c] + R[2 * 3 + r] * Rb[2 * 3 + c];
    }
  const double g0 = A[7] - A[5], g1 = A[2] - A[6], g2 = A[3] - A[1];
  const double tr = S[0] + S[4] + S[8];
  // M = tr I - sym(S)
  const double m00 = tr - S[0], m11 = tr - S[4], m22 = tr - S[8];
  const double m01 = -0.5 * (S[1] + S[3]), m02 = -0.5 * (S[2] + S[6]), m12 = -0.5 * (S[5] + S[7]);
  const double c00 = m11 * m22 - m12 * m12, c01 = m02 * m12 - m01 * m22, c02 = m01 * m12 - m02 * m11;
  const double c11 = m00 * m22 - m02 * m02, c12 = m01 * m02 - m00 * m12, c22 = m00 * m11 - m01 * m01;
  const double det = m00 * c00 + m01 * c01 + m02 * c02;
  const double id = det != 0.0 ? 1.0 / det : 0.0;
  const double h0 = (c00 * g0 + c01 * g1 + c02 * g2) * id;
  const double h1 = (c01 * g0 + c11 * g1 + c12 * g2) * id;
  const double h2 = (c02 * g0 + c12 * g1 + c22 * g2) * id;
  const double H[9] = {0.0, -h2, h1, h2, 0.0, -h0, -h1, h0, 0.0};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      Kb[r * 3 + c] = R[r * 3 + 0] * H[0 * 3 + c] + R[r * 3 + 1] * H[1 * 3 + c] + R[r * 3 + 2] * H[2 * 3 + c];
}

// Intermediates of one S-CAM alternation kept for the reverse sweep.
struct ScamTape {
  double ct[3], cd[3];   // (t, d) entering the alternation
  double K[9], R[9];     // R-step matrix and its polar factor
  double G[3][6];        // W H - B^T
  double W[3][6];
  bool td;               // the (t, d)-step was taken (its system positive definite)
  double v[3], rhs[6], alpha, h[3], f4, f2, S[3][3], yd[3], yt[3], dM0[6][3], dv[6];
};

// S-CAM forward (as cam_scam) recording the tape; n_alt <= 4.
__device__ inline void scam_tape(const double* st, const CamT<double>& z, double xi, int n_alt, CamT<double>& c,
                                 ScamTape* tp) {
  using N = Num<double>;
  c = z;
  for (int it = 0; it < n_alt; ++it) {
    ScamTape& T = tp[it];
    for (int k = 0; k < 3; ++k) {
      T.ct[k] = c.t[k];
      T.cd[k] = c.d[k];
    }
    for (int a = 0; a < 6; ++a) {
      double mz[3];
      mcol(z, a, mz);
      T.W[0][a] = mz[0];
      T.W[1][a] = mz[1];
      T.W[2][a] = mz[2];
    }
    for (int r = 0; r < 3; ++r) T.W[r][5] = z.t[r] - c.t[r];
    for (int r = 0; r < 3; ++r)
      for (int a = 0; a < 6; ++a) {
        double s = -st_B(st, a, r);
        for (int b = 0; b < 6; ++b) s = s + T.W[r][b] * st_H(st, b, a);
        T.G[r][a] = s;
      }
    for (int r = 0; r < 3; ++r) {
      T.K[r * 3 + 0] = xi * z.R[r * 3 + 0] + 2.0 * T.G[r][0];
      T.K[r * 3 + 1] = xi * z.R[r * 3 + 1] + 2.0 * T.G[r][1];
      T.K[r * 3 + 2] = xi * z.R[r * 3 + 2] + 2.0 * (c.d[0] * T.G[r][2] + c.d[1] * T.G[r][3] + c.d[2] * T.G[r][4]);
    }
    double Rn[9];
    if (proj_rot3d_from(T.K, c.R, Rn)) {
      for (int a = 0; a < 9; ++a) c.R[a] = Rn[a];
    } else {
      proj_rot3d_polar(T.K, c.R);
    }
    for (int a = 0; a < 9; ++a) T.R[a] = c.R[a];
    const double v[3] = {c.R[2], c.R[5], c.R[8]};
    const double vz[3] = {z.R[2], z.R[5], z.R[8]};
    for (int k = 0; k < 3; ++k) {
      T.v[k] = v[k];
      T.dM0[0][k] = c.R[k * 3 + 0] - z.R[k * 3 + 0];
      T.dM0[1][k] = c.R[k * 3 + 1] - z.R[k * 3 + 1];
      T.dM0[2][k] = z.d[0] * (v[k] - vz[k]);
      T.dM0[3][k] = z.d[1] * (v[k] - vz[k]);
      T.dM0[4][k] = z.d[2] * (v[k] - vz[k]);
      T.dM0[5][k] = 0.0;
    }
    for (int a = 0; a < 6; ++a) T.dv[a] = T.dM0[a][0] * v[0] + T.dM0[a][1] * v[1] + T.dM0[a][2] * v[2];
    for (int k = 0; k < 3; ++k) {
      double s = st_B(st, 5, k);
      for (int a = 0; a < 6; ++a) s = s + T.dM0[a][k] * st_H(st, a, 5);
      T.rhs[k] = -2.0 * s;
    }
    for (int m = 0; m < 3; ++m) {
      double s = st_B(st, 2 + m, 0) * v[0] + st_B(st, 2 + m, 1) * v[1] + st_B(st, 2 + m, 2) * v[2];
      for (int a = 0; a < 6; ++a) s = s + st_H(st, 2 + m, a) * T.dv[a];
      T.rhs[3 + m] = -2.0 * s;
    }
    T.td = false;
    T.alpha = 2.0 * st_H(st, 5, 5) + xi;
    if (N::pos(T.alpha)) {
      const double ia = 1.0 / T.alpha;
      for (int m = 0; m < 3; ++m) T.h[m] = st_H(st, 2 + m, 5);
      const double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
      const double vr = v[0] * T.rhs[0] + v[1] * T.rhs[1] + v[2] * T.rhs[2];
      T.f4 = 4.0 * vv * ia;
      T.f2 = 2.0 * vr * ia;
      double r[3];
      for (int m = 0; m < 3; ++m) {
        for (int n = 0; n < 3; ++n) T.S[m][n] = 2.0 * st_H(st, 2 + m, 2 + n) - T.f4 * T.h[m] * T.h[n];
        T.S[m][m] = T.S[m][m] + xi;
        r[m] = T.rhs[3 + m] - T.f2 * T.h[m];
      }
      const double m1 = T.S[0][0] * T.S[1][1] - T.S[0][1] * T.S[0][1];
      const double c00 = T.S[1][1] * T.S[2][2] - T.S[1][2] * T.S[1][2], c01 = T.S[0][2] * T.S[1][2] - T.S[0][1] * T.S[2][2];
      const double c02 = T.S[0][1] * T.S[1][2] - T.S[0][2] * T.S[1][1], c11 = T.S[0][0] * T.S[2][2] - T.S[0][2] * T.S[0][2];
      const double c12 = T.S[0][1] * T.S[0][2] - T.S[0][0] * T.S[1][2];
      const double det = T.S[0][0] * c00 + T.S[0][1] * c01 + T.S[0][2] * c02;
      if (T.S[0][0] > 0.0 && m1 > 0.0 && det > 0.0) {
        const double id = 1.0 / det;
        T.yd[0] = (c00 * r[0] + c01 * r[1] + c02 * r[2]) * id;
        T.yd[1] = (c01 * r[0] + c11 * r[1] + c12 * r[2]) * id;
        T.yd[2] = (c02 * r[0] + c12 * r[1] + m1 * r[2]) * id;
        const double hy = 2.0 * (T.h[0] * T.yd[0] + T.h[1] * T.yd[1] + T.h[2] * T.yd[2]);
        for (int k = 0; k < 3; ++k) {
          T.yt[k] = (T.rhs[k] - v[k] * hy) * ia;
          c.t[k] = z.t[k] + T.yt[k];
          c.d[k] = z.d[k] + T.yd[k];
        }
        T.td = true;
      }
    }
  }
}

// 3x3 symmetric solve (Cramer) of the tape's S for a right-hand side
__device__ inline void solve_S(const double S[3][3], const double* b, double* x) {
  const double m1 = S[0][0] * S[1][1] - S[0][1] * S[0][1];
  const double c00 = S[1][1] * S[2][2] - S[1][2] * S[1][2], c01 = S[0][2] * S[1][2] - S[0][1] * S[2][2];
  const double c02 = S[0][1] * S[1][2] - S[0][2] * S[1][1], c11 = S[0][0] * S[2][2] - S[0][2] * S[0][2];
  const double c12 = S[0][1] * S[0][2] - S[0][0] * S[1][2];
  const double id = 1.0 / (S[0][0] * c00 + S[0][1] * c01 + S[0][2] * c02);
  x[0] = (c00 * b[0] + c01 * b[1] + c02 * b[2]) * id;
  x[1] = (c01 * b[0] + c11 * b[1] + c12 * b[2]) * id;
  x[2] = (c02 * b[0] + c12 * b[1] + m1 * b[2]) * id;
}

// Reverse sweep of S-CAM: from the adjoint of its result (cb: R ambient, t, d) to the adjoint
// of the statistics (Hb full 6x6, Bb 6x3) and of the conditioning point (zb).
__device__ inline void scam_adjoint(const double* st, const CamT<double>& z, double xi, int n_alt, const ScamTape* tp,
                                    CamT<double> cb, double Hb[6][6], double Bb[6][3], CamT<double>& zb) {
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) Hb[a][b] = 0.0;
  for (int a = 0; a < 6; ++a)
    for (int c = 0; c < 3; ++c) Bb[a][c] = 0.0;
  for (int a = 0; a < 9; ++a) zb.R[a] = 0.0;
  for (int k = 0; k < 3; ++k) zb.t[k] = zb.d[k] = 0.0;
  for (int it = n_alt - 1; it >= 0; --it) {
    const ScamTape& T = tp[it];
    // ---- (t, d)-step: c.t = z.t + yt, c.d = z.d + yd (or unchanged when skipped)
    double ctb[3], cdb[3];   // adjoint of (t, d) entering the alternation (from this step)
    double Rb[9];            // adjoint of this alternation's R (ambient)
    for (int a = 0; a < 9; ++a) Rb[a] = cb.R[a];
    if (!T.td) {
      for (int k = 0; k < 3; ++k) {
        ctb[k] = cb.t[k];
        cdb[k] = cb.d[k];
      }
    } else {
      for (int k = 0; k < 3; ++k) {
        zb.t[k] += cb.t[k];
        zb.d[k] += cb.d[k];
        ctb[k] = 0.0;
        cdb[k] = 0.0;
      }
      const double ia = 1.0 / T.alpha;
      const double hy = 2.0 * (T.h[0] * T.yd[0] + T.h[1] * T.yd[1] + T.h[2] * T.yd[2]);
      double rhsb[6] = {0, 0, 0, 0, 0, 0}, vb[3] = {0, 0, 0}, hb[3] = {0, 0, 0}, alphab = 0.0;
      // yt = (rhs_t - v hy) / alpha
      double hyb = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double ytb = cb.t[k];
        rhsb[k] += ytb * ia;
        vb[k] += -hy * ytb * ia;
        hyb += -T.v[k] * ytb * ia;
        alphab += -T.yt[k] * ytb * ia;
      }
      // hy = 2 h . yd
      double ydb[3];
      for (int m = 0; m < 3; ++m) {
        hb[m] += 2.0 * hyb * T.yd[m];
        ydb[m] = cb.d[m] + 2.0 * hyb * T.h[m];
      }
      // yd = S^-1 r
      double rb[3];
      solve_S(T.S, ydb, rb);
      double Sb[3][3];
      for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) Sb[m][n] = -rb[m] * T.yd[n];
      // S = 2 H[2:5,2:5] - f4 h h^T + xi I ;  r = rhs_d - f2 h
      double f4b = 0.0, f2b = 0.0;
      for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) {
          Hb[2 + m][2 + n] += 2.0 * Sb[m][n];
          f4b += -Sb[m][n] * T.h[m] * T.h[n];
        }
      // d(h_m h_n) = h_n dh_m + h_m dh_n
      for (int m = 0; m < 3; ++m) {
        double s = 0.0;
        for (int n = 0; n < 3; ++n) s += (Sb[m][n] + Sb[n][m]) * T.h[n];
        hb[m] += -T.f4 * s;
      }
      for (int m = 0; m < 3; ++m) {
        rhsb[3 + m] += rb[m];
        f2b += -rb[m] * T.h[m];
        hb[m] += -T.f2 * rb[m];
      }
      // f4 = 4 vv / alpha, f2 = 2 vr / alpha
      const double vvb = 4.0 * f4b * ia, vrb = 2.0 * f2b * ia;
      alphab += -T.f4 * f4b * ia - T.f2 * f2b * ia;
      for (int k = 0; k < 3; ++k) {
        vb[k] += 2.0 * vvb * T.v[k] + vrb * T.rhs[k];
        rhsb[k] += vrb * T.v[k];
      }
      // alpha = 2 H55 + xi ; h = H[2:5, 5]
      Hb[5][5] += 2.0 * alphab;
      for (int m = 0; m < 3; ++m) Hb[2 + m][5] += hb[m];
      // rhs_t[k] = -2 (B[5][k] + sum_a dM0[a][k] H[a][5])
      double dM0b[6][3];
      for (int a = 0; a < 6; ++a)
        for (int k = 0; k < 3; ++k) dM0b[a][k] = 0.0;
      for (int k = 0; k < 3; ++k) {
        Bb[5][k] += -2.0 * rhsb[k];
        for (int a = 0; a < 6; ++a) {
          dM0b[a][k] += -2.0 * rhsb[k] * st_H(st, a, 5);
          Hb[a][5] += -2.0 * rhsb[k] * T.dM0[a][k];
        }
      }
      // rhs_d[m] = -2 (B[2+m] . v + sum_a H[2+m][a] dv[a])
      double dvb[6] = {0, 0, 0, 0, 0, 0};
      for (int m = 0; m < 3; ++m) {
        const double g = -2.0 * rhsb[3 + m];
        for (int k = 0; k < 3; ++k) {
          Bb[2 + m][k] += g * T.v[k];
          vb[k] += g * st_B(st, 2 + m, k);
        }
        for (int a = 0; a < 6; ++a) {
          Hb[2 + m][a] += g * T.dv[a];
          dvb[a] += g * st_H(st, 2 + m, a);
        }
      }
      // dv[a] = dM0[a] . v
      for (int a = 0; a < 6; ++a)
        for (int k = 0; k < 3; ++k) {
          dM0b[a][k] += dvb[a] * T.v[k];
          vb[k] += dvb[a] * T.dM0[a][k];
        }
      // dM0: columns 0, 1 of R - R_z; rows 2..4 z.d[m] (v - vz)
      for (int k = 0; k < 3; ++k) {
        Rb[k * 3 + 0] += dM0b[0][k];
        zb.R[k * 3 + 0] -= dM0b[0][k];
        Rb[k * 3 + 1] += dM0b[1][k];
        zb.R[k * 3 + 1] -= dM0b[1][k];
        const double vzk = z.R[k * 3 + 2];
        for (int m = 0; m < 3; ++m) {
          zb.d[m] += dM0b[2 + m][k] * (T.v[k] - vzk);
          vb[k] += z.d[m] * dM0b[2 + m][k];
          zb.R[k * 3 + 2] -= z.d[m] * dM0b[2 + m][k];
        }
      }
      for (int k = 0; k < 3; ++k) Rb[k * 3 + 2] += vb[k];
    }
    // ---- R-step: R = polar(K), K = xi R_z + 2 G P(c.d)^T, G = W H - B^T
    double Kb[9];
    polar_vjp(T.K, T.R, Rb, Kb);
    double Gb[3][6];
    for (int r = 0; r < 3; ++r) {
      zb.R[r * 3 + 0] += xi * Kb[r * 3 + 0];
      zb.R[r * 3 + 1] += xi * Kb[r * 3 + 1];
      zb.R[r * 3 + 2] += xi * Kb[r * 3 + 2];
      Gb[r][0] = 2.0 * Kb[r * 3 + 0];
      Gb[r][1] = 2.0 * Kb[r * 3 + 1];
      for (int m = 0; m < 3; ++m) {
        Gb[r][2 + m] = 2.0 * T.cd[m] * Kb[r * 3 + 2];
        cdb[m] += 2.0 * T.G[r][2 + m] * Kb[r * 3 + 2];
      }
      Gb[r][5] = 0.0;
    }
    // G[r][a] = sum_b W[r][b] H[b][a] - B[a][r]
    double Wb[3][6];
    for (int r = 0; r < 3; ++r)
      for (int b = 0; b < 6; ++b) {
        double s = 0.0;
        for (int a = 0; a < 6; ++a) s += Gb[r][a] * st_H(st, b, a);
        Wb[r][b] = s;
      }
    for (int b = 0; b < 6; ++b)
      for (int a = 0; a < 6; ++a) {
        double s = 0.0;
        for (int r = 0; r < 3; ++r) s += T.W[r][b] * Gb[r][a];
        Hb[b][a] += s;
      }
    for (int a = 0; a < 6; ++a)
      for (int r = 0; r < 3; ++r) Bb[a][r] += -Gb[r][a];
    // W[:, a] = mcol(z, a) (a < 5), W[:, 5] = z.t - c.t
    for (int r = 0; r < 3; ++r) {
      zb.R[r * 3 + 0] += Wb[r][0];
      zb.R[r * 3 + 1] += Wb[r][1];
      for (int m = 0; m < 3; ++m) {
        zb.d[m] += Wb[r][2 + m] * z.R[r * 3 + 2];
        zb.R[r * 3 + 2] += z.d[m] * Wb[r][2 + m];
      }
      zb.t[r] += Wb[r][5];
      ctb[r] += -Wb[r][5];
    }
    // the adjoint of (R, t, d) entering this alternation: R entering only seeds the warm start
    // (no derivative); (t, d) entering are the previous alternation's results (or z)
    for (int a = 0; a < 9; ++a) cb.R[a] = 0.0;
    for (int k = 0; k < 3; ++k) {
      cb.t[k] = ctb[k];
      cb.d[k] = cdb[k];
    }
  }
  // entering the first alternation c = z
  for (int k = 0; k < 3; ++k) {
    zb.t[k] += cb.t[k];
    zb.d[k] += cb.d[k];
  }
}

// Reverse sweep of the LM camera step (cam_lm): from the adjoint of its result (cb: R ambient,
// t, d) to the adjoint of the statistics (Hb full 6x6, Bb 6x3) and of the conditioning point (zb).
// The forward step is replayed with the same arithmetic to find the damping trial it took; the
// choice is piecewise constant and carries no derivative. Taken step: c = (z.R Exp(phi),
// z.t + tau, z.d + delta) with theta = -(A + mu diag A)^-1 g, so with v = (A_mu)^-1 theta_bar,
// g_bar = -v and A_mu_bar = -v theta^T; no step taken: c = z.
__device__ inline void lm_model_adjoint(const double* st, const CamT<double>& z, const double* Ab, const double* gb,
                                        double Hb[6][6], double Bb[6][3], CamT<double>& zb);

__device__ inline void lm_adjoint(const double* st, const CamT<double>& z, double xi, const CamT<double>& cb,
                                  double Hb[6][6], double Bb[6][3], CamT<double>& zb) {
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) Hb[a][b] = 0.0;
  for (int a = 0; a < 6; ++a)
    for (int c = 0; c < 3; ++c) Bb[a][c] = 0.0;
  for (int a = 0; a < 9; ++a) zb.R[a] = 0.0;
  for (int k = 0; k < 3; ++k) zb.t[k] = zb.d[k] = 0.0;
  double A[45], g[9], L[45], th[9], mu = LM_MU0;
  cam_lm_model(st, z, xi, A, g);
  bool taken = false;
  for (int tr = 0; tr < LM_TRIES && !taken; ++tr, mu *= 10.0) {   // replay of cam_lm
    bool ok = true;
    for (int i = 0; i < 9; ++i)
      for (int j = 0; j <= i; ++j) {
        double v = A[lt9(i, j)] * (i == j ? 1.0 + mu : 1.0);
        for (int k = 0; k < j; ++k) v -= L[lt9(i, k)] * L[lt9(j, k)];
        if (i == j) {
          if (!(v > 0.0)) ok = false;
          L[lt9(i, i)] = sqrt(ok ? v : 1.0);
        } else {
          L[lt9(i, j)] = v / L[lt9(j, j)];
        }
      }
    if (!ok) continue;
    double y[9];
    for (int i = 0; i < 9; ++i) {
      double v = -g[i];
      for (int k = 0; k < i; ++k) v -= L[lt9(i, k)] * y[k];
      y[i] = v / L[lt9(i, i)];
    }
    for (int i = 8; i >= 0; --i) {
      double v = y[i];
      for (int k = i + 1; k < 9; ++k) v -= L[lt9(k, i)] * th[k];
      th[i] = v / L[lt9(i, i)];
    }
    CamT<double> cand;
    double E[9];
    rodrigues(th, E);
    for (int r = 0; r < 3; ++r)
      for (int cc = 0; cc < 3; ++cc)
        cand.R[r * 3 + cc] = z.R[r * 3 + 0] * E[0 * 3 + cc] + z.R[r * 3 + 1] * E[1 * 3 + cc] + z.R[r * 3 + 2] * E[2 * 3 + cc];
    for (int k = 0; k < 3; ++k) {
      cand.t[k] = z.t[k] + th[3 + k];
      cand.d[k] = z.d[k] + th[6 + k];
    }
    if (cam_phi(st, z, cand, xi) < 0.0) {
      taken = true;
      break;
    }
  }
  if (!taken) {   // the camera stayed at c_z
    for (int a = 0; a < 9; ++a) zb.R[a] = cb.R[a];
    for (int k = 0; k < 3; ++k) zb.t[k] = cb.t[k], zb.d[k] = cb.d[k];
    return;
  }
  // R = z.R E(phi): z.R_bar = R_bar E^T; E_bar = z.R^T R_bar, then phi_bar = J_r(phi)^T vee(E^T E_bar)
  double E[9];
  rodrigues(th, E);
  for (int r = 0; r < 3; ++r)
    for (int cc = 0; cc < 3; ++cc)
      zb.R[r * 3 + cc] = cb.R[r * 3 + 0] * E[cc * 3 + 0] + cb.R[r * 3 + 1] * E[cc * 3 + 1] + cb.R[r * 3 + 2] * E[cc * 3 + 2];
  double Eb[9], Mx[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      Eb[i * 3 + j] = z.R[0 * 3 + i] * cb.R[0 * 3 + j] + z.R[1 * 3 + i] * cb.R[1 * 3 + j] + z.R[2 * 3 + i] * cb.R[2 * 3 + j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      Mx[i * 3 + j] = E[0 * 3 + i] * Eb[0 * 3 + j] + E[1 * 3 + i] * Eb[1 * 3 + j] + E[2 * 3 + i] * Eb[2 * 3 + j];
  const double v2[3] = {Mx[7] - Mx[5], Mx[2] - Mx[6], Mx[3] - Mx[1]};
  // J_r(phi)^T = I + b [phi]x + c [phi]x^2, b = (1 - cos t)/t^2, c = (t - sin t)/t^3
  const double t2 = th[0] * th[0] + th[1] * th[1] + th[2] * th[2], tn = sqrt(t2);
  double bj, cj;
  if (tn < 1e-4) {
    bj = 0.5 - t2 / 24.0;
    cj = 1.0 / 6.0 - t2 / 120.0;
  } else {
    bj = (1.0 - cos(tn)) / t2;
    cj = (tn - sin(tn)) / (t2 * tn);
  }
  const double px[3] = {th[1] * v2[2] - th[2] * v2[1], th[2] * v2[0] - th[0] * v2[2], th[0] * v2[1] - th[1] * v2[0]};
  const double ppx[3] = {th[1] * px[2] - th[2] * px[1], th[2] * px[0] - th[0] * px[2], th[0] * px[1] - th[1] * px[0]};
  double thb[9];
  for (int k = 0; k < 3; ++k) thb[k] = v2[k] + bj * px[k] + cj * ppx[k];
  for (int k = 0; k < 3; ++k) {
    thb[3 + k] = cb.t[k];
    thb[6 + k] = cb.d[k];
    zb.t[k] = cb.t[k];
    zb.d[k] = cb.d[k];
  }
  // theta = -(A_mu)^-1 g: v = (A_mu)^-1 theta_bar by the Cholesky factor of the taken trial
  double y[9], v[9];
  for (int i = 0; i < 9; ++i) {
    double s = thb[i];
    for (int k = 0; k < i; ++k) s -= L[lt9(i, k)] * y[k];
    y[i] = s / L[lt9(i, i)];
  }
  for (int i = 8; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 9; ++k) s -= L[lt9(k, i)] * v[k];
    v[i] = s / L[lt9(i, i)];
  }
  double gbar[9], Abp[45];   // adjoints of g and of the packed lower A (A_mu = A (1 + mu on the diagonal))
  for (int i = 0; i < 9; ++i) {
    gbar[i] = -v[i];
    for (int j = 0; j <= i; ++j)
      Abp[lt9(i, j)] = i == j ? -v[i] * th[i] * (1.0 + mu) : -(v[i] * th[j] + v[j] * th[i]);
  }
  lm_model_adjoint(st, z, Abp, gbar, Hb, Bb, zb);
}

// Adjoint of cam_lm_model: from the adjoints of the packed lower model Hessian (Ab) and of its
// gradient (gb) to the statistics (added to Hb[a][b] for st_H(a, b), Bb) and to z.R, z.d (added
// to zb; the model does not depend on z.t). Each block below reverses the matching forward line.
__device__ inline void lm_model_adjoint(const double* st, const CamT<double>& z, const double* Ab, const double* gb,
                                        double Hb[6][6], double Bb[6][3], CamT<double>& zb) {
  double q[6][3];
  for (int b = 0; b < 6; ++b) {
    q[b][0] = st_H(st, 0, b);
    q[b][1] = st_H(st, 1, b);
    q[b][2] = z.d[0] * st_H(st, 2, b) + z.d[1] * st_H(st, 3, b) + z.d[2] * st_H(st, 4, b);
  }
  double qb[6][3] = {}, Qb[3][3] = {};
  // gradient: g[3+k] = 2 B5k; g[6+n] = 2 sum_r R[r][2] B(2+n, r); g[0..2] from bc = R^T B_a
  for (int k = 0; k < 3; ++k) Bb[5][k] += 2.0 * gb[3 + k];
  for (int n = 0; n < 3; ++n)
    for (int r = 0; r < 3; ++r) {
      Bb[2 + n][r] += 2.0 * gb[6 + n] * z.R[r * 3 + 2];
      zb.R[r * 3 + 2] += 2.0 * gb[6 + n] * st_B(st, 2 + n, r);
    }
  double bc[5][3], bcb[5][3] = {};
  for (int a = 0; a < 5; ++a)
    for (int k = 0; k < 3; ++k)
      bc[a][k] = z.R[0 * 3 + k] * st_B(st, a, 0) + z.R[1 * 3 + k] * st_B(st, a, 1) + z.R[2 * 3 + k] * st_B(st, a, 2);
  const double g0 = 2.0 * gb[0], g1 = 2.0 * gb[1], g2 = 2.0 * gb[2];
  bcb[1][2] += g0;
  bcb[0][2] -= g1;
  bcb[0][1] += g2;
  bcb[1][0] -= g2;
  for (int m = 0; m < 3; ++m) {
    bcb[2 + m][1] -= z.d[m] * g0;
    bcb[2 + m][0] += z.d[m] * g1;
    zb.d[m] += -g0 * bc[2 + m][1] + g1 * bc[2 + m][0];
  }
  for (int a = 0; a < 5; ++a)
    for (int k = 0; k < 3; ++k)
      for (int r = 0; r < 3; ++r) {
        Bb[a][r] += bcb[a][k] * z.R[r * 3 + k];
        zb.R[r * 3 + k] += bcb[a][k] * st_B(st, a, r);
      }
  // phi block: A_ij = 2 (delta_ij tr Q - (Q_ij + Q_ji) / 2) + 2 xi delta_ij
  double trQb = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j <= i; ++j) {
      const double a = Ab[lt9(i, j)];
      if (i == j) trQb += 2.0 * a;
      Qb[i][j] -= a;
      Qb[j][i] -= a;
    }
  for (int r = 0; r < 3; ++r) Qb[r][r] += trQb;
  // tau rows: A[3+c][.] = -2 r_c x q_5 (r_c row c of R_z), diagonal 2 H55 + xi
  for (int cc = 0; cc < 3; ++cc) {
    const double r0 = z.R[cc * 3 + 0], r1 = z.R[cc * 3 + 1], r2 = z.R[cc * 3 + 2];
    const double a0 = Ab[lt9(3 + cc, 0)], a1 = Ab[lt9(3 + cc, 1)], a2 = Ab[lt9(3 + cc, 2)];
    zb.R[cc * 3 + 1] += -2.0 * a0 * q[5][2] + 2.0 * a2 * q[5][0];
    zb.R[cc * 3 + 2] += 2.0 * a0 * q[5][1] - 2.0 * a1 * q[5][0];
    zb.R[cc * 3 + 0] += 2.0 * a1 * q[5][2] - 2.0 * a2 * q[5][1];
    qb[5][2] += -2.0 * a0 * r1 + 2.0 * a1 * r0;
    qb[5][1] += 2.0 * a0 * r2 - 2.0 * a2 * r0;
    qb[5][0] += -2.0 * a1 * r2 + 2.0 * a2 * r1;
    Hb[5][5] += 2.0 * Ab[lt9(3 + cc, 3 + cc)];
  }
  // delta rows: A[6+n][0] = 2 q[2+n][1], A[6+n][1] = -2 q[2+n][0], A[6+n][3+c] = 2 H(5, 2+n) R[c][2],
  // A[6+n][6+m] = 2 H(2+n, 2+m) (+ xi on the diagonal)
  for (int n = 0; n < 3; ++n) {
    qb[2 + n][1] += 2.0 * Ab[lt9(6 + n, 0)];
    qb[2 + n][0] -= 2.0 * Ab[lt9(6 + n, 1)];
    for (int cc = 0; cc < 3; ++cc) {
      const double a = Ab[lt9(6 + n, 3 + cc)];
      Hb[5][2 + n] += 2.0 * a * z.R[cc * 3 + 2];
      zb.R[cc * 3 + 2] += 2.0 * a * st_H(st, 5, 2 + n);
    }
    for (int m = 0; m <= n; ++m) Hb[2 + n][2 + m] += 2.0 * Ab[lt9(6 + n, 6 + m)];
  }
  // Q[r] = (q0_r, q1_r, sum_m d_m q(2+m)_r), then q from H
  for (int r = 0; r < 3; ++r) {
    qb[0][r] += Qb[r][0];
    qb[1][r] += Qb[r][1];
    for (int m = 0; m < 3; ++m) {
      qb[2 + m][r] += z.d[m] * Qb[r][2];
      zb.d[m] += Qb[r][2] * q[2 + m][r];
    }
  }
  for (int b = 0; b < 6; ++b) {
    Hb[0][b] += qb[b][0];
    Hb[1][b] += qb[b][1];
    for (int m = 0; m < 3; ++m) {
      Hb[2 + m][b] += z.d[m] * qb[b][2];
      zb.d[m] += qb[b][2] * st_H(st, 2 + m, b);
    }
  }
}

// Adjoint buffers: per camera 16 doubles (R ambient 9, t 3, d 3, pad), per landmark 4 (l, pad).
enum { AC_R = 0, AC_T = 9, AC_D = 12, AC_N = 16, AL_N = 4 };

__device__ inline void load_cam(const double* x, CamT<double>& c) {
  for (int a = 0; a < 9; ++a) c.R[a] = x[CS_R + a];
  for (int k = 0; k < 3; ++k) {
    c.t[k] = x[CS_T + k];
    c.d[k] = x[CS_D + k];
  }
}

// x̄^k of a camera: R̄ = ProjRot3D(R + gamma dR) as the forward computes it, t, d linear
__device__ inline void cam_bar(const CamT<double>& ck, const double* dx, double gamma, CamT<double>& cb, double* Kx) {
  for (int a = 0; a < 9; ++a) Kx[a] = ck.R[a] + gamma * dx[CS_R + a];
  proj_rot3d_near(Kx, cb.R);
  for (int k = 0; k < 3; ++k) {
    cb.t[k] = ck.t[k] + gamma * dx[CS_T + k];
    cb.d[k] = ck.d[k] + gamma * dx[CS_D + k];
  }
}

// 1. The camera solve reversed per camera (S-CAM, or with lm the LM step): adjoint of the chosen
//    statistics (packed, 40 per camera) and of the conditioning point (added to zb_bar or zb_k by
//    the camera's decision).
__global__ void k_adj_cams(int M, const int* __restrict__ cam_chunk_ptr, const double* __restrict__ part,
                           const double* __restrict__ sx, const double* __restrict__ sdx, double gamma,
                           const uint8_t* __restrict__ rs_cam, int accelerated, double xi, int n_alt, int lm,
                           const double* __restrict__ a_next, double* __restrict__ st_bar,
                           double* __restrict__ zb_bar, double* __restrict__ zb_k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const bool mm = !accelerated || rs_cam[i];
  const int c0 = cam_chunk_ptr[i], c1 = cam_chunk_ptr[i + 1];
  double st[39];
  sum_stats<double, double>(part, c0, c1, mm ? PART_XK : PART_XB, st);
  CamT<double> ck, z, cn;
  load_cam(sx + (size_t)i * CSTRIDE, ck);
  if (mm) {
    z = ck;
  } else {
    double Kx[9];
    cam_bar(ck, sdx + (size_t)i * CSTRIDE, gamma, z, Kx);
  }
  CamT<double> cb, zb;
  const double* an = a_next + (size_t)i * AC_N;
  for (int a = 0; a < 9; ++a) cb.R[a] = an[AC_R + a];
  for (int k = 0; k < 3; ++k) {
    cb.t[k] = an[AC_T + k];
    cb.d[k] = an[AC_D + k];
  }
  double Hb[6][6], Bb[6][3];
  if (lm) {   // the LM camera solver variant
    lm_adjoint(st, z, xi, cb, Hb, Bb, zb);
  } else {
    ScamTape tp[4];
    scam_tape(st, z, xi, n_alt, cn, tp);
    scam_adjoint(st, z, xi, n_alt, tp, cb, Hb, Bb, zb);
  }
  double* so = st_bar + (size_t)i * 40;
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) so[tri6(a, b)] = a == b ? Hb[a][a] : Hb[a][b] + Hb[b][a];
  for (int a = 0; a < 6; ++a)
    for (int c = 0; c < 3; ++c) so[21 + a * 3 + c] = Bb[a][c];
  so[39] = 0.0;
  double* zo = (mm ? zb_k : zb_bar) + (size_t)i * AC_N;
  for (int a = 0; a < 9; ++a) zo[AC_R + a] += zb.R[a];
  for (int k = 0; k < 3; ++k) {
    zo[AC_T + k] += zb.t[k];
    zo[AC_D + k] += zb.d[k];
  }
}

// 2. the landmark solve reversed, per landmark: l = l_z - b / (a + xi/2) with (a, b) the sums of
//    its records at the chosen point (kept by the landmark pass of the forward sweep: x̄ in
//    sums[0..3], x^k in sums[4..7]); writes (abar, bbar) and adds the adjoint of l_z.
__global__ void k_adj_lms(int N, const double* __restrict__ sums, const uint8_t* __restrict__ rs_lm, int accelerated,
                          double xi, const double* __restrict__ a_next, double* __restrict__ ab_bar,
                          double* __restrict__ zb_bar, double* __restrict__ zb_k) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const bool mm = !accelerated || rs_lm[j];
  const double* sm = sums + (size_t)j * 8 + (mm ? 4 : 0);
  const double a = sm[0], b0 = sm[1], b1 = sm[2], b2 = sm[3];
  const double den = a + 0.5 * xi;
  const double* an = a_next + (size_t)j * AL_N;
  const double g0 = an[0], g1 = an[1], g2 = an[2];
  double* o = ab_bar + (size_t)j * 4;
  o[0] = (g0 * b0 + g1 * b1 + g2 * b2) / (den * den);
  o[1] = -g0 / den;
  o[2] = -g1 / den;
  o[3] = -g2 / den;
  double* zo = (mm ? zb_k : zb_bar) + (size_t)j * AL_N;
  zo[0] += g0;
  zo[1] += g1;
  zo[2] += g2;
}

// Per observation at one point (R, t, d, l), pixel u: the contributions w h h^T, w h (E/2)^T to
// the camera statistics and w lambda^2, -w lambda E/2 to the landmark's (a, b), pulled back from
// their adjoints (sb: 39 packed camera-statistics adjoints or null; ab: (abar, bbar[3]) or null)
// to R (ambient), t, d, l and the pixel u (internal units). Results are added to the outputs.
template <int LOSS>
__device__ inline void obs_pullback(const double* R, const double* t, const double* d, const double* l, double u0,
                                    double u1, const double* sb, const double* ab, const LossC<double>& L, double* Rb,
                                    double* tb, double* db, double* lb, double* ub) {
  const double sq = u0 * u0 + u1 * u1;
  const double p[3] = {u0, u1, d[0] + d[1] * sq + d[2] * sq * sq};
  const double q[3] = {l[0] - t[0], l[1] - t[1], l[2] - t[2]};
  double Rp[3];
  for (int r = 0; r < 3; ++r) Rp[r] = R[r * 3 + 0] * p[0] + R[r * 3 + 1] * p[1] + R[r * 3 + 2] * p[2];
  const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
  const double lam = (q[0] * Rp[0] + q[1] * Rp[1] + q[2] * Rp[2]) / qq;
  const double E[3] = {Rp[0] - lam * q[0], Rp[1] - lam * q[1], Rp[2] - lam * q[2]};
  const double r2 = E[0] * E[0] + E[1] * E[1] + E[2] * E[2];
  double rho, w;
  rho_w<LOSS, double>(L, r2, rho, w);
  double wb = 0.0, hb[6] = {0, 0, 0, 0, 0, 0}, Eb[3] = {0.0, 0.0, 0.0};
  if (sb) {   // H = sum w h h^T (packed upper triangle), B = sum w h (E/2)^T
    const double h[6] = {u0, u1, 1.0, sq, sq * sq, lam};
    for (int a = 0; a < 6; ++a)
      for (int c = a; c < 6; ++c) {
        const double cf = sb[tri6(a, c)];
        wb += cf * h[a] * h[c];
        hb[a] += cf * w * h[c];
        hb[c] += cf * w * h[a];
      }
    for (int a = 0; a < 6; ++a)
      for (int c = 0; c < 3; ++c) {
        const double cf = sb[21 + a * 3 + c];
        wb += cf * h[a] * 0.5 * E[c];
        hb[a] += cf * w * 0.5 * E[c];
        Eb[c] += cf * w * h[a] * 0.5;
      }
  }
  if (ab) {   // a = sum w lambda^2, b = sum -w lambda E / 2
    const double bE = ab[1] * E[0] + ab[2] * E[1] + ab[3] * E[2];
    wb += ab[0] * lam * lam - 0.5 * lam * bE;
    hb[5] += 2.0 * ab[0] * w * lam - 0.5 * w * bE;
    for (int c = 0; c < 3; ++c) Eb[c] += -0.5 * w * lam * ab[1 + c];
  }
  // w = rho'(|E|^2)
  const double rb = wb * rho_dd<LOSS>(L, r2);
  for (int c = 0; c < 3; ++c) Eb[c] += 2.0 * rb * E[c];
  // E = Rp - lambda q ; lambda = q . Rp / |q|^2
  const double lt = hb[5] - (Eb[0] * q[0] + Eb[1] * q[1] + Eb[2] * q[2]);
  double Rpb[3], qb[3];
  for (int c = 0; c < 3; ++c) {
    Rpb[c] = Eb[c] + lt * q[c] / qq;
    qb[c] = -lam * Eb[c] + lt * (Rp[c] - 2.0 * lam * q[c]) / qq;
  }
  // Rp = R p
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Rb[r * 3 + c] += Rpb[r] * p[c];
  double pb[3];
  for (int c = 0; c < 3; ++c) pb[c] = R[0 * 3 + c] * Rpb[0] + R[1 * 3 + c] * Rpb[1] + R[2 * 3 + c] * Rpb[2];
  db[0] += pb[2];
  db[1] += pb[2] * sq;
  db[2] += pb[2] * sq * sq;
  // u enters p (p_z through s) and h (u1, u2, s, s^2)
  const double sb_ = pb[2] * (d[1] + 2.0 * d[2] * sq) + hb[3] + 2.0 * sq * hb[4];
  ub[0] += pb[0] + hb[0] + 2.0 * u0 * sb_;
  ub[1] += pb[1] + hb[1] + 2.0 * u1 * sb_;
  // q = l - t
  for (int c = 0; c < 3; ++c) {
    lb[c] += qb[c];
    tb[c] -= qb[c];
  }
}

// 3. per observation: the statistics' adjoints pulled back to (camera, landmark, pixel) at the
//    point of each block's decision (x̄^k for an accelerated block, x^k after a restart). Camera
//    terms are summed per chunk (30 values: x̄ then x^k), landmark terms are stored at the
//    record position (lg_bar: x̄, lg_k: x^k), pixel terms added to g_u (input order).
template <int LOSS>
__global__ void __launch_bounds__(32)
    k_adj_obs(int n_chunks, const int* __restrict__ chunk_cam, const int* __restrict__ chunk_beg,
              const int* __restrict__ c_lm, const double2* __restrict__ c_u, const int* __restrict__ c_rpos,
              const int* __restrict__ ci_order, const V4<double>* __restrict__ pack,
              const V4<double>* __restrict__ lmrec, double gamma, const uint8_t* __restrict__ rs_cam,
              const uint8_t* __restrict__ rs_lm, int accelerated, LossC<double> L, double inv_s,
              const double* __restrict__ st_bar, const double* __restrict__ ab_bar, double* __restrict__ part,
              V4<double>* __restrict__ lg_bar, V4<double>* __restrict__ lg_k, double2* __restrict__ g_u) {
  const int warp = blockIdx.x;
  const int lane = threadIdx.x;
  if (warp >= n_chunks) return;
  const int cam = chunk_cam[warp];
  const int b = chunk_beg[warp], e = chunk_beg[warp + 1];
  const V4<double>* pk = pack + (size_t)cam * P4N;
  // the camera at x^k and at x̄^k from the pass pack (R̄ is the pack's; t̄, d̄ as the pass forms them)
  double Rpt[2][9], tpt[2][3], dpt[2][3];
  for (int r = 0; r < 3; ++r) {
    const V4<double> a = pk[P4_RK + r], bb = pk[P4_RB + r];
    Rpt[1][r * 3 + 0] = a.x, Rpt[1][r * 3 + 1] = a.y, Rpt[1][r * 3 + 2] = a.z;
    Rpt[0][r * 3 + 0] = bb.x, Rpt[0][r * 3 + 1] = bb.y, Rpt[0][r * 3 + 2] = bb.z;
    tpt[1][r] = a.w;
    tpt[0][r] = a.w + gamma * bb.w;
  }
  {
    const V4<double> dv = pk[P4_D], ddv = pk[P4_DD];
    dpt[1][0] = dv.x, dpt[1][1] = dv.y, dpt[1][2] = dv.z;
    dpt[0][0] = dv.x + gamma * ddv.x, dpt[0][1] = dv.y + gamma * ddv.y, dpt[0][2] = dv.z + gamma * ddv.z;
  }
  const int cam_pt = (!accelerated || rs_cam[cam]) ? 1 : 0;   // 0: x̄, 1: x^k
  double sb[39];
  for (int k = 0; k < 39; ++k) sb[k] = st_bar[(size_t)cam * 40 + k];
  double acc[30];
  for (int k = 0; k < 30; ++k) acc[k] = 0.0;
  const V4<double> zero4 = {0.0, 0.0, 0.0, 0.0};
  for (int o = b + lane; o < e; o += 32) {
    const int j = c_lm[o];
    const double2 uu = c_u[o];
    const V4<double> A = lmrec[2 * (size_t)j], B = lmrec[2 * (size_t)j + 1];
    const int lm_pt = (!accelerated || rs_lm[j]) ? 1 : 0;
    const int rp = c_rpos[o];
    double ub[2] = {0.0, 0.0};
    for (int pt = 0; pt < 2; ++pt) {
      const bool use_c = cam_pt == pt, use_l = lm_pt == pt;
      if (!use_c && !use_l) {
        (pt == 0 ? lg_bar : lg_k)[rp] = zero4;
        continue;
      }
      const double g = pt == 0 ? gamma : 0.0;
      const double l[3] = {A.x + g * A.w, A.y + g * B.x, A.z + g * B.y};
      double lb[3] = {0.0, 0.0, 0.0};
      double* ac = acc + pt * 15;
      obs_pullback<LOSS>(Rpt[pt], tpt[pt], dpt[pt], l, uu.x, uu.y, use_c ? sb : nullptr,
                         use_l ? ab_bar + (size_t)j * 4 : nullptr, L, ac + AC_R, ac + AC_T, ac + AC_D, lb, ub);
      V4<double> lv;
      lv.x = lb[0], lv.y = lb[1], lv.z = lb[2], lv.w = 0.0;
      (pt == 0 ? lg_bar : lg_k)[rp] = lv;
    }
    const size_t ui = (size_t)ci_order[o];
    double2 gu = g_u[ui];
    gu.x += ub[0] * inv_s;
    gu.y += ub[1] * inv_s;
    g_u[ui] = gu;
  }
  for (int k = 0; k < 30; ++k) {
    double v = acc[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    acc[k] = v;
  }
  if (lane == 0) {
    double* out = part + (size_t)warp * CP_STRIDE;
    for (int k = 0; k < 30; ++k) out[k] = acc[k];
  }
}

// 4. cameras: sum of the chunk terms, then the extrapolation x̄ = x^k + gamma (x^k - x^(k-1))
//    (R̄ through its polar factor) into the adjoints of x^k and x^(k-1).
__global__ void k_adj_cams_sum(int M, const int* __restrict__ cam_chunk_ptr, const double* __restrict__ part,
                               const double* __restrict__ sx, const double* __restrict__ sdx, double gamma,
                               const double* __restrict__ zb_bar, const double* __restrict__ zb_k,
                               double* __restrict__ a_k, double* __restrict__ a_km1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double zbar[15], zk[15];
  const double* zb0 = zb_bar + (size_t)i * AC_N;
  const double* zk0 = zb_k + (size_t)i * AC_N;
  for (int k = 0; k < 15; ++k) {
    zbar[k] = zb0[k];
    zk[k] = zk0[k];
  }
  for (int c = cam_chunk_ptr[i]; c < cam_chunk_ptr[i + 1]; ++c) {
    const double* p = part + (size_t)c * CP_STRIDE;
    for (int k = 0; k < 15; ++k) {
      zbar[k] += p[k];
      zk[k] += p[15 + k];
    }
  }
  CamT<double> ck, cb;
  load_cam(sx + (size_t)i * CSTRIDE, ck);
  double Kx[9], Kb[9];
  cam_bar(ck, sdx + (size_t)i * CSTRIDE, gamma, cb, Kx);
  polar_vjp(Kx, cb.R, zbar + AC_R, Kb);
  double* ak = a_k + (size_t)i * AC_N;
  double* am = a_km1 + (size_t)i * AC_N;
  for (int a = 0; a < 9; ++a) {
    ak[AC_R + a] += zk[AC_R + a] + (1.0 + gamma) * Kb[a];
    am[AC_R + a] += -gamma * Kb[a];
  }
  for (int k = 0; k < 3; ++k) {
    ak[AC_T + k] += zk[AC_T + k] + (1.0 + gamma) * zbar[AC_T + k];
    am[AC_T + k] += -gamma * zbar[AC_T + k];
    ak[AC_D + k] += zk[AC_D + k] + (1.0 + gamma) * zbar[AC_D + k];
    am[AC_D + k] += -gamma * zbar[AC_D + k];
  }
}

// 5. landmarks: sum of the observation terms (x̄ and x^k) plus the solve's, then the
//    extrapolation into the adjoints of l^k and l^(k-1).
__global__ void __launch_bounds__(LPASS_THREADS)
    k_adj_lms_sum(const int* __restrict__ tile_lm, const int* __restrict__ lm_ptr, const uint16_t* __restrict__ t_inv,
                  const V4<double>* __restrict__ lg_bar, const V4<double>* __restrict__ lg_k,
                  const double* __restrict__ zb_bar, const double* __restrict__ zb_k, double gamma,
                  double* __restrict__ a_k, double* __restrict__ a_km1) {
  const int lb = tile_lm[blockIdx.x], le = tile_lm[blockIdx.x + 1];
  const int jl = threadIdx.x;
  if (jl >= le - lb) return;
  const int j = lb + jl;
  const int ob = lm_ptr[lb];
  double gb[3] = {zb_bar[(size_t)j * AL_N + 0], zb_bar[(size_t)j * AL_N + 1], zb_bar[(size_t)j * AL_N + 2]};
  double gk[3] = {zb_k[(size_t)j * AL_N + 0], zb_k[(size_t)j * AL_N + 1], zb_k[(size_t)j * AL_N + 2]};
  for (int sl = lm_ptr[j]; sl < lm_ptr[j + 1]; ++sl) {
    const int rp = ob + t_inv[sl];
    const V4<double> x = lg_bar[rp], y = lg_k[rp];
    gb[0] += x.x, gb[1] += x.y, gb[2] += x.z;
    gk[0] += y.x, gk[1] += y.y, gk[2] += y.z;
  }
  double* ak = a_k + (size_t)j * AL_N;
  double* am = a_km1 + (size_t)j * AL_N;
  for (int c = 0; c < 3; ++c) {
    ak[c] += gk[c] + (1.0 + gamma) * gb[c];
    am[c] += -gamma * gb[c];
  }
}

// Seed: the adjoint of the boundary state after K iterations (cams M x 9, lms N x 3, external
// landmark order) as an adjoint of the internal state. Rotation: with w the axis-angle vector
// of R and dR = R [phi]x, dw = J_r(w)^-1 phi, so the tangent adjoint is g = J_r(w)^-T wbar and
// the ambient R [g]x / 2 carries it (vee(R^T G - G^T R) = g).
__global__ void k_adj_seed_cams(int M, const double* __restrict__ cam_x, const double* __restrict__ g_cams, double s,
                                double* __restrict__ a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double* x = cam_x + (size_t)i * CSTRIDE;
  const double* gc = g_cams + (size_t)i * 9;
  double R[9], w[3];
  for (int k = 0; k < 9; ++k) R[k] = x[CS_R + k];
  rot_log(R, w);
  // J_r^-1(w) = I + [w]x / 2 + (1/th^2 - (1 + cos th) / (2 th sin th)) [w]x^2
  const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const double th = sqrt(th2);
  const double c2 = th < 1e-6 ? 1.0 / 12.0 + th2 / 720.0 : 1.0 / th2 - (1.0 + cos(th)) / (2.0 * th * sin(th));
  const double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
  double Ji[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double k2 = 0.0;
      for (int m = 0; m < 3; ++m) k2 += K[r * 3 + m] * K[m * 3 + c];
      Ji[r * 3 + c] = (r == c ? 1.0 : 0.0) + 0.5 * K[r * 3 + c] + c2 * k2;
    }
  double g[3];
  for (int c = 0; c < 3; ++c) g[c] = Ji[0 * 3 + c] * gc[0] + Ji[1 * 3 + c] * gc[1] + Ji[2 * 3 + c] * gc[2];
  const double Gx[9] = {0.0, -g[2], g[1], g[2], 0.0, -g[0], -g[1], g[0], 0.0};
  double* o = a + (size_t)i * AC_N;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      o[AC_R + r * 3 + c] = 0.5 * (R[r * 3 + 0] * Gx[0 * 3 + c] + R[r * 3 + 1] * Gx[1 * 3 + c] + R[r * 3 + 2] * Gx[2 * 3 + c]);
  for (int k = 0; k < 3; ++k) o[AC_T + k] = gc[3 + k];
  // f = d1 s, k1 = d2 d1, k2 = d3 d1^3
  const double d1 = x[CS_D + 0], d2 = x[CS_D + 1], d3 = x[CS_D + 2];
  o[AC_D + 0] = s * gc[6] + d2 * gc[7] + 3.0 * d3 * d1 * d1 * gc[8];
  o[AC_D + 1] = d1 * gc[7];
  o[AC_D + 2] = d1 * d1 * d1 * gc[8];
}

__global__ void k_adj_seed_lms(int N, const double* __restrict__ g_lms, const int* __restrict__ linv,
                               double* __restrict__ a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double* o = a + (size_t)linv[j] * AL_N;
  o[0] = g_lms[(size_t)j * 3 + 0];
  o[1] = g_lms[(size_t)j * 3 + 1];
  o[2] = g_lms[(size_t)j * 3 + 2];
  o[3] = 0.0;
}

// Result: adjoint of x^0 (= x^(-1): both adjoints added) to the boundary parameters.
__global__ void k_adj_out_cams(int M, const double* __restrict__ cam_x, const double* __restrict__ a0,
                               const double* __restrict__ am, double s, double* __restrict__ g_cams) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double* x = cam_x + (size_t)i * CSTRIDE;
  double G[9], R[9], w[3], gw[3];
  for (int k = 0; k < 9; ++k) {
    G[k] = a0[(size_t)i * AC_N + AC_R + k] + am[(size_t)i * AC_N + AC_R + k];
    R[k] = x[CS_R + k];
  }
  double A[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) A[r * 3 + c] = R[0 * 3 + r] * G[0 * 3 + c] + R[1 * 3 + r] * G[1 * 3 + c] + R[2 * 3 + r] * G[2 * 3 + c];
  const double gphi[3] = {A[7] - A[5], A[2] - A[6], A[3] - A[1]};
  rot_log(R, w);
  right_jacobian_t(w, gphi, gw);
  double* o = g_cams + (size_t)i * 9;
  for (int k = 0; k < 3; ++k) {
    o[k] = gw[k];
    o[3 + k] = a0[(size_t)i * AC_N + AC_T + k] + am[(size_t)i * AC_N + AC_T + k];
  }
  const double gd[3] = {a0[(size_t)i * AC_N + AC_D + 0] + am[(size_t)i * AC_N + AC_D + 0],
                        a0[(size_t)i * AC_N + AC_D + 1] + am[(size_t)i * AC_N + AC_D + 1],
                        a0[(size_t)i * AC_N + AC_D + 2] + am[(size_t)i * AC_N + AC_D + 2]};
  const double d1 = x[CS_D + 0], d2 = x[CS_D + 1], d3 = x[CS_D + 2];
  const double f = d1 * s, k1 = d2 * f / s, k2 = d3 * f * f * f / (s * s * s);
  o[6] = gd[0] / s - gd[1] * k1 * s / (f * f) - 3.0 * gd[2] * k2 * s * s * s / (f * f * f * f);
  o[7] = gd[1] * s / f;
  o[8] = gd[2] * s * s * s / (f * f * f);
}

__global__ void k_adj_out_lms(int N, const double* __restrict__ a0, const double* __restrict__ am,
                              const int* __restrict__ lperm, double* __restrict__ g_lms) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  double* o = g_lms + (size_t)lperm[q] * 3;
  for (int c = 0; c < 3; ++c) o[c] = a0[(size_t)q * AL_N + c] + am[(size_t)q * AL_N + c];
}

}  // namespace daba
