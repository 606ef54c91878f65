// Central-difference checks of the library's device math, compiled for the host
// (tests/host/include holds the CUDA stand-ins). Each check compares a derivative the library
// computes with central differences of the matching forward function, and reports per group the
// largest error of a case divided by the largest finite-difference component of that case:
//   polar       the ProjRot3D pullback (K -> R = polar factor of K),
//   scam        the S-CAM camera solve's pullback to its statistics and conditioning point,
//   scam_tape   the taped forward solve against the plain one (must be the same bits),
//   obs_*       the per-observation pullback of the camera statistics and landmark terms, per loss,
//   boundary    the seed and result conversions between the boundary and internal cameras,
//   lm_gradient the gradient of the Levenberg-Marquardt camera model against the surrogate E^alpha,
//   lm_hessian  its Gauss-Newton matrix against the surrogate's Hessian where they coincide (zero
//               residual statistics), and lm_no_decrease the count of LM steps that failed to
//               lower the surrogate (reported in the error column).
#include "../../paper_2305_07026_b300/csrc/daba_adjoint.cuh"

#include <cstdio>
#include <random>
#include <vector>

using namespace daba;

namespace {

std::mt19937_64 rng(7);
double U(double a = -1, double b = 1) { return std::uniform_real_distribution<double>(a, b)(rng); }

struct Group {
  const char* name;
  double worst = 0.0;
  int cases = 0;
  // one case: analytic and finite-difference values of the same directional derivatives
  void add(const std::vector<double>& an, const std::vector<double>& fd) {
    double scale = 1e-12, err = 0.0;
    for (size_t k = 0; k < fd.size(); ++k) scale = std::max(scale, std::fabs(fd[k]));
    for (size_t k = 0; k < fd.size(); ++k) err = std::max(err, std::fabs(an[k] - fd[k]));
    worst = std::max(worst, err / scale);
    ++cases;
  }
  void print() const { std::printf("%s %.3e %d\n", name, worst, cases); }
};

void matmul3(const double* A, const double* B, double* C) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int m = 0; m < 3; ++m) s += A[r * 3 + m] * B[m * 3 + c];
      C[r * 3 + c] = s;
    }
}

// skew matrix [e_a]x of the unit vector e_a
void skew_unit(int a, double* P) {
  for (int k = 0; k < 9; ++k) P[k] = 0.0;
  if (a == 0) P[7] = 1, P[5] = -1;
  if (a == 1) P[2] = 1, P[6] = -1;
  if (a == 2) P[3] = 1, P[1] = -1;
}

void check_polar(Group& g) {
  for (int rep = 0; rep < 20; ++rep) {
    double w[3] = {U(), U(), U()}, Q[9], S[9], K[9], R[9], Rb[9], Kb[9];
    rodrigues(w, Q);
    for (int a = 0; a < 9; ++a) S[a] = 0.3 * U();
    for (int a = 0; a < 3; ++a) S[a * 4] += 2.0;
    matmul3(Q, S, K);
    proj_rot3d_polar(K, R);
    for (int a = 0; a < 9; ++a) Rb[a] = U();
    polar_vjp(K, R, Rb, Kb);
    std::vector<double> an(9), fd(9);
    for (int a = 0; a < 9; ++a) {
      const double h = 1e-6;
      double Kp[9], Km[9], Rp[9], Rm[9];
      for (int b = 0; b < 9; ++b) Kp[b] = Km[b] = K[b];
      Kp[a] += h, Km[a] -= h;
      proj_rot3d_polar(Kp, Rp);
      proj_rot3d_polar(Km, Rm);
      double f = 0;
      for (int b = 0; b < 9; ++b) f += Rb[b] * (Rp[b] - Rm[b]) / (2 * h);
      an[a] = Kb[a], fd[a] = f;
    }
    g.add(an, fd);
  }
}

// camera statistics of n synthetic observations, the layout the camera pass accumulates
void make_stats(double* st, int n) {
  for (int k = 0; k < 39; ++k) st[k] = 0.0;
  for (int o = 0; o < n; ++o) {
    const double u0 = U(-0.5, 0.5), u1 = U(-0.5, 0.5), s = u0 * u0 + u1 * u1, lam = U(2, 6), w = U(0.2, 1.0);
    const double h[6] = {u0, u1, 1.0, s, s * s, lam};
    const double r0[3] = {0.05 * U(), 0.05 * U(), 0.05 * U()};
    for (int a = 0; a < 6; ++a)
      for (int c = a; c < 6; ++c) st[tri6(a, c)] += w * h[a] * h[c];
    for (int a = 0; a < 6; ++a)
      for (int c = 0; c < 3; ++c) st[21 + a * 3 + c] += w * h[a] * r0[c];
  }
}

double scam_L(const double* st, const CamT<double>& z, double xi, int n_alt, const CamT<double>& cb) {
  CamT<double> c;
  cam_scam<double>(st, z, xi, n_alt, c);
  double f = 0;
  for (int a = 0; a < 9; ++a) f += cb.R[a] * c.R[a];
  for (int k = 0; k < 3; ++k) f += cb.t[k] * c.t[k] + cb.d[k] * c.d[k];
  return f;
}

void check_scam(Group& g, Group& tape) {
  for (int rep = 0; rep < 12; ++rep) {
    double st[39];
    make_stats(st, 40 + rep * 10);
    const double xi = rep % 3 == 0 ? 1e-4 : 0.5;
    const int n_alt = 1 + rep % 3;
    CamT<double> z, cb, zb, c1, c2;
    double w[3] = {U(), U(), U()};
    rodrigues(w, z.R);
    for (int k = 0; k < 3; ++k) z.t[k] = U();
    z.d[0] = 1.0 + 0.1 * U(), z.d[1] = 0.1 * U(), z.d[2] = 0.05 * U();
    for (int a = 0; a < 9; ++a) cb.R[a] = U();
    for (int k = 0; k < 3; ++k) cb.t[k] = U(), cb.d[k] = U();
    // the taped forward solve is the plain one
    ScamTape tp[4];
    scam_tape(st, z, xi, n_alt, c2, tp);
    cam_scam<double>(st, z, xi, n_alt, c1);
    std::vector<double> a1, a2;
    for (int a = 0; a < 9; ++a) a1.push_back(c1.R[a]), a2.push_back(c2.R[a]);
    for (int k = 0; k < 3; ++k) a1.push_back(c1.t[k]), a2.push_back(c2.t[k]), a1.push_back(c1.d[k]), a2.push_back(c2.d[k]);
    tape.add(a2, a1);
    double Hb[6][6], Bb[6][3];
    scam_adjoint(st, z, xi, n_alt, tp, cb, Hb, Bb, zb);
    double sb[39];
    for (int a = 0; a < 6; ++a)
      for (int b = a; b < 6; ++b) sb[tri6(a, b)] = a == b ? Hb[a][a] : Hb[a][b] + Hb[b][a];
    for (int a = 0; a < 6; ++a)
      for (int c = 0; c < 3; ++c) sb[21 + a * 3 + c] = Bb[a][c];
    std::vector<double> an, fd;
    for (int k = 0; k < 39; ++k) {
      const double h = 1e-6 * std::max(1.0, std::fabs(st[k]));
      double sp[39], sm[39];
      for (int q = 0; q < 39; ++q) sp[q] = sm[q] = st[q];
      sp[k] += h, sm[k] -= h;
      an.push_back(sb[k]);
      fd.push_back((scam_L(sp, z, xi, n_alt, cb) - scam_L(sm, z, xi, n_alt, cb)) / (2 * h));
    }
    g.add(an, fd);
    an.clear(), fd.clear();
    const double h = 1e-6;
    // z.R along the tangent directions z.R Exp(h e_a): every conditioning rotation is a rotation
    for (int a = 0; a < 3; ++a) {
      double ph[3] = {0, 0, 0}, mh[3] = {0, 0, 0}, Ep[9], Em[9], P[9], dR[9];
      ph[a] = h, mh[a] = -h;
      rodrigues(ph, Ep), rodrigues(mh, Em);
      CamT<double> zp = z, zm = z;
      matmul3(z.R, Ep, zp.R), matmul3(z.R, Em, zm.R);
      skew_unit(a, P);
      matmul3(z.R, P, dR);
      double d = 0;
      for (int q = 0; q < 9; ++q) d += zb.R[q] * dR[q];
      an.push_back(d);
      fd.push_back((scam_L(st, zp, xi, n_alt, cb) - scam_L(st, zm, xi, n_alt, cb)) / (2 * h));
    }
    for (int a = 0; a < 6; ++a) {
      CamT<double> zp = z, zm = z;
      double* vp = a < 3 ? &zp.t[a] : &zp.d[a - 3];
      double* vm = a < 3 ? &zm.t[a] : &zm.d[a - 3];
      *vp += h, *vm -= h;
      an.push_back(a < 3 ? zb.t[a] : zb.d[a - 3]);
      fd.push_back((scam_L(st, zp, xi, n_alt, cb) - scam_L(st, zm, xi, n_alt, cb)) / (2 * h));
    }
    g.add(an, fd);
  }
}

// <sb, camera statistics> + <ab, landmark terms> of one observation, by the pass's own evaluation
template <int LOSS>
double obs_L(const double* R, const double* t, const double* d, const double* l, double u0, double u1,
             const double* sb, const double* ab, const LossC<double>& L) {
  V4<double> pk[P4N];
  for (int r = 0; r < 3; ++r) {
    pk[P4_RK + r] = {R[r * 3], R[r * 3 + 1], R[r * 3 + 2], t[r]};
    pk[P4_RB + r] = {R[r * 3], R[r * 3 + 1], R[r * 3 + 2], 0.0};
    pk[P4_DR + r] = {0.0, 0.0, 0.0, 0.0};
  }
  pk[P4_D] = {d[0], d[1], d[2], 0.0};
  pk[P4_DD] = {0.0, 0.0, 0.0, 0.0};
  ObsEval<double> ev;
  eval_obs<LOSS, double>(pk, l[0], l[1], l[2], 0.0, 0.0, 0.0, u0, u1, 0.0, L, ev);
  double acc[80] = {0};
  accumulate_cam<double>(acc, ev, u0, u1);
  double f = 0;
  for (int k = 0; k < 21; ++k) f += sb[k] * acc[CP_H + k];
  for (int k = 0; k < 18; ++k) f += sb[21 + k] * acc[CP_B + k];
  const double wl = ev.w * ev.lam;
  f += ab[0] * wl * ev.lam + ab[1] * (-0.5 * wl * ev.Re0) + ab[2] * (-0.5 * wl * ev.Re1) + ab[3] * (-0.5 * wl * ev.Re2);
  return f;
}

template <int LOSS>
void check_obs(Group& g) {
  LossC<double> L;
  L.c = 0.02, L.c2 = L.c * L.c, L.inv_c2 = 1.0 / L.c2;
  for (int rep = 0; rep < 30; ++rep) {
    double w[3] = {U(), U(), U()}, R[9], t[3], d[3], l[3], u0 = U(-0.5, 0.5), u1 = U(-0.5, 0.5);
    rodrigues(w, R);
    for (int a = 0; a < 9; ++a) R[a] += 1e-2 * U();   // conditioning matrices need not be rotations here
    for (int k = 0; k < 3; ++k) t[k] = U();
    d[0] = 1.0 + 0.1 * U(), d[1] = 0.1 * U(), d[2] = 0.05 * U();
    // a landmark in front along the ray, displaced so that |E| falls on both sides of the loss scale
    const double s = u0 * u0 + u1 * u1, p[3] = {u0, u1, d[0] + d[1] * s + d[2] * s * s};
    const double lamt = U(2, 6), sc = rep % 2 ? 0.005 : 0.05;
    for (int r = 0; r < 3; ++r) l[r] = t[r] + (R[r * 3] * p[0] + R[r * 3 + 1] * p[1] + R[r * 3 + 2] * p[2]) / lamt + sc * U();
    double sb[39], ab[4];
    for (int k = 0; k < 39; ++k) sb[k] = U();
    for (int k = 0; k < 4; ++k) ab[k] = U();
    double Rb[9] = {0}, tb[3] = {0}, db[3] = {0}, lb[3] = {0}, ub[2] = {0};
    obs_pullback<LOSS>(R, t, d, l, u0, u1, sb, ab, L, Rb, tb, db, lb, ub);
    const double h = 1e-7;
    auto fd1 = [&](double* v) {
      const double o = *v;
      *v = o + h;
      const double fp = obs_L<LOSS>(R, t, d, l, u0, u1, sb, ab, L);
      *v = o - h;
      const double fm = obs_L<LOSS>(R, t, d, l, u0, u1, sb, ab, L);
      *v = o;
      return (fp - fm) / (2 * h);
    };
    std::vector<double> an, fd;
    for (int a = 0; a < 9; ++a) an.push_back(Rb[a]), fd.push_back(fd1(&R[a]));
    for (int k = 0; k < 3; ++k) {
      an.push_back(tb[k]), fd.push_back(fd1(&t[k]));
      an.push_back(db[k]), fd.push_back(fd1(&d[k]));
      an.push_back(lb[k]), fd.push_back(fd1(&l[k]));
    }
    an.push_back(ub[0]), fd.push_back(fd1(&u0));
    an.push_back(ub[1]), fd.push_back(fd1(&u1));
    g.add(an, fd);
  }
}

void check_boundary(Group& g) {
  const double s = 700.0;
  for (int rep = 0; rep < 10; ++rep) {
    double x[CSTRIDE] = {0}, w[3] = {U(), U(), U()}, gcam[9], a[AC_N] = {0};
    rodrigues(w, x + CS_R);
    x[CS_D + 0] = 1.0 + 0.1 * U(), x[CS_D + 1] = 0.1 * U(), x[CS_D + 2] = 0.05 * U();
    for (int k = 0; k < 9; ++k) gcam[k] = U();
    threadIdx.x = blockIdx.x = 0, blockDim.x = 1;
    k_adj_seed_cams(1, x, gcam, s, a);
    // the boundary camera [w, t, f, k1, k2] of an internal (R, d), translation left out
    auto bnd = [&](const double* R, const double* d, double* out) {
      rot_log(R, out);
      const double f = d[0] * s;
      out[3] = out[4] = out[5] = 0.0;
      out[6] = f, out[7] = d[1] * f / s, out[8] = d[2] * f * f * f / (s * s * s);
    };
    std::vector<double> an, fd;
    for (int dir = 0; dir < 6; ++dir) {
      const double h = 1e-6;
      double phi[3] = {0, 0, 0}, dd[3] = {0, 0, 0};
      if (dir < 3) phi[dir] = 1.0; else dd[dir - 3] = 1.0;
      double op[9], om[9], Rp[9], Rm[9], Ep[9], Em[9], dp[3], dm[3];
      double pp[3] = {h * phi[0], h * phi[1], h * phi[2]}, pm[3] = {-h * phi[0], -h * phi[1], -h * phi[2]};
      rodrigues(pp, Ep), rodrigues(pm, Em);
      matmul3(x + CS_R, Ep, Rp), matmul3(x + CS_R, Em, Rm);
      for (int k = 0; k < 3; ++k) dp[k] = x[CS_D + k] + h * dd[k], dm[k] = x[CS_D + k] - h * dd[k];
      bnd(Rp, dp, op), bnd(Rm, dm, om);
      double f = 0;
      for (int k = 0; k < 9; ++k) f += gcam[k] * (op[k] - om[k]) / (2 * h);
      const double P[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
      double dR[9], v = 0;
      matmul3(x + CS_R, P, dR);
      for (int q = 0; q < 9; ++q) v += a[AC_R + q] * dR[q];
      for (int k = 0; k < 3; ++k) v += a[AC_D + k] * dd[k];
      an.push_back(v), fd.push_back(f);
    }
    g.add(an, fd);
    // result conversion: ambient adjoints on R = Exp(w) and d -> gradient on [w, f, k1, k2]
    double a0[AC_N] = {0}, am[AC_N] = {0}, go[9], wb[3];
    for (int k = 0; k < 15; ++k) a0[k] = U(), am[k] = U();
    k_adj_out_cams(1, x, a0, am, s, go);
    rot_log(x + CS_R, wb);
    const double f0 = x[CS_D] * s, k10 = x[CS_D + 1] * f0 / s, k20 = x[CS_D + 2] * f0 * f0 * f0 / (s * s * s);
    auto val = [&](const double* bw, double f, double k1, double k2) {
      double R[9];
      rodrigues(bw, R);
      const double d[3] = {f / s, k1 * s / f, k2 * s * s * s / (f * f * f)};
      double v = 0;
      for (int k = 0; k < 9; ++k) v += (a0[AC_R + k] + am[AC_R + k]) * R[k];
      for (int k = 0; k < 3; ++k) v += (a0[AC_D + k] + am[AC_D + k]) * d[k];
      return v;
    };
    an.clear(), fd.clear();
    for (int k = 0; k < 3; ++k) {
      const double h = 1e-6;
      double wp[3] = {wb[0], wb[1], wb[2]}, wm[3] = {wb[0], wb[1], wb[2]};
      wp[k] += h, wm[k] -= h;
      an.push_back(go[k]), fd.push_back((val(wp, f0, k10, k20) - val(wm, f0, k10, k20)) / (2 * h));
    }
    const double hf = 1e-4, hk = 1e-7;
    an.push_back(go[6]), fd.push_back((val(wb, f0 + hf, k10, k20) - val(wb, f0 - hf, k10, k20)) / (2 * hf));
    an.push_back(go[7]), fd.push_back((val(wb, f0, k10 + hk, k20) - val(wb, f0, k10 - hk, k20)) / (2 * hk));
    an.push_back(go[8]), fd.push_back((val(wb, f0, k10, k20 + hk) - val(wb, f0, k10, k20 - hk)) / (2 * hk));
    g.add(an, fd);
  }
}

// the camera z Exp(theta[0:3]), t + theta[3:6], d + theta[6:9]
void cam_at(const CamT<double>& z, const double* th, CamT<double>& c) {
  double E[9];
  rodrigues(th, E);
  matmul3(z.R, E, c.R);
  for (int k = 0; k < 3; ++k) c.t[k] = z.t[k] + th[3 + k], c.d[k] = z.d[k] + th[6 + k];
}

void make_stats_b(double* st, int n, double bscale) {
  for (int k = 0; k < 39; ++k) st[k] = 0.0;
  for (int o = 0; o < n; ++o) {
    const double u0 = U(-0.5, 0.5), u1 = U(-0.5, 0.5), s = u0 * u0 + u1 * u1, lam = U(2, 6), w = U(0.2, 1.0);
    const double h[6] = {u0, u1, 1.0, s, s * s, lam};
    const double r0[3] = {bscale * U(), bscale * U(), bscale * U()};
    for (int a = 0; a < 6; ++a)
      for (int c = a; c < 6; ++c) st[tri6(a, c)] += w * h[a] * h[c];
    for (int a = 0; a < 6; ++a)
      for (int c = 0; c < 3; ++c) st[21 + a * 3 + c] += w * h[a] * r0[c];
  }
}

void check_lm(Group& grad, Group& hess, Group& fails) {
  int no_decrease = 0;
  for (int rep = 0; rep < 20; ++rep) {
    double st[39];
    const bool zero_b = rep % 2 == 0;
    make_stats_b(st, 60, zero_b ? 0.0 : 0.05);
    CamT<double> z;
    double w[3] = {U(), U(), U()};
    rodrigues(w, z.R);
    for (int k = 0; k < 3; ++k) z.t[k] = U();
    z.d[0] = 1.0 + 0.1 * U(), z.d[1] = 0.1 * U(), z.d[2] = 0.05 * U();
    const double xi = 1e-3;
    double A[45], g[9];
    cam_lm_model(st, z, xi, A, g);
    auto E = [&](const double* th) {
      CamT<double> c;
      cam_at(z, th, c);
      return cam_phi(st, z, c, xi);
    };
    if (!zero_b) {
      const double h = 1e-6;
      std::vector<double> an, fd;
      for (int i = 0; i < 9; ++i) {
        double tp[9] = {0}, tm[9] = {0};
        tp[i] = h, tm[i] = -h;
        an.push_back(g[i]), fd.push_back((E(tp) - E(tm)) / (2 * h));
      }
      grad.add(an, fd);
      CamT<double> c;
      cam_lm(st, z, xi, c);
      if (!(cam_phi(st, z, c, xi) < 0)) ++no_decrease;
    } else {
      const double hh = 1e-4;
      std::vector<double> an, fd;
      for (int i = 0; i < 9; ++i)
        for (int j = 0; j <= i; ++j) {
          double a[9] = {0}, b[9] = {0}, c[9] = {0}, d[9] = {0};
          a[i] += hh, a[j] += hh, b[i] += hh, b[j] -= hh, c[i] -= hh, c[j] += hh, d[i] -= hh, d[j] -= hh;
          an.push_back(A[lt9(i, j)]), fd.push_back((E(a) - E(b) - E(c) + E(d)) / (4 * hh * hh));
        }
      hess.add(an, fd);
    }
  }
  fails.worst = no_decrease;
  fails.cases = 10;
}

// <cb, c> for the camera c of one LM step (cam_lm) from c_z
double lm_L(const double* st, const CamT<double>& z, double xi, const CamT<double>& cb) {
  CamT<double> c;
  cam_lm(st, z, xi, c);
  double f = 0;
  for (int a = 0; a < 9; ++a) f += cb.R[a] * c.R[a];
  for (int k = 0; k < 3; ++k) f += cb.t[k] * c.t[k] + cb.d[k] * c.d[k];
  return f;
}

// the reverse sweep of the LM step (lm_adjoint) against central differences of lm_L in the 39
// statistics, the tangent directions of z.R and z.t, z.d; taken counts the cases with a step
void check_lm_adjoint(Group& g, Group& taken) {
  int steps = 0;
  for (int rep = 0; rep < 16; ++rep) {
    double st[39];
    make_stats_b(st, 40 + rep * 5, 0.02 + 0.02 * (rep % 4));
    const double xi = rep % 2 ? 1e-3 : 0.2;
    CamT<double> z, cb, zb, c;
    double w[3] = {U(), U(), U()};
    rodrigues(w, z.R);
    for (int k = 0; k < 3; ++k) z.t[k] = U();
    z.d[0] = 1.0 + 0.1 * U(), z.d[1] = 0.1 * U(), z.d[2] = 0.05 * U();
    for (int a = 0; a < 9; ++a) cb.R[a] = U();
    for (int k = 0; k < 3; ++k) cb.t[k] = U(), cb.d[k] = U();
    cam_lm(st, z, xi, c);
    if (c.t[0] != z.t[0]) ++steps;
    double Hb[6][6], Bb[6][3];
    lm_adjoint(st, z, xi, cb, Hb, Bb, zb);
    double sb[39];
    for (int a = 0; a < 6; ++a)
      for (int b = a; b < 6; ++b) sb[tri6(a, b)] = a == b ? Hb[a][a] : Hb[a][b] + Hb[b][a];
    for (int a = 0; a < 6; ++a)
      for (int cc = 0; cc < 3; ++cc) sb[21 + a * 3 + cc] = Bb[a][cc];
    std::vector<double> an, fd;
    for (int k = 0; k < 39; ++k) {
      const double h = 1e-6 * std::max(1.0, std::fabs(st[k]));
      double sp[39], sm[39];
      for (int q = 0; q < 39; ++q) sp[q] = sm[q] = st[q];
      sp[k] += h, sm[k] -= h;
      an.push_back(sb[k]);
      fd.push_back((lm_L(sp, z, xi, cb) - lm_L(sm, z, xi, cb)) / (2 * h));
    }
    const double h = 1e-6;
    for (int a = 0; a < 3; ++a) {   // z.R along z.R Exp(h e_a)
      double ph[3] = {0, 0, 0}, mh[3] = {0, 0, 0}, Ep[9], Em[9], P[9], dR[9];
      ph[a] = h, mh[a] = -h;
      rodrigues(ph, Ep), rodrigues(mh, Em);
      CamT<double> zp = z, zm = z;
      matmul3(z.R, Ep, zp.R), matmul3(z.R, Em, zm.R);
      skew_unit(a, P);
      matmul3(z.R, P, dR);
      double d = 0;
      for (int q = 0; q < 9; ++q) d += zb.R[q] * dR[q];
      an.push_back(d);
      fd.push_back((lm_L(st, zp, xi, cb) - lm_L(st, zm, xi, cb)) / (2 * h));
    }
    for (int a = 0; a < 6; ++a) {
      CamT<double> zp = z, zm = z;
      double* vp = a < 3 ? &zp.t[a] : &zp.d[a - 3];
      double* vm = a < 3 ? &zm.t[a] : &zm.d[a - 3];
      *vp += h, *vm -= h;
      an.push_back(a < 3 ? zb.t[a] : zb.d[a - 3]);
      fd.push_back((lm_L(st, zp, xi, cb) - lm_L(st, zm, xi, cb)) / (2 * h));
    }
    g.add(an, fd);
  }
  taken.worst = -steps;   // reported negated: the test wants most cases to have taken a step
  taken.cases = 16;
}

}  // namespace

int main() {
  Group polar{"polar"}, scam{"scam"}, tape{"scam_tape"}, triv{"obs_trivial"}, hub{"obs_huber"}, cau{"obs_cauchy"},
      wel{"obs_welsch"}, bnd{"boundary"};
  check_polar(polar);
  check_scam(scam, tape);
  check_obs<LOSS_TRIVIAL>(triv);
  check_obs<LOSS_HUBER>(hub);
  check_obs<LOSS_CAUCHY>(cau);
  check_obs<LOSS_WELSCH>(wel);
  check_boundary(bnd);
  Group lmg{"lm_gradient"}, lmh{"lm_hessian"}, lmf{"lm_no_decrease"};
  check_lm(lmg, lmh, lmf);
  Group lma{"lm_adjoint"}, lms{"lm_adjoint_steps"};
  check_lm_adjoint(lma, lms);
  for (const Group* g : {&polar, &scam, &tape, &triv, &hub, &cau, &wel, &bnd, &lmg, &lmh, &lmf, &lma, &lms}) g->print();
  return 0;
}
