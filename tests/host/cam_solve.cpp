// The library's camera block solves built for the host and driven from stdin, so that a test can
// compare them with the oracle: the camera pass's statistics of one camera's observations at x^k
// (eval_obs + accumulate_cam), then the S-CAM solve, its surrogate decrease (cam_phi) and the
// Levenberg-Marquardt step (cam_lm), all from z = x^k. With bits = 64 everything is FP64; with
// bits = 32 the statistics are evaluated and accumulated in FP32 (one chunk, widened to FP64 as
// the camera solve sums chunks) and the S-CAM solve is the MIXED path's FP32 one (cam_solve<.., float>).
// stdin: "bits loss c xi n_alt m", then R (9, row-major) t (3) d (3) of the camera, then m lines of
// l (3) u (2). stdout: S-CAM R t d and its decrease (16 numbers), then LM R t d and its decrease.
#include "../../paper_2305_07026_b300/csrc/daba_kernels.cuh"

#include <cstdio>
#include <vector>

using namespace daba;

template <int LOSS, class Real>
void stats(double c, const CamT<double>& z, int m, double* st) {
  LossC<Real> L;
  L.c = Real(c), L.c2 = Real(c * c), L.inv_c2 = Real(1.0 / (c * c));
  CamT<double> dz;
  for (double& v : dz.R) v = 0.0;
  for (int k = 0; k < 3; ++k) dz.t[k] = dz.d[k] = 0.0;
  V4<Real> pk[P4N];
  write_pack_t<Real>(z, dz, z.R, pk);
  Real acc[CP_NACC];
  for (Real& a : acc) a = Real(0);
  for (int o = 0; o < m; ++o) {
    double v[5];
    for (double& x : v)
      if (std::scanf("%lf", &x) != 1) return;
    Real l[3], lo[3];
    for (int a = 0; a < 3; ++a) split_real(v[a], l[a], lo[a]);
    const Real u0 = to_real<Real>(v[3]), u1 = to_real<Real>(v[4]);
    ObsEval<Real> ev;
    eval_obs<LOSS, Real>(pk, l[0], l[1], l[2], Real(0), Real(0), Real(0), u0, u1, Real(0), L,
                         ev);
    accumulate_cam<Real>(acc, ev, u0, u1);
  }
  for (int k = 0; k < 39; ++k) st[k] = double(acc[CP_H + k]);   // H (21) then B (18) at x^k
}

template <class Real>
void statistics(int loss, double c, const CamT<double>& z, int m, double* st) {
  if (loss == LOSS_TRIVIAL) stats<LOSS_TRIVIAL, Real>(c, z, m, st);
  if (loss == LOSS_HUBER) stats<LOSS_HUBER, Real>(c, z, m, st);
  if (loss == LOSS_CAUCHY) stats<LOSS_CAUCHY, Real>(c, z, m, st);
  if (loss == LOSS_WELSCH) stats<LOSS_WELSCH, Real>(c, z, m, st);
}

void print(const CamT<double>& c, double dec) {
  for (double v : c.R) std::printf("%.17g ", v);
  for (double v : c.t) std::printf("%.17g ", v);
  for (double v : c.d) std::printf("%.17g ", v);
  std::printf("%.17g\n", dec);
}

int main() {
  int bits = 64, loss = 0, n_alt = 2, m = 0;
  double c = 1.0, xi = 1e-10;
  if (std::scanf("%d %d %lf %lf %d %d", &bits, &loss, &c, &xi, &n_alt, &m) != 6) return 1;
  CamT<double> z;
  double* zv[15];
  for (int k = 0; k < 9; ++k) zv[k] = &z.R[k];
  for (int k = 0; k < 3; ++k) zv[9 + k] = &z.t[k], zv[12 + k] = &z.d[k];
  for (double* v : zv)
    if (std::scanf("%lf", v) != 1) return 1;
  double st[39];
  CamT<double> cs, cl;
  if (bits == 32) {
    statistics<float>(loss, c, z, m, st);
    cam_solve<CAM_SCAM, float>(st, z, xi, n_alt, cs);
  } else {
    statistics<double>(loss, c, z, m, st);
    cam_solve<CAM_SCAM, double>(st, z, xi, n_alt, cs);
  }
  print(cs, cam_phi(st, z, cs, xi));
  cam_lm(st, z, xi, cl);
  print(cl, cam_phi(st, z, cl, xi));
  return 0;
}
