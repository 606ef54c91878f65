// The library's camera block solves (FP64) built for the host and driven from stdin, so that a
// test can compare them with the oracle: the camera pass's statistics of one camera's
// observations at x^k (eval_obs + accumulate_cam), then the S-CAM solve (cam_scam), its
// surrogate decrease (cam_phi) and the Levenberg-Marquardt step (cam_lm), all from z = x^k.
// stdin: "loss c xi n_alt m", then R (9, row-major) t (3) d (3) of the camera, then m lines of
// l (3) u (2). stdout: S-CAM R t d and its decrease (16 numbers), then LM R t d and its decrease.
#include "../../paper_2305_07026_b300/csrc/daba_kernels.cuh"

#include <cstdio>
#include <vector>

using namespace daba;

template <int LOSS>
void stats(const LossC<double>& L, const CamT<double>& z, int m, double* st) {
  V4<double> pk[P4N];
  for (int r = 0; r < 3; ++r) {
    pk[P4_RK + r] = {z.R[3 * r], z.R[3 * r + 1], z.R[3 * r + 2], z.t[r]};
    pk[P4_RB + r] = {z.R[3 * r], z.R[3 * r + 1], z.R[3 * r + 2], 0.0};
    pk[P4_DR + r] = {0.0, 0.0, 0.0, 0.0};
  }
  pk[P4_D] = {z.d[0], z.d[1], z.d[2], 0.0};
  pk[P4_DD] = {0.0, 0.0, 0.0, 0.0};
  double acc[CP_NACC] = {0};
  for (int o = 0; o < m; ++o) {
    double v[5];
    for (double& x : v)
      if (std::scanf("%lf", &x) != 1) return;
    ObsEval<double> ev;
    eval_obs<LOSS, double>(pk, v[0], v[1], v[2], 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, v[3], v[4], 0.0, L, ev);
    accumulate_cam<double>(acc, ev, v[3], v[4]);
  }
  for (int k = 0; k < 39; ++k) st[k] = acc[CP_H + k];   // H (21) then B (18) at x^k
}

void print(const CamT<double>& c, double dec) {
  for (double v : c.R) std::printf("%.17g ", v);
  for (double v : c.t) std::printf("%.17g ", v);
  for (double v : c.d) std::printf("%.17g ", v);
  std::printf("%.17g\n", dec);
}

int main() {
  int loss = 0, n_alt = 2, m = 0;
  double c = 1.0, xi = 1e-10;
  if (std::scanf("%d %lf %lf %d %d", &loss, &c, &xi, &n_alt, &m) != 5) return 1;
  CamT<double> z;
  double* zv[15];
  for (int k = 0; k < 9; ++k) zv[k] = &z.R[k];
  for (int k = 0; k < 3; ++k) zv[9 + k] = &z.t[k], zv[12 + k] = &z.d[k];
  for (double* v : zv)
    if (std::scanf("%lf", v) != 1) return 1;
  LossC<double> L;
  L.c = c, L.c2 = c * c, L.inv_c2 = 1.0 / (c * c);
  double st[39];
  if (loss == LOSS_TRIVIAL) stats<LOSS_TRIVIAL>(L, z, m, st);
  if (loss == LOSS_HUBER) stats<LOSS_HUBER>(L, z, m, st);
  if (loss == LOSS_CAUCHY) stats<LOSS_CAUCHY>(L, z, m, st);
  if (loss == LOSS_WELSCH) stats<LOSS_WELSCH>(L, z, m, st);
  CamT<double> cs, cl;
  cam_scam<double>(st, z, xi, n_alt, cs);
  print(cs, cam_phi(st, z, cs, xi));
  cam_lm(st, z, xi, cl);
  print(cl, cam_phi(st, z, cl, xi));
  return 0;
}
