// The landmark pass's work for one landmark (lpass_landmark, FP64: the code nvcc compiles into
// k_lpass) built for the host and driven from stdin, so that a test can compare it with the
// oracle's iteration: the sums of the landmark's records, Eqs. DEalpha, Fak and lFak in slack
// form, the accelerated update (Eq. update_amm), the restart test (Eq. Eak) and the MM update
// (Eq. update_mm).
// stdin: "n_lm first gamma xi eta accelerated", then per landmark "n l0 l1 l2 dl0 dl1 dl2 S E"
// and n lines "abar bbar0 bbar1 bbar2 ak bk0 bk1 bk2 F gap" (a, b of its terms Q_ij at the
// extrapolated iterate and at x^k, F_ij(x^k) and the surrogate gap, as the camera pass records
// them). stdout per landmark: l^(k+1) (3), l^(k+1) - l^k (3), the next slack S, E^(k+1),
// F^(k), Fbar^(k), restarted.
#include "../../paper_2305_07026_b300/csrc/daba_kernels.cuh"

#include <cstdio>
#include <vector>

using namespace daba;

int main() {
  int n_lm, first, accelerated;
  double gamma, xi, eta;
  if (std::scanf("%d %d %lf %lf %lf %d", &n_lm, &first, &gamma, &xi, &eta, &accelerated) != 6) return 1;
  IterParams P{};
  P.xi = xi, P.eta = eta, P.eta1 = 1.0 - eta, P.hxi = 0.5 * xi;
  P.accelerated = accelerated, P.restart_global = 0;
  for (int j = 0; j < n_lm; ++j) {
    int n;
    double v[8];
    if (std::scanf("%d", &n) != 1) return 1;
    for (double& x : v)
      if (std::scanf("%lf", &x) != 1) return 1;
    std::vector<V4<double>> sca(n), scb(n);
    std::vector<double2> cc(n);
    std::vector<uint16_t> inv(n);
    for (int q = 0; q < n; ++q) {
      double r[10];
      for (double& x : r)
        if (std::scanf("%lf", &x) != 1) return 1;
      sca[q] = {r[0], r[1], r[2], r[3]};
      scb[q] = {r[4], r[5], r[6], r[7]};
      cc[q] = RecC<double>::make(r[8], r[9]);
      inv[q] = (uint16_t)q;
    }
    const V4<double> A = {v[0], v[1], v[2], v[3]}, B = {v[4], v[5], v[6], v[7]};
    const V4<float> lo0 = {0.f, 0.f, 0.f, 0.f};
    V4<double> out[2];
    uint8_t rs = 0;
    double Fd = 0.0, Fbd = 0.0, gsum = 0.0;
    LpassOut<double> O;
    O.lmrec_out = out, O.lm_rs = &rs, O.lm_Fdiag = &Fd, O.lm_Fbdiag = &Fbd;
    const int r = lpass_landmark<double, false>(sca.data(), scb.data(), cc.data(), inv.data(), 0, n, A, B, lo0, 0,
                                                gamma, first, P, O, gsum);
    std::printf("%.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %d\n", out[0].x, out[0].y, out[0].z,
                out[0].w, out[1].x, out[1].y, out[1].z, out[1].w, Fd, Fbd, r);
  }
  return 0;
}
