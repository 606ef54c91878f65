// The landmark pass's work for one landmark (lpass_landmark, FP64: the code nvcc compiles into
// k_lpass) built for the host and driven from stdin, so that a test can compare it with the
// oracle's iteration: the sums of the landmark's records, Eqs. DEalpha, Fak and lFak in slack
// form, the accelerated update (Eq. update_amm), the restart test (Eq. Eak) and the MM update
// (Eq. update_mm).
// With global = 1 the global restart variant runs (no per-block test; the MM alternative's step
// and slack, and E after a restart, kept in lm_alt; the landmark's E^(k+1) - Fbar^(k) returned).
// stdin: "bits global n_lm first gamma xi eta accelerated", then per landmark "n l0 l1 l2 dl0 dl1 dl2 S E"
// and n lines "abar bbar0 bbar1 bbar2 ak bk0 bk1 bk2 F gap" (a, b of its terms Q_ij at the
// extrapolated iterate and at x^k, F_ij(x^k) and the surrogate gap, as the camera pass records
// them). stdout per landmark: l^(k+1) (3), l^(k+1) - l^k (3), the next slack S, E^(k+1),
// F^(k), Fbar^(k), restarted. With bits = 32 the MIXED instantiation runs: records, slack and
// step in FP32, the landmark as an FP32 high and low part (split from the FP64 input), F_ij not
// recorded; l^(k+1) is then high + low, and E^(k+1), F^(k), Fbar^(k) (kept by the FP64 path
// only) are printed as 0. With global = 1 each line adds the landmark's term of the global test
// and its MM alternative: step (3), slack, E (FP64 only).
#include "../../paper_2305_07026_b300/csrc/daba_kernels.cuh"

#include <cstdio>
#include <vector>

using namespace daba;

template <class Real>
int run(int global, int n_lm, int first, double gamma, double xi, double eta, int accelerated) {
  constexpr bool LO = sizeof(Real) == 4;
  IterParams P{};
  P.xi = xi, P.eta = eta, P.eta1 = 1.0 - eta, P.hxi = 0.5 * xi;
  P.eta1f = float(1.0 - eta), P.hxif = float(0.5 * xi);
  P.accelerated = accelerated, P.restart_global = global;
  using RC = typename RecC<Real>::type;
  for (int j = 0; j < n_lm; ++j) {
    int n;
    double v[8];
    if (std::scanf("%d", &n) != 1) return 1;
    for (double& x : v)
      if (std::scanf("%lf", &x) != 1) return 1;
    std::vector<V4<Real>> sca(n), scb(n);
    std::vector<RC> cc(n);
    std::vector<uint16_t> inv(n);
    for (int q = 0; q < n; ++q) {
      double r[10];
      for (double& x : r)
        if (std::scanf("%lf", &x) != 1) return 1;
      sca[q] = {Real(r[0]), Real(r[1]), Real(r[2]), Real(r[3])};
      scb[q] = {Real(r[4]), Real(r[5]), Real(r[6]), Real(r[7])};
      cc[q] = RecC<Real>::make(Real(r[8]), Real(r[9]));
      inv[q] = (uint16_t)q;
    }
    V4<Real> A, B = {Real(v[4]), Real(v[5]), Real(v[6]), Real(LO ? 0.0 : v[7])};
    V4<float> lo0 = {0.f, 0.f, 0.f, 0.f};
    if constexpr (LO) {
      float h[3], o[3];
      for (int a = 0; a < 3; ++a) split_df(v[a], h[a], o[a]);
      A = {h[0], h[1], h[2], float(v[3])};
      lo0 = {o[0], o[1], o[2], 0.f};
    } else {
      A = {v[0], v[1], v[2], v[3]};
    }
    V4<Real> out[2], alt[2] = {};
    V4<float> lo_out[1];
    uint8_t rs = 0;
    double Fd = 0.0, Fbd = 0.0, gsum = 0.0;
    LpassOut<Real> O;
    O.lmrec_out = out, O.lm_lo_out = lo_out, O.lm_rs = &rs, O.lm_Fdiag = &Fd, O.lm_Fbdiag = &Fbd, O.lm_alt = alt;
    const int r = lpass_landmark<Real, LO>(sca.data(), scb.data(), cc.data(), inv.data(), 0, n, A, B, lo0, 0,
                                           Real(gamma), first, P, O, gsum);
    double l[3] = {double(out[0].x), double(out[0].y), double(out[0].z)};
    if (LO) l[0] += double(lo_out[0].x), l[1] += double(lo_out[0].y), l[2] += double(lo_out[0].z);
    std::printf("%.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %d", l[0], l[1], l[2],
                double(out[0].w), double(out[1].x), double(out[1].y), double(out[1].z), LO ? 0.0 : double(out[1].w),
                Fd, Fbd, r);
    if (global)
      std::printf(" %.17g %.17g %.17g %.17g %.17g %.17g", gsum, double(alt[0].x), double(alt[0].y), double(alt[0].z),
                  double(alt[0].w), double(alt[1].x));
    std::printf("\n");
  }
  return 0;
}

int main() {
  int bits, global, n_lm, first, accelerated;
  double gamma, xi, eta;
  if (std::scanf("%d %d %d %d %lf %lf %lf %d", &bits, &global, &n_lm, &first, &gamma, &xi, &eta, &accelerated) != 8)
    return 1;
  return bits == 32 ? run<float>(global, n_lm, first, gamma, xi, eta, accelerated)
                    : run<double>(global, n_lm, first, gamma, xi, eta, accelerated);
}
