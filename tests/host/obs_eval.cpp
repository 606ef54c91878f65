// The library's per-observation evaluation (eval_obs, FP64 instantiation) compiled for the host,
// driven from stdin so that a test can compare it with the oracle on the same inputs.
// stdin: "loss c n" (loss 0 trivial, 1 Huber, 2 Cauchy, 3 Welsch; c the loss scale), then n lines
// of 48 numbers: R^k (9, row-major), t^k (3), d^k (3), R^(k-1) (9), t^(k-1) (3), d^(k-1) (3),
// Rbar (9), l^k (3), l^(k-1) (3), u (2), gamma.
// stdout per observation: lambda, R e (3), r = |e|^2, rho(r), w at x^k; lambda, Rbar ebar (3),
// w at the extrapolated iterate; the surrogate gap.
#include "../../paper_2305_07026_b300/csrc/daba_device.cuh"

#include <cstdio>

using namespace daba;

template <int LOSS>
void run(const LossC<double>& L, int n) {
  for (int o = 0; o < n; ++o) {
    double v[48];
    for (double& x : v)
      if (std::scanf("%lf", &x) != 1) return;
    const double *Rk = v, *tk = v + 9, *dk = v + 12, *Rp = v + 15, *tp = v + 24, *dp = v + 27, *Rb = v + 30,
                 *lk = v + 39, *lp = v + 42, *u = v + 45;
    const double gamma = v[47];
    // the camera pack as the library writes it (FP64: no low parts)
    V4<double> pk[P4N];
    for (int r = 0; r < 3; ++r) {
      pk[P4_RK + r] = {Rk[3 * r], Rk[3 * r + 1], Rk[3 * r + 2], tk[r]};
      pk[P4_RB + r] = {Rb[3 * r], Rb[3 * r + 1], Rb[3 * r + 2], tk[r] - tp[r]};
      pk[P4_DR + r] = {Rk[3 * r] - Rp[3 * r], Rk[3 * r + 1] - Rp[3 * r + 1], Rk[3 * r + 2] - Rp[3 * r + 2], 0.0};
    }
    pk[P4_D] = {dk[0], dk[1], dk[2], 0.0};
    pk[P4_DD] = {dk[0] - dp[0], dk[1] - dp[1], dk[2] - dp[2], 0.0};
    ObsEval<double> ev;
    eval_obs<LOSS, double>(pk, lk[0], lk[1], lk[2], 0.0, 0.0, 0.0, lk[0] - lp[0], lk[1] - lp[1], lk[2] - lp[2], u[0],
                           u[1], gamma, L, ev);
    std::printf("%.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g\n", ev.lam, ev.Re0,
                ev.Re1, ev.Re2, ev.r, ev.rho, ev.w, ev.lamb, ev.Reb0, ev.Reb1, ev.Reb2, ev.wb, ev.gap);
  }
}

int main() {
  int loss = 0, n = 0;
  double c = 1.0;
  if (std::scanf("%d %lf %d", &loss, &c, &n) != 3) return 1;
  LossC<double> L;
  L.c = c, L.c2 = c * c, L.inv_c2 = 1.0 / (c * c);
  if (loss == LOSS_TRIVIAL) run<LOSS_TRIVIAL>(L, n);
  if (loss == LOSS_HUBER) run<LOSS_HUBER>(L, n);
  if (loss == LOSS_CAUCHY) run<LOSS_CAUCHY>(L, n);
  if (loss == LOSS_WELSCH) run<LOSS_WELSCH>(L, n);
  return 0;
}
