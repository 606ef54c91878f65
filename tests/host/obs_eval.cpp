// The library's per-observation evaluation (eval_obs, as the camera pass calls it, in FP64 or
// in FP32) compiled for the host and driven from stdin, so that a test can compare it with the
// oracle on the same inputs. The camera pack is written by the library's own write_pack_t; the
// FP32 landmark position is its high part and its displacement is rounded to FP32, as in the
// pass's landmark records.
// stdin: "bits loss c n" (bits 64 or 32; loss 0 trivial, 1 Huber, 2 Cauchy, 3 Welsch; c the loss
// scale), then n lines of 48 numbers: R^k (9, row-major), t^k (3), d^k (3), R^(k-1) (9),
// t^(k-1) (3), d^(k-1) (3), Rbar (9), l^k (3), l^(k-1) (3), u (2), gamma.
// stdout per observation: lambda, R e (3), r = |e|^2, rho(r), w at x^k; lambda, Rbar ebar (3),
// w at the extrapolated iterate; the surrogate gap.
#include "../../paper_2305_07026_b300/csrc/daba_kernels.cuh"

#include <cstdio>

using namespace daba;

template <int LOSS, class Real>
void run(double c, int n) {
  LossC<Real> L;
  L.c = Real(c), L.c2 = Real(c * c), L.inv_c2 = Real(1.0 / (c * c));
  for (int o = 0; o < n; ++o) {
    double v[48];
    for (double& x : v)
      if (std::scanf("%lf", &x) != 1) return;
    const double *Rk = v, *tk = v + 9, *dk = v + 12, *Rp = v + 15, *tp = v + 24, *dp = v + 27, *Rb = v + 30,
                 *lk = v + 39, *lp = v + 42, *u = v + 45;
    CamT<double> x, dx;
    for (int a = 0; a < 9; ++a) x.R[a] = Rk[a], dx.R[a] = Rk[a] - Rp[a];
    for (int a = 0; a < 3; ++a) x.t[a] = tk[a], dx.t[a] = tk[a] - tp[a], x.d[a] = dk[a], dx.d[a] = dk[a] - dp[a];
    V4<Real> pk[P4N];
    write_pack_t<Real>(x, dx, Rb, pk);
    Real l[3], lo[3], dl[3];
    for (int a = 0; a < 3; ++a) {
      split_real(lk[a], l[a], lo[a]);
      dl[a] = to_real<Real>(lk[a] - lp[a]);
    }
    ObsEval<Real> ev;
    eval_obs<LOSS, Real>(pk, l[0], l[1], l[2], dl[0], dl[1], dl[2], to_real<Real>(u[0]),
                         to_real<Real>(u[1]), Real(v[47]), L, ev);
    const double out[13] = {double(ev.lam), double(ev.Re0), double(ev.Re1), double(ev.Re2), double(ev.r),
                            double(ev.rho), double(ev.w),   double(ev.lamb), double(ev.Reb0), double(ev.Reb1),
                            double(ev.Reb2), double(ev.wb), double(ev.gap)};
    for (int k = 0; k < 13; ++k) std::printf(k ? " %.17g" : "%.17g", out[k]);
    std::printf("\n");
  }
}

template <class Real>
void dispatch(int loss, double c, int n) {
  if (loss == LOSS_TRIVIAL) run<LOSS_TRIVIAL, Real>(c, n);
  if (loss == LOSS_HUBER) run<LOSS_HUBER, Real>(c, n);
  if (loss == LOSS_CAUCHY) run<LOSS_CAUCHY, Real>(c, n);
  if (loss == LOSS_WELSCH) run<LOSS_WELSCH, Real>(c, n);
}

int main() {
  int bits = 64, loss = 0, n = 0;
  double c = 1.0;
  if (std::scanf("%d %d %lf %d", &bits, &loss, &c, &n) != 4) return 1;
  if (bits == 32)
    dispatch<float>(loss, c, n);
  else
    dispatch<double>(loss, c, n);
  return 0;
}
