// The objective-only evaluations of F_ij (Eq. Fij) built for the host and driven from stdin:
// eval_F4 (the camera-pack form of k_objective behind daba_objective; FP64, and FP32 with the
// landmark and the camera centre as FP32 high and low parts) and eval_F (the flat-pack form of
// the allocation-free objective, FP64, q = l - t formed by the caller).
// stdin: "loss c n", then n lines R (9, row-major) t (3) d (3) l (3) u (2).
// stdout per line: eval_F4 in FP64, eval_F4 in FP32, eval_F in FP64.
#include "../../paper_2305_07026_b300/csrc/daba_kernels.cuh"

#include <cstdio>

using namespace daba;

template <int LOSS>
void run(double c, int n) {
  LossC<double> L64;
  L64.c = c, L64.c2 = c * c, L64.inv_c2 = 1.0 / (c * c);
  LossC<float> L32;
  L32.c = float(c), L32.c2 = float(c * c), L32.inv_c2 = float(1.0 / (c * c));
  for (int o = 0; o < n; ++o) {
    double v[20];
    for (double& x : v)
      if (std::scanf("%lf", &x) != 1) return;
    CamT<double> x, dx;
    for (int a = 0; a < 9; ++a) x.R[a] = v[a], dx.R[a] = 0.0;
    for (int a = 0; a < 3; ++a) x.t[a] = v[9 + a], x.d[a] = v[12 + a], dx.t[a] = dx.d[a] = 0.0;
    const double* l = v + 15;
    V4<double> pk64[P4N];
    V4<float> pk32[P4N];
    write_pack_t<double>(x, dx, x.R, pk64);
    write_pack_t<float>(x, dx, x.R, pk32);
    const double f64 = eval_F4<LOSS, double>(pk64, l[0], l[1], l[2], 0.0, 0.0, 0.0, v[18], v[19], L64);
    float h[3], lo[3];
    for (int a = 0; a < 3; ++a) split_df(l[a], h[a], lo[a]);
    const float f32 = eval_F4<LOSS, float>(pk32, h[0], h[1], h[2], lo[0], lo[1], lo[2], float(v[18]), float(v[19]),
                                           L32);
    double flat[18];
    for (int a = 0; a < 9; ++a) flat[PK_R + a] = v[a];
    for (int a = 0; a < 3; ++a) flat[PK_D + a] = v[12 + a];
    const double fflat = eval_F<LOSS, double>(flat, l[0] - v[9], l[1] - v[10], l[2] - v[11], v[18], v[19], L64);
    std::printf("%.17g %.9g %.17g\n", f64, double(f32), fflat);
  }
}

int main() {
  int loss = 0, n = 0;
  double c = 1.0;
  if (std::scanf("%d %lf %d", &loss, &c, &n) != 3) return 1;
  if (loss == LOSS_TRIVIAL) run<LOSS_TRIVIAL>(c, n);
  if (loss == LOSS_HUBER) run<LOSS_HUBER>(c, n);
  if (loss == LOSS_CAUCHY) run<LOSS_CAUCHY>(c, n);
  if (loss == LOSS_WELSCH) run<LOSS_WELSCH>(c, n);
  return 0;
}
