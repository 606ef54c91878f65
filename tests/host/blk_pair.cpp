// The block solve's per-pair math (the code nvcc compiles into k_blk_solve) built for the host
// and driven from stdin, so that a test can compare it with the oracle and with central
// differences of its own residual:
//   blk_intra_jac  R e = (I - q q^T/|q|^2) R p of an intra-block pair and its Jacobians with
//                  respect to the camera step (phi, tau, delta) and the landmark step epsilon,
//   blk_F          F_ij = rho(|e|^2) / 2 of the pair,
//   sym3_inv       the inverse of a packed symmetric 3 x 3 matrix (a landmark's damped block).
// stdin: "pair loss c n" and n lines of 20 numbers R (9, row-major), t (3), d (3), l (3), u (2);
// stdout per line: R e (3), Jc (3 x 9, row-major), Jl (3 x 3, row-major), F.
// Or stdin: "sym3 n" and n lines of 6 numbers (xx, yx, yy, zx, zy, zz); stdout the inverse, packed.
#include "../../paper_2305_07026_b300/csrc/daba_blocks.cuh"

#include <cstdio>
#include <cstring>

using namespace daba;

int main() {
  char mode[16];
  if (std::scanf("%15s", mode) != 1) return 1;
  if (std::strcmp(mode, "sym3") == 0) {
    int n;
    if (std::scanf("%d", &n) != 1) return 1;
    for (int o = 0; o < n; ++o) {
      double C[6], I[6];
      for (double& x : C)
        if (std::scanf("%lf", &x) != 1) return 1;
      sym3_inv(C, I);
      for (double x : I) std::printf("%.17g ", x);
      std::printf("\n");
    }
    return 0;
  }
  int loss, n;
  double c;
  if (std::scanf("%d %lf %d", &loss, &c, &n) != 3) return 1;
  LossC<double> L;
  L.c = c, L.c2 = c * c, L.inv_c2 = 1.0 / (c * c);
  for (int o = 0; o < n; ++o) {
    double v[20];
    for (double& x : v)
      if (std::scanf("%lf", &x) != 1) return 1;
    CamT<double> cam;
    for (int a = 0; a < 9; ++a) cam.R[a] = v[a];
    for (int a = 0; a < 3; ++a) cam.t[a] = v[9 + a], cam.d[a] = v[12 + a];
    const double* l = v + 15;
    double f[3], Jc[3][9], Jl[3][3];
    blk_intra_jac(cam, l, v[18], v[19], f, Jc, Jl);
    const double F = blk_F(cam, l, v[18], v[19], L, loss);
    for (double x : f) std::printf("%.17g ", x);
    for (auto& r : Jc)
      for (double x : r) std::printf("%.17g ", x);
    for (auto& r : Jl)
      for (double x : r) std::printf("%.17g ", x);
    std::printf("%.17g\n", F);
  }
  return 0;
}
