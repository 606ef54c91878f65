// The library's ProjRot3D variants built for the host and driven from stdin, so that a test can
// compare them with the oracle's SVD projection: proj_rot3d (Horn's quaternion method with Jacobi
// rotations) in FP64 and FP32, proj_rot3d_polar (scaled Newton for det K > 0, else Jacobi),
// proj_rot3d_from (warm-started Newton on the rotation, may decline), proj_rot3d_near
// (Newton-Schulz for K near a rotation, else Jacobi) in FP64 and FP32.
// stdin: "n", then n lines of K (9, row-major) and a warm start Q0 (9).
// stdout per line: jacobi64 (9) jacobi32 (9) polar64 (9) from64_ok (1) from64 (9) near64 (9) near32 (9).
#include "../../paper_2305_07026_b300/csrc/daba_device.cuh"

#include <cstdio>

using namespace daba;

int main() {
  int n = 0;
  if (std::scanf("%d", &n) != 1) return 1;
  for (int i = 0; i < n; ++i) {
    double K[9], Q0[9];
    for (double& v : K)
      if (std::scanf("%lf", &v) != 1) return 1;
    for (double& v : Q0)
      if (std::scanf("%lf", &v) != 1) return 1;
    float Kf[9], Rf[9], Nf[9];
    for (int a = 0; a < 9; ++a) Kf[a] = float(K[a]);
    double J[9], P[9], F[9], Nd[9];
    proj_rot3d<double>(K, J);
    proj_rot3d<float>(Kf, Rf);
    proj_rot3d_polar<double>(K, P);
    for (double& v : F) v = 0.0;
    const bool ok = proj_rot3d_from<double>(K, Q0, F);
    proj_rot3d_near<double>(K, Nd);
    proj_rot3d_near<float>(Kf, Nf);
    for (double v : J) std::printf("%.17g ", v);
    for (float v : Rf) std::printf("%.9g ", double(v));
    for (double v : P) std::printf("%.17g ", v);
    std::printf("%d ", ok ? 1 : 0);
    for (double v : F) std::printf("%.17g ", v);
    for (double v : Nd) std::printf("%.17g ", v);
    for (int a = 0; a < 9; ++a) std::printf(a < 8 ? "%.9g " : "%.9g\n", double(Nf[a]));
  }
  return 0;
}
