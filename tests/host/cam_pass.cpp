// The camera half of one iteration built for the host (FP64, the code nvcc compiles into k_cpass
// and k_camsolve) and driven from stdin, so that a test can compare it with the oracle's
// iteration per camera block: each camera's statistics at the extrapolated iterate and at x^k,
// its F_ij and surrogate-gap sums (eval_obs + accumulate_cam, one chunk per camera), then
// camsolve_group: Eqs. DEalpha, Fak, lFak in slack form, the accelerated S-CAM solve
// (Eq. update_amm), the restart test (Eq. Eak) and the MM solve (Eq. update_mm). The group's
// two warps hand the MM solution over through shared memory and share no lane data, so they
// are run one after the other per camera: warp 1 (MM) first, then warp 0.
// With bits = 32 the MIXED instantiation runs: statistics evaluated and accumulated in FP32
// (one chunk per camera), the FP32 S-CAM solve on displacements added to the FP64 state, FP64
// restart metrics.
// With global = 1 the global restart variant runs: no per-block test, the accelerated solution
// kept, the MM alternative and E, S after a restart in cam_alt, E^(k+1) - Fbar^(k) in g_cam.
// With lm = 1 the camera solver is the LM variant (one successful Levenberg-Marquardt step).
// stdin: "bits global lm loss c xi eta n_alt accelerated first gamma gamma_next M", then per camera
// "m", R^k (9, row-major) t^k (3) d^k (3) R^(k-1) (9) t^(k-1) (3) d^(k-1) (3) Rbar (9) S E,
// then m lines l^k (3) l^(k-1) (3) u (2). stdout per camera: R t d of x^(k+1) (15), F^(k),
// Fbar^(k), E^(k+1), the next slack, restarted, sum of F_ij(x^k); with global = 1 also the
// camera's term of the global test and its MM alternative R t d, E, S (18).
#include "../../paper_2305_07026_b300/csrc/daba_kernels.cuh"

#include <cstdio>
#include <vector>

using namespace daba;

template <int LOSS, class Real>
bool camera_stats(double c, double gamma, const CamT<double>& x, const CamT<double>& dx, const double* Rb, int m,
                  Real* out) {
  LossC<Real> L;
  L.c = Real(c), L.c2 = Real(c * c), L.inv_c2 = Real(1.0 / (c * c));
  V4<Real> pk[P4N];
  write_pack_t<Real>(x, dx, Rb, pk);
  Real acc[CP_NACC];
  for (Real& a : acc) a = Real(0);
  for (int o = 0; o < m; ++o) {
    double v[8];
    for (double& q : v)
      if (std::scanf("%lf", &q) != 1) return false;
    Real l[3], lo[3];
    for (int a = 0; a < 3; ++a) split_real(v[a], l[a], lo[a]);
    const Real u0 = to_real<Real>(v[6]), u1 = to_real<Real>(v[7]);
    ObsEval<Real> ev;
    eval_obs<LOSS, Real>(pk, l[0], l[1], l[2], to_real<Real>(v[0] - v[3]), to_real<Real>(v[1] - v[4]),
                         to_real<Real>(v[2] - v[5]), u0, u1, Real(gamma), L, ev);
    accumulate_cam<Real>(acc, ev, u0, u1);
  }
  for (int k = 0; k < CP_NACC; ++k) out[part_slot(k)] = acc[k];
  return true;
}

template <class Real, int SOLVER>
int run(int global, int loss, double c, double xi, double eta, int n_alt, int accelerated, int first, double gamma,
        double gamma_next, int M) {
  std::vector<Real> part((size_t)M * CP_STRIDE, Real(0));
  std::vector<double> cam_x((size_t)M * CSTRIDE, 0.0), cam_dx((size_t)M * CSTRIDE, 0.0), cam_Rbar((size_t)M * 9),
      cam_S(M), cam_E(M), cam_F(M), cam_Fb(M), cam_Fsum(M);
  std::vector<uint8_t> cam_rs(M);
  std::vector<int> chunk_ptr(M + 1);
  std::vector<V4<Real>> pack_next((size_t)M * P4N);
  for (int i = 0; i < M; ++i) {
    int m;
    double v[41];
    if (std::scanf("%d", &m) != 1) return 1;
    for (double& q : v)
      if (std::scanf("%lf", &q) != 1) return 1;
    CamT<double> x, dx;
    for (int a = 0; a < 9; ++a) x.R[a] = v[a], dx.R[a] = v[a] - v[15 + a];
    for (int a = 0; a < 3; ++a) {
      x.t[a] = v[9 + a], dx.t[a] = v[9 + a] - v[24 + a];
      x.d[a] = v[12 + a], dx.d[a] = v[12 + a] - v[27 + a];
    }
    double* xs = &cam_x[(size_t)i * CSTRIDE];
    double* dxs = &cam_dx[(size_t)i * CSTRIDE];
    for (int a = 0; a < 9; ++a) xs[CS_R + a] = x.R[a], dxs[CS_R + a] = dx.R[a], cam_Rbar[(size_t)i * 9 + a] = v[30 + a];
    for (int a = 0; a < 3; ++a) {
      xs[CS_T + a] = x.t[a], dxs[CS_T + a] = dx.t[a];
      xs[CS_D + a] = x.d[a], dxs[CS_D + a] = dx.d[a];
    }
    cam_S[i] = v[39], cam_E[i] = v[40];
    chunk_ptr[i] = i;
    Real* out = &part[(size_t)i * CP_STRIDE];
    bool ok = false;
    if (loss == LOSS_TRIVIAL) ok = camera_stats<LOSS_TRIVIAL, Real>(c, gamma, x, dx, v + 30, m, out);
    if (loss == LOSS_HUBER) ok = camera_stats<LOSS_HUBER, Real>(c, gamma, x, dx, v + 30, m, out);
    if (loss == LOSS_CAUCHY) ok = camera_stats<LOSS_CAUCHY, Real>(c, gamma, x, dx, v + 30, m, out);
    if (loss == LOSS_WELSCH) ok = camera_stats<LOSS_WELSCH, Real>(c, gamma, x, dx, v + 30, m, out);
    if (!ok) return 1;
  }
  chunk_ptr[M] = M;
  const double gam[2] = {gamma, gamma_next};
  IterParams P{};
  P.gam = gam, P.xi = xi, P.eta = eta, P.eta1 = 1.0 - eta, P.hxi = 0.5 * xi;
  P.eta1f = float(1.0 - eta), P.hxif = float(0.5 * xi);
  P.accelerated = accelerated, P.n_alt = n_alt, P.restart_global = global;
  std::vector<double> cam_alt((size_t)M * 32, 0.0), g_cam(M, 0.0);
  P.cam_alt = cam_alt.data(), P.g_cam = g_cam.data();
  double sh_mm[32][16];
  for (int i = 0; i < M; ++i)
    for (int role = 1; role >= 0; --role)
      camsolve_group<Real, SOLVER, false>(i / 32, role, i % 32, sh_mm, 0, first, 0, M, chunk_ptr.data(),
                                            part.data(), cam_x.data(), cam_dx.data(), cam_Rbar.data(), P,
                                            cam_S.data(), cam_E.data(), cam_F.data(), cam_Fb.data(), cam_rs.data(),
                                            cam_Fsum.data(), pack_next.data());
  for (int i = 0; i < M; ++i) {
    const double* xs = &cam_x[(size_t)i * CSTRIDE];
    for (int a = 0; a < 15; ++a) std::printf("%.17g ", xs[a]);
    std::printf("%.17g %.17g %.17g %.17g %d %.17g", cam_F[i], cam_Fb[i], cam_E[i], cam_S[i], (int)cam_rs[i],
                cam_Fsum[i]);
    if (global) {
      const double* a = &cam_alt[(size_t)i * 32];
      std::printf(" %.17g", g_cam[i]);
      for (int q = 0; q < 15; ++q) std::printf(" %.17g", a[q]);
      std::printf(" %.17g %.17g", a[30], a[31]);
    }
    std::printf("\n");
  }
  return 0;
}

int main() {
  int bits, global, lm, loss, n_alt, accelerated, first, M;
  double c, xi, eta, gamma, gamma_next;
  if (std::scanf("%d %d %d %d %lf %lf %lf %d %d %d %lf %lf %d", &bits, &global, &lm, &loss, &c, &xi, &eta, &n_alt,
                 &accelerated, &first, &gamma, &gamma_next, &M) != 13)
    return 1;
  if (lm)
    return bits == 32 ? run<float, CAM_LM>(global, loss, c, xi, eta, n_alt, accelerated, first, gamma, gamma_next, M)
                      : run<double, CAM_LM>(global, loss, c, xi, eta, n_alt, accelerated, first, gamma, gamma_next, M);
  return bits == 32 ? run<float, CAM_SCAM>(global, loss, c, xi, eta, n_alt, accelerated, first, gamma, gamma_next, M)
                    : run<double, CAM_SCAM>(global, loss, c, xi, eta, n_alt, accelerated, first, gamma, gamma_next, M);
}
