// The boundary's state conversions (the code nvcc compiles into daba_set_state and
// daba_get_state) built for the host and run one element at a time: k_check_state (the first
// camera with a non-finite parameter, the first landmark with a non-finite coordinate, the
// first finite camera with a non-positive focal length), k_set_cams (boundary camera
// [w, t, f, k1, k2] -> internal R, t, d in units of s pixels), k_get_cams (back), and the
// landmark records of both paths, k_set_lms / k_get_lms (FP64; MIXED as an FP32 high and low
// part). stdin: "M N s", M lines of 9 camera parameters, N lines of 3 coordinates. stdout: the
// three check indices (INT_MAX where none); per camera its internal R (9) t (3) d (3) and its
// boundary parameters read back (9); per landmark its coordinates read back from the FP64 and
// from the MIXED records (6).
#include "../../paper_2305_07026_b300/csrc/daba_state.cuh"

#include <cstdio>
#include <vector>

using namespace daba;

int main() {
  int M, N;
  double s;
  if (std::scanf("%d %d %lf", &M, &N, &s) != 3) return 1;
  std::vector<double> cams((size_t)M * 9), lms((size_t)N * 3);
  for (double& v : cams)
    if (std::scanf("%lf", &v) != 1) return 1;
  for (double& v : lms)
    if (std::scanf("%lf", &v) != 1) return 1;
  // one thread per block, one block after the other
  blockDim.x = 1, gridDim.x = 1, threadIdx.x = 0, blockIdx.x = 0;
  int chk[CHK_N];
  unsigned long long bad = 0;
  for (unsigned t = 0; t < CHK_N; ++t) {
    threadIdx.x = t;
    k_chk_init(chk, &bad);
  }
  threadIdx.x = 0;
  k_check_state(M, N, cams.data(), lms.data(), chk);
  std::printf("%d %d %d\n", chk[CHK_CAM_NONFINITE], chk[CHK_LM_NONFINITE], chk[CHK_FOCAL]);
  std::vector<double> cam_x((size_t)M * CSTRIDE), cam_dx((size_t)M * CSTRIDE), cS(M), cE(M), back((size_t)M * 9);
  for (int i = 0; i < M; ++i) {
    blockIdx.x = (unsigned)i;
    k_set_cams(M, cams.data(), s, cam_x.data(), cam_dx.data(), cS.data(), cE.data());
  }
  for (int i = 0; i < M; ++i) {
    blockIdx.x = (unsigned)i;
    k_get_cams(M, cam_x.data(), s, back.data());
  }
  for (int i = 0; i < M; ++i) {
    for (int a = 0; a < 15; ++a) std::printf("%.17g ", cam_x[(size_t)i * CSTRIDE + a]);
    for (int a = 0; a < 9; ++a) std::printf(a < 8 ? "%.17g " : "%.17g\n", back[(size_t)i * 9 + a]);
  }
  std::vector<int> linv(N);
  for (int j = 0; j < N; ++j) linv[j] = N - 1 - j;   // an internal order other than the input's
  std::vector<V4<double>> rec64((size_t)N * 2);
  std::vector<V4<float>> rec32((size_t)N * 2), lo((size_t)N);
  std::vector<double> l64((size_t)N * 3), l32((size_t)N * 3);
  for (int j = 0; j < N; ++j) {
    blockIdx.x = (unsigned)j;
    k_set_lms<double, false>(N, lms.data(), linv.data(), rec64.data(), nullptr);
    k_set_lms<float, true>(N, lms.data(), linv.data(), rec32.data(), lo.data());
  }
  for (int j = 0; j < N; ++j) {
    blockIdx.x = (unsigned)j;
    k_get_lms<double, false>(N, rec64.data(), nullptr, linv.data(), l64.data());
    k_get_lms<float, true>(N, rec32.data(), lo.data(), linv.data(), l32.data());
  }
  for (int j = 0; j < N; ++j)
    std::printf("%.17g %.17g %.17g %.17g %.17g %.17g\n", l64[3 * j], l64[3 * j + 1], l64[3 * j + 2], l32[3 * j],
                l32[3 * j + 1], l32[3 * j + 2]);
  return 0;
}
