// Assumption 2 on the host: the library's k_check_degenerate (the check daba_run makes of the
// current iterate before it runs: every observed landmark away from its camera's centre, with a
// scale-aware threshold), built for the host and run one chunk at a time, FP64 and MIXED (l and
// t as FP32 high and low parts). stdin: "M N nnz", M lines of camera centres t (3), N lines of
// landmarks l (3), then nnz lines "camera landmark" sorted by camera. One chunk per camera.
// stdout: the smallest failing observation position of the FP64 and of the MIXED check
// (18446744073709551615 where none fails).
#include "../../paper_2305_07026_b300/csrc/daba_state.cuh"

#include <cstdio>
#include <vector>

using namespace daba;

int main() {
  int M, N, nnz;
  if (std::scanf("%d %d %d", &M, &N, &nnz) != 3) return 1;
  std::vector<double> cam_x((size_t)M * CSTRIDE, 0.0);
  for (int i = 0; i < M; ++i)
    for (int a = 0; a < 3; ++a)
      if (std::scanf("%lf", &cam_x[(size_t)i * CSTRIDE + CS_T + a]) != 1) return 1;
  std::vector<V4<double>> rec64((size_t)N * 2);
  std::vector<V4<float>> rec32((size_t)N * 2), lo(N);
  for (int j = 0; j < N; ++j) {
    double l[3];
    for (double& v : l)
      if (std::scanf("%lf", &v) != 1) return 1;
    rec64[2 * j] = {l[0], l[1], l[2], 0.0};
    float h[3], o[3];
    for (int a = 0; a < 3; ++a) split_df(l[a], h[a], o[a]);
    rec32[2 * j] = {h[0], h[1], h[2], 0.f};
    lo[j] = {o[0], o[1], o[2], 0.f};
  }
  std::vector<int> c_lm(nnz), chunk_cam, chunk_beg;
  int prev = -1;
  for (int o = 0; o < nnz; ++o) {
    int i;
    if (std::scanf("%d %d", &i, &c_lm[o]) != 2) return 1;
    if (i != prev) chunk_cam.push_back(i), chunk_beg.push_back(o), prev = i;
  }
  chunk_beg.push_back(nnz);
  unsigned long long bad64 = ~0ull, bad32 = ~0ull;
  blockDim.x = 1, gridDim.x = (unsigned)chunk_cam.size(), threadIdx.x = 0;
  for (size_t c = 0; c < chunk_cam.size(); ++c) {
    blockIdx.x = (unsigned)c;
    k_check_degenerate<double, false>(chunk_cam.data(), chunk_beg.data(), c_lm.data(), cam_x.data(), rec64.data(),
                                      nullptr, &bad64);
    k_check_degenerate<float, true>(chunk_cam.data(), chunk_beg.data(), c_lm.data(), cam_x.data(), rec32.data(),
                                    lo.data(), &bad32);
  }
  std::printf("%llu %llu\n", bad64, bad32);
  return 0;
}
