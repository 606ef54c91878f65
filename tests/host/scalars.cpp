// The device's continuation of Nesterov's scalar (nesterov_next, used when the momentum reset
// keeps s on the device) built for the host: prints s^(0) = 1, s^(1), ..., s^(n) as 64-bit
// patterns (hex), one per line. stdin: "n".
#include "../../paper_2305_07026_b300/csrc/daba_kernels.cuh"

#include <cstdio>

using namespace daba;

int main() {
  int n = 0;
  if (std::scanf("%d", &n) != 1) return 1;
  double s = 1.0;
  for (int k = 0; k <= n; ++k) {
    std::printf("%016llx\n", (unsigned long long)__double_as_longlong(s));
    s = nesterov_next(s);
  }
  return 0;
}
