// The library's double-float addition (df_add: the MIXED landmark pass adds each landmark's
// FP32 step to its (hi, lo) FP32 pair with it) built for the host and driven from stdin, so that
// a test can compare it with exact rational arithmetic. stdin: "n", then n lines of three floats
// hi, lo, x given as 32-bit patterns (hex). stdout per line: hi and lo after df_add(hi, lo, x),
// as 32-bit patterns.
#include "../../paper_2305_07026_b300/csrc/daba_kernels.cuh"

#include <cstdio>

using namespace daba;

int main() {
  int n = 0;
  if (std::scanf("%d", &n) != 1) return 1;
  for (int i = 0; i < n; ++i) {
    unsigned h = 0, l = 0, x = 0;
    if (std::scanf("%x %x %x", &h, &l, &x) != 3) return 1;
    float hi = __uint_as_float(h), lo = __uint_as_float(l);
    df_add(hi, lo, __uint_as_float(x));
    std::printf("%08x %08x\n", __float_as_uint(hi), __float_as_uint(lo));
  }
  return 0;
}
