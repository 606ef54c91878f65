// The library's integer-only FP64 <-> FP32 conversions (narrow, split_df, widen) built for the
// host and driven from stdin, so that a test can compare them bit for bit with IEEE-754
// conversions. stdin: "n", then n lines of one double given as its 64-bit pattern (hex) and one
// float given as its 32-bit pattern (hex). stdout per line: narrow(d), split_df(d) hi and lo
// (32-bit patterns), widen(f) (64-bit pattern), all in hex.
#include "../../paper_2305_07026_b300/csrc/daba_device.cuh"

#include <cinttypes>
#include <cstdio>

using namespace daba;

int main() {
  int n = 0;
  if (std::scanf("%d", &n) != 1) return 1;
  for (int i = 0; i < n; ++i) {
    unsigned long long db = 0;
    unsigned fb = 0;
    if (std::scanf("%llx %x", &db, &fb) != 2) return 1;
    const double d = __longlong_as_double((long long)db);
    float hi, lo;
    split_df(d, hi, lo);
    const double w = widen(__uint_as_float(fb));
    std::printf("%08x %08x %08x %016llx\n", __float_as_uint(narrow(d)), __float_as_uint(hi), __float_as_uint(lo),
                (unsigned long long)__double_as_longlong(w));
  }
  return 0;
}
