// Host stand-ins for the CUDA names the library's device headers use, so that their math
// (compiled with g++ as plain inline C++) can be checked on the CPU. Every stand-in is the
// operation's definition: warp shuffles return the caller's own value (one-lane warps), the
// rounded arithmetic intrinsics are the plain IEEE operations, the packed FP32 ones act per
// component. Nothing here runs on a GPU.
#pragma once
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
using std::isfinite;
struct float2 { float x, y; };
struct double2 { double x, y; };
struct float4 { float x, y, z, w; };
struct int4 { int x, y, z, w; };
inline double2 make_double2(double a, double b) { return {a, b}; }
inline float2 make_float2(float a, float b) { return {a, b}; }
inline int4 make_int4(int a, int b, int c, int d) { return {a, b, c, d}; }
struct host_dim3 { unsigned x = 0, y = 0, z = 0; };
static host_dim3 threadIdx, blockIdx, blockDim, gridDim;
inline unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
inline float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
inline long long __double_as_longlong(double d) { long long u; std::memcpy(&u, &d, 8); return u; }
inline double __longlong_as_double(long long u) { double d; std::memcpy(&d, &u, 8); return d; }
template <class T> T __shfl_xor_sync(unsigned, T v, int) { return v; }
template <class T> T __shfl_sync(unsigned, T v, int) { return v; }
template <class T> T __ldg(const T* p) { return *p; }
template <class T> T __ldcg(const T* p) { return *p; }
inline void __nanosleep(unsigned) {}
inline unsigned atomicExch(unsigned* p, unsigned v) { const unsigned o = *p; *p = v; return o; }
inline void __syncwarp() {}
inline void __syncthreads() {}
inline void __threadfence() {}
inline int atomicOr(int* p, int v) { const int o = *p; *p |= v; return o; }
inline int atomicMin(int* p, int v) { const int o = *p; *p = std::min(o, v); return o; }
inline unsigned long long atomicMin(unsigned long long* p, unsigned long long v) {
  const unsigned long long o = *p;
  *p = std::min(o, v);
  return o;
}
inline unsigned atomicAdd(unsigned* p, unsigned v) { const unsigned o = *p; *p += v; return o; }
inline float __fdividef(float a, float b) { return a / b; }
inline float rsqrtf(float a) { return 1.0f / std::sqrt(a); }
inline size_t __cvta_generic_to_shared(const void*) { return 0; }
typedef int cudaError_t;
inline double __dmul_rn(double a, double b) { return a * b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline float __fadd_rn(float a, float b) { return a + b; }
inline double __dadd_rn(double a, double b) { return a + b; }
inline double __dsub_rn(double a, double b) { return a - b; }
inline double __ddiv_rn(double a, double b) { return a / b; }
inline float2 __fmul2_rn(float2 a, float2 b) { return {a.x * b.x, a.y * b.y}; }
inline float2 __fadd2_rn(float2 a, float2 b) { return {a.x + b.x, a.y + b.y}; }
inline float2 __ffma2_rn(float2 a, float2 b, float2 c) { return {std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y)}; }
