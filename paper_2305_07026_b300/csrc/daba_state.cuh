// daba_state.cuh -- the boundary state of daba_set_state / daba_get_state converted on the
// device: cameras [w, t, f, k1, k2] <-> internal (R, t, d) in units of s pixels, landmarks
// gathered / scattered through the internal landmark numbering, validation and the
// Assumption 2 check (landmark away from every camera centre that observes it).
#pragma once

#include <limits.h>

#include "daba_kernels.cuh"

namespace daba {

// Validation flags (int): [0] first camera with a non-finite parameter, [1] first landmark
// with a non-finite coordinate, [2] first camera with a non-positive focal length (among the
// cameras whose parameters are finite); INT_MAX where there is none.
enum { CHK_CAM_NONFINITE = 0, CHK_LM_NONFINITE = 1, CHK_FOCAL = 2, CHK_N = 4 };

__global__ void k_chk_init(int* __restrict__ chk, unsigned long long* __restrict__ bad_obs) {
  if (threadIdx.x < CHK_N) chk[threadIdx.x] = INT_MAX;
  if (threadIdx.x == 0) *bad_obs = ~0ull;
}

__global__ void k_check_state(int M, int N, const double* __restrict__ cams, const double* __restrict__ lms,
                              int* __restrict__ chk) {
  const int n = M > N ? M : N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < M) {
      const double* c = cams + (size_t)i * 9;
      bool fin = true;
#pragma unroll
      for (int a = 0; a < 9; ++a) fin = fin && isfinite(c[a]);
      if (!fin)
        atomicMin(&chk[CHK_CAM_NONFINITE], i);
      else if (!(c[6] > 0.0))
        atomicMin(&chk[CHK_FOCAL], i);
    }
    if (i < N) {
      const double* l = lms + (size_t)i * 3;
      if (!(isfinite(l[0]) && isfinite(l[1]) && isfinite(l[2]))) atomicMin(&chk[CHK_LM_NONFINITE], i);
    }
  }
}

// x^0 = x^(-1) of the cameras: R = exp([w]x), t, d = (f, k1 s / f, k2 s^3 / f^3) / (s, 1, 1)
// with f in units of s pixels; displacement and restart metrics zero.
__global__ void k_set_cams(int M, const double* __restrict__ cams, double s, double* __restrict__ cam_x,
                           double* __restrict__ cam_dx, double* __restrict__ cam_S, double* __restrict__ cam_E) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double* c = cams + (size_t)i * 9;
  double x[CSTRIDE];
#pragma unroll
  for (int a = 0; a < CSTRIDE; ++a) x[a] = 0.0;
  rodrigues(c, x + CS_R);
  const double f = c[6];
#pragma unroll
  for (int a = 0; a < 3; ++a) x[CS_T + a] = c[3 + a];
  x[CS_D + 0] = f / s;
  x[CS_D + 1] = c[7] * s / f;
  x[CS_D + 2] = c[8] * s * s * s / (f * f * f);
  double* xo = cam_x + (size_t)i * CSTRIDE;
  double* dxo = cam_dx + (size_t)i * CSTRIDE;
#pragma unroll
  for (int a = 0; a < CSTRIDE; ++a) {
    xo[a] = x[a];
    dxo[a] = 0.0;
  }
  cam_S[i] = 0.0;
  cam_E[i] = 0.0;
}

// landmark record (l, delta = 0, S = 0, E = 0) at the internal index; MIXED keeps l as a
// float high part in the record and the float low part l - hi in lm_lo
template <class Real, bool HAS_LO>
__global__ void k_set_lms(int N, const double* __restrict__ lms, const int* __restrict__ linv,
                          V4<Real>* __restrict__ rec, V4<float>* __restrict__ lo) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const size_t q = (size_t)linv[j];
  const double v0 = lms[(size_t)j * 3 + 0], v1 = lms[(size_t)j * 3 + 1], v2 = lms[(size_t)j * 3 + 2];
  V4<Real> A, Z;
  Real l0, l1, l2;
  split_real(v0, A.x, l0);
  split_real(v1, A.y, l1);
  split_real(v2, A.z, l2);
  A.w = Real(0);
  Z.x = Z.y = Z.z = Z.w = Real(0);
  rec[2 * q] = A;
  rec[2 * q + 1] = Z;
  if (HAS_LO) {
    V4<float> L;
    L.x = float(l0);
    L.y = float(l1);
    L.z = float(l2);
    L.w = 0.f;
    lo[q] = L;
  }
}

__global__ void k_get_cams(int M, const double* __restrict__ cam_x, double s, double* __restrict__ cams) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double* x = cam_x + (size_t)i * CSTRIDE;
  double R[9], c[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) R[a] = x[CS_R + a];
  rot_log(R, c);
#pragma unroll
  for (int a = 0; a < 3; ++a) c[3 + a] = x[CS_T + a];
  const double f = x[CS_D + 0] * s;
  c[6] = f;
  c[7] = x[CS_D + 1] * f / s;
  c[8] = x[CS_D + 2] * f * f * f / (s * s * s);
  double* o = cams + (size_t)i * 9;
#pragma unroll
  for (int a = 0; a < 9; ++a) o[a] = c[a];
}

template <class Real, bool HAS_LO>
__global__ void k_get_lms(int N, const V4<Real>* __restrict__ rec, const V4<float>* __restrict__ lo,
                          const int* __restrict__ linv, double* __restrict__ lms) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const size_t q = (size_t)linv[j];
  const V4<Real> A = rec[2 * q];
  double v0 = double(A.x), v1 = double(A.y), v2 = double(A.z);
  if (HAS_LO) {
    const V4<float> L = lo[q];
    v0 += double(L.x);
    v1 += double(L.y);
    v2 += double(L.z);
  }
  lms[(size_t)j * 3 + 0] = v0;
  lms[(size_t)j * 3 + 1] = v1;
  lms[(size_t)j * 3 + 2] = v2;
}

// A MIXED landmark state (float records, float low parts) as the FP64 path's records: l = high +
// low part (exact in FP64), the displacement and the slack S widened, E (kept by the FP64 path
// only) zero. Internal order is kept. The reverse mode of MIXED contexts runs its FP64 adjoint
// on these.
__global__ void k_lm_widen(int N, const V4<float>* __restrict__ rec, const V4<float>* __restrict__ lo,
                           V4<double>* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const V4<float> A = rec[2 * (size_t)q], B = rec[2 * (size_t)q + 1], L = lo[q];
  V4<double> a, b;
  a.x = double(A.x) + double(L.x);
  a.y = double(A.y) + double(L.y);
  a.z = double(A.z) + double(L.z);
  a.w = double(A.w);
  b.x = double(B.x);
  b.y = double(B.y);
  b.z = double(B.z);
  b.w = 0.0;
  out[2 * (size_t)q] = a;
  out[2 * (size_t)q + 1] = b;
}

// Assumption 2 on the current iterate: |l_j - t_i|^2 > 1e-24 max(1, |t_i|^2) for every
// observation; one block per camera chunk, the smallest failing device position kept.
// FP64 path: in FP64. MIXED: l and t as FP32 high + low parts and q = (l_hi - t_hi) +
// (l_lo - t_lo) in FP32 (the high-part difference is exact when l is near t, so q keeps
// about 2^-48 relative accuracy where the test matters), no FP64 instruction per observation.
template <class Real, bool HAS_LO>
__global__ void k_check_degenerate(const int* __restrict__ chunk_cam, const int* __restrict__ chunk_beg,
                                   const int* __restrict__ c_lm, const double* __restrict__ cam_x,
                                   const V4<Real>* __restrict__ rec, const V4<float>* __restrict__ lo,
                                   unsigned long long* __restrict__ bad_obs) {
  const int cam = chunk_cam[blockIdx.x];
  const int b = chunk_beg[blockIdx.x], e = chunk_beg[blockIdx.x + 1];
  const double* x = cam_x + (size_t)cam * CSTRIDE;
  Real th[3], tl[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) split_real(x[CS_T + a], th[a], tl[a]);
  const Real tt = th[0] * th[0] + th[1] * th[1] + th[2] * th[2];
  const Real thr = Real(1e-24) * (tt > Real(1) ? tt : Real(1));
  for (int o = b + threadIdx.x; o < e; o += blockDim.x) {
    const size_t j = (size_t)c_lm[o];
    const V4<Real> A = rec[2 * j];
    Real q0 = A.x - th[0], q1 = A.y - th[1], q2 = A.z - th[2];
    if (HAS_LO) {
      const V4<float> L = lo[j];
      q0 += Real(L.x) - tl[0];
      q1 += Real(L.y) - tl[1];
      q2 += Real(L.z) - tl[2];
    }
    if (!(q0 * q0 + q1 * q1 + q2 * q2 > thr)) atomicMin(bad_obs, (unsigned long long)o);
  }
}

__global__ void k_iota(int n, int* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = i;
}

}  // namespace daba
