// daba_grad.cuh -- gradient of the objective F(x) (Eq. Fobj) w.r.t. the boundary cameras
// [w, t, f, k1, k2], landmarks and observed pixels, by hand-written adjoint kernels.
//
// Per observation (internal units, lambda the minimiser of Eq. lambdaij, so its own
// variation drops out): with E = R p - lambda q (world frame, q = l - t), r = |E|^2 and
// w = rho'(r), dF_ij/d(R p) = w E. Hence (Eq. DFij)
//   dF/dR = w E p^T,   dF/dt = lambda w E,   dF/dl = -lambda w E,
//   dF/dd = (w E . R e3) (1, s, s^2),   dF/du'_a = (w R^T E)_a + 2 u'_a (d2 + 2 d3 s)(w R^T E)_3.
// The camera terms are summed per chunk (one warp per chunk, as the camera pass) and carried
// to the boundary per camera: rotation through the tangent gradient vee(R^T G - G^T R) and
// the right Jacobian of Exp at the boundary axis-angle vector, intrinsics through
// d = (f/s, k1 s/f, k2 s^3/f^3), everything times s^2 (F in pixel^2) and pixels times s.
// Landmark terms go through the landmark-side records and are summed per landmark.
#pragma once

#include "daba_kernels.cuh"

namespace daba {

enum { GP_R = 0, GP_T = 9, GP_D = 12, GP_F = 15, GP_N = 16 };   // chunk partial of the gradient pass

template <int LOSS, class Real, class Real2, bool HAS_LO>
__global__ void __launch_bounds__(32)
    k_grad_obs(int n_chunks, const int* __restrict__ chunk_cam, const int* __restrict__ chunk_beg,
               const int* __restrict__ c_lm, const Real2* __restrict__ c_u, const int* __restrict__ c_rpos,
               const int* __restrict__ ci_order, const V4<Real>* __restrict__ pack, const V4<Real>* __restrict__ lmrec,
               const V4<float>* __restrict__ lm_lo, LossC<Real> L, double s, Real* __restrict__ part,
               V4<Real>* __restrict__ g_lrec, double2* __restrict__ g_u) {
  __shared__ V4<Real> spk[P4N];
  const int warp = blockIdx.x;
  const int lane = threadIdx.x;
  if (warp >= n_chunks) return;
  const int cam = chunk_cam[warp];
  const int b = chunk_beg[warp], e = chunk_beg[warp + 1];
  if (lane < P4N) spk[lane] = pack[(size_t)cam * P4N + lane];
  __syncwarp();
  const V4<Real> a0 = spk[P4_RK + 0], a1 = spk[P4_RK + 1], a2 = spk[P4_RK + 2];
  const V4<Real> g0 = spk[P4_DR + 0], g1 = spk[P4_DR + 1], g2 = spk[P4_DR + 2];
  const V4<Real> d = spk[P4_D];
  Real acc[GP_N];
#pragma unroll
  for (int k = 0; k < GP_N; ++k) acc[k] = Real(0);
  for (int o = b + lane; o < e; o += 32) {
    const int j = c_lm[o];
    const Real2 uu = c_u[o];
    const V4<Real> A = lmrec[2 * (size_t)j];
    Real q0 = A.x - a0.w, q1 = A.y - a1.w, q2 = A.z - a2.w;
    if (HAS_LO) {
      const V4<float> lo = lm_lo[j];
      q0 += Real(lo.x) - g0.w;
      q1 += Real(lo.y) - g1.w;
      q2 += Real(lo.z) - g2.w;
    }
    const Real u0 = uu.x, u1 = uu.y;
    const Real sq = u0 * u0 + u1 * u1;
    const Real pz = d.x + d.y * sq + d.z * sq * sq;
    const Real Rp0 = a0.x * u0 + a0.y * u1 + a0.z * pz;
    const Real Rp1 = a1.x * u0 + a1.y * u1 + a1.z * pz;
    const Real Rp2 = a2.x * u0 + a2.y * u1 + a2.z * pz;
    const Real lam = (q0 * Rp0 + q1 * Rp1 + q2 * Rp2) / (q0 * q0 + q1 * q1 + q2 * q2);
    const Real E0 = Rp0 - lam * q0, E1 = Rp1 - lam * q1, E2 = Rp2 - lam * q2;
    Real rho, w;
    rho_w<LOSS, Real>(L, E0 * E0 + E1 * E1 + E2 * E2, rho, w);
    const Real G0 = w * E0, G1 = w * E1, G2 = w * E2;   // dF/d(R p)
    acc[GP_R + 0] += G0 * u0;
    acc[GP_R + 1] += G0 * u1;
    acc[GP_R + 2] += G0 * pz;
    acc[GP_R + 3] += G1 * u0;
    acc[GP_R + 4] += G1 * u1;
    acc[GP_R + 5] += G1 * pz;
    acc[GP_R + 6] += G2 * u0;
    acc[GP_R + 7] += G2 * u1;
    acc[GP_R + 8] += G2 * pz;
    acc[GP_T + 0] += lam * G0;
    acc[GP_T + 1] += lam * G1;
    acc[GP_T + 2] += lam * G2;
    // camera-frame dF/dp = R^T G
    const Real c0 = a0.x * G0 + a1.x * G1 + a2.x * G2;
    const Real c1 = a0.y * G0 + a1.y * G1 + a2.y * G2;
    const Real c2 = a0.z * G0 + a1.z * G1 + a2.z * G2;
    acc[GP_D + 0] += c2;
    acc[GP_D + 1] += c2 * sq;
    acc[GP_D + 2] += c2 * sq * sq;
    acc[GP_F] += Real(0.5) * rho;
    V4<Real> gl;
    gl.x = -lam * G0;
    gl.y = -lam * G1;
    gl.z = -lam * G2;
    gl.w = Real(0);
    g_lrec[c_rpos[o]] = gl;
    const Real dpz = Real(2) * (d.y + Real(2) * d.z * sq);
    g_u[ci_order[o]] = make_double2(double(c0 + c2 * dpz * u0) * s, double(c1 + c2 * dpz * u1) * s);
  }
#pragma unroll
  for (int k = 0; k < GP_N; ++k) {
    Real v = acc[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    acc[k] = v;
  }
  if (lane == 0) {
    Real* out = part + (size_t)warp * CP_STRIDE;
#pragma unroll
    for (int k = 0; k < GP_N; ++k) out[k] = acc[k];
  }
}

// J_r(w)^T v with J_r = I - (1 - cos th)/th^2 [w]x + (th - sin th)/th^3 [w]x^2 (series below 1e-6)
__device__ inline void right_jacobian_t(const double* w, const double* v, double* out) {
  const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const double th = sqrt(th2);
  double a, b;
  if (th < 1e-6) {
    a = 0.5 - th2 / 24.0;
    b = 1.0 / 6.0 - th2 / 120.0;
  } else {
    a = (1.0 - cos(th)) / th2;
    b = (th - sin(th)) / (th2 * th);
  }
  const double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
  double J[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double k2 = 0.0;
      for (int m = 0; m < 3; ++m) k2 += K[i * 3 + m] * K[m * 3 + j];
      J[i * 3 + j] = (i == j ? 1.0 : 0.0) - a * K[i * 3 + j] + b * k2;
    }
  for (int j = 0; j < 3; ++j) out[j] = J[0 * 3 + j] * v[0] + J[1 * 3 + j] * v[1] + J[2 * 3 + j] * v[2];
}

// One thread per camera: chunk partials summed in FP64, carried to the boundary parameters;
// also F of the camera's observations (FP64) into cam_F.
template <class Real>
__global__ void k_grad_cams(int M, const int* __restrict__ cam_chunk_ptr, const Real* __restrict__ part,
                            const double* __restrict__ cam_x, double s, double* __restrict__ g_cams,
                            double* __restrict__ cam_F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double acc[GP_N];
  for (int k = 0; k < GP_N; ++k) acc[k] = 0.0;
  for (int c = cam_chunk_ptr[i]; c < cam_chunk_ptr[i + 1]; ++c)
    for (int k = 0; k < GP_N; ++k) acc[k] += widen(part[(size_t)c * CP_STRIDE + k]);
  const double* x = cam_x + (size_t)i * CSTRIDE;
  double R[9];
  for (int a = 0; a < 9; ++a) R[a] = x[CS_R + a];
  // tangent gradient of F(R Exp(phi)): vee(R^T G - G^T R), G = acc[GP_R..] (row-major 3x3)
  double A[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      A[r * 3 + c] = R[0 * 3 + r] * acc[GP_R + 0 * 3 + c] + R[1 * 3 + r] * acc[GP_R + 1 * 3 + c] +
                     R[2 * 3 + r] * acc[GP_R + 2 * 3 + c];
  const double gphi[3] = {A[7] - A[5], A[2] - A[6], A[3] - A[1]};
  double wv[3], gw[3];
  rot_log(R, wv);
  right_jacobian_t(wv, gphi, gw);
  const double d1 = x[CS_D + 0], d2 = x[CS_D + 1], d3 = x[CS_D + 2];
  const double f = d1 * s, k1 = d2 * f / s, k2 = d3 * f * f * f / (s * s * s);
  const double gf = acc[GP_D + 0] / s - acc[GP_D + 1] * k1 * s / (f * f) - 3.0 * acc[GP_D + 2] * k2 * s * s * s / (f * f * f * f);
  const double gk1 = acc[GP_D + 1] * s / f;
  const double gk2 = acc[GP_D + 2] * s * s * s / (f * f * f);
  const double s2 = s * s;
  double* o = g_cams + (size_t)i * 9;
  for (int a = 0; a < 3; ++a) {
    o[a] = gw[a] * s2;
    o[3 + a] = acc[GP_T + a] * s2;
  }
  o[6] = gf * s2;
  o[7] = gk1 * s2;
  o[8] = gk2 * s2;
  cam_F[i] = acc[GP_F];
}

// One CTA per landmark tile, one thread per landmark: its records' landmark gradients summed
// (through the slot map), times s^2, to the landmark's boundary (external) index.
template <class Real>
__global__ void __launch_bounds__(LPASS_THREADS)
    k_grad_lms(const int* __restrict__ tile_lm, const int* __restrict__ lm_ptr, const uint16_t* __restrict__ t_inv,
               const V4<Real>* __restrict__ g_lrec, const int* __restrict__ lperm, double s2,
               double* __restrict__ g_lms) {
  const int lb = tile_lm[blockIdx.x], le = tile_lm[blockIdx.x + 1];
  const int jl = threadIdx.x;
  if (jl >= le - lb) return;
  const int ob = lm_ptr[lb];
  const int s0 = lm_ptr[lb + jl], s1 = lm_ptr[lb + jl + 1];
  double gx = 0.0, gy = 0.0, gz = 0.0;
  for (int sl = s0; sl < s1; ++sl) {
    const V4<Real> g = g_lrec[ob + t_inv[sl]];
    gx += widen(g.x);
    gy += widen(g.y);
    gz += widen(g.z);
  }
  double* o = g_lms + (size_t)lperm[lb + jl] * 3;
  o[0] = gx * s2;
  o[1] = gy * s2;
  o[2] = gz * s2;
}

// pixels re-uploaded in camera order, in internal units (input: user order, nnz x 2 doubles)
template <class Real2>
__global__ void k_set_pixels(long long nnz, const int* __restrict__ ci_order, const double* __restrict__ uv,
                             double s, Real2* __restrict__ c_u, int* __restrict__ bad) {
  const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nnz) return;
  const size_t k = (size_t)ci_order[o];
  const double x = uv[2 * k], y = uv[2 * k + 1];
  if (!(isfinite(x) && isfinite(y))) atomicMin(bad, (int)k);
  Real2 v;
  v.x = decltype(v.x)(x / s);
  v.y = decltype(v.y)(y / s);
  c_u[o] = v;
}

}  // namespace daba
