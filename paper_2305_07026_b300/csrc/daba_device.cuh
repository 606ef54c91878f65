// daba_device.cuh -- device-side math of one DABA iteration (arXiv 2305.07026).
//
// Notation follows the paper: camera c_i = (R_i, t_i, d_i) with R_i camera-to-world
// and t_i the centre, landmark l_j, observed pixel u_ij (internal units of s_norm
// pixels). For a conditioning iterate z the per-observation quantities of
// Proposition 1 are
//   p = [u; d1 + d2 s + d3 s^2] (Eq. ray, s = |u|^2), q = l - t,
//   lambda = q^T R p / |q|^2 (Eq. lambdaij), R e = R p - lambda q (Eq. error),
//   r = |e|^2, w = rho'(r) (Eq. w), and the centred residuals
//   R p + lambda t - g = R e / 2 (camera side), lambda l - g = -R e / 2 (landmark side)
// which follow from Eq. g. Everything a block solve needs is a weighted sum of
// products of these terms (see daba_kernels.cuh).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace daba {

enum { LOSS_TRIVIAL = 0, LOSS_HUBER = 1, LOSS_CAUCHY = 2, LOSS_WELSCH = 3 };

// Loss constants in internal units: c (scale) and 1/c^2.
template <class Real>
struct LossC {
  Real c, c2, inv_c2;
};

// Division and reciprocal square root: the FP32 path uses the fast approximate
// instructions (a few ulp); FP64 is exact.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float frsqrt(float a) { return rsqrtf(a); }
__device__ __forceinline__ double frsqrt(double a) { return 1.0 / sqrt(a); }

// Multiply and add rounded separately (never contracted into a fused multiply-add), so that
// every kernel that inlines the loss evaluates it to the same bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// rho(r) and rho'(r) of the robust losses of Assumption 1 (App. B).
template <int LOSS, class Real>
__device__ __forceinline__ void rho_w(const LossC<Real>& L, Real r, Real& rho, Real& w) {
  if (LOSS == LOSS_TRIVIAL) {
    rho = r;
    w = Real(1);
  } else if (LOSS == LOSS_HUBER) {
    if (r > L.c2) {
      const Real is = frsqrt(r);
      rho = Real(2) * L.c * (r * is) - L.c2;
      w = L.c * is;
    } else {
      rho = r;
      w = Real(1);
    }
  } else if (LOSS == LOSS_CAUCHY) {
    const Real x = mul_rn(r, L.inv_c2);
    rho = mul_rn(L.c2, log1p(x));
    w = fdiv(Real(1), add_rn(Real(1), x));
  } else {
    const Real ex = exp(-mul_rn(r, L.inv_c2));
    rho = mul_rn(L.c2, add_rn(Real(1), -ex));
    w = ex;
  }
}

// Flat camera layout read by eval_F (Real offsets): R[9] (row-major), t[3], pad[3], d[3].
enum { PK_R = 0, PK_TH = 9, PK_D = 15 };

// 16-byte (float) / 32-byte (double) vector used for the camera pack and landmark records.
template <class Real>
struct alignas(4 * sizeof(Real)) V4 {
  Real x, y, z, w;
};

// Camera pack read by the observation passes (V4 entries, one pack per camera):
//   [P4_RK + r] = (R^k row r, t^k_r hi)      [P4_RB + r] = (Rbar row r, dt_r)
//   [P4_DR + r] = (dR row r, t^k_r lo)       [P4_D] = (d^k, 0)      [P4_DD] = (dd, 0)
// with dR = R^k - R^(k-1), dt = t^k - t^(k-1), dd = d^k - d^(k-1) formed in FP64 and
// Rbar the extrapolated rotation of Eq. nesterov_R. R^(k-1) = R^k - dR is formed in registers.
enum { P4_RK = 0, P4_RB = 3, P4_DR = 6, P4_D = 9, P4_DD = 10, P4N = 12 };

// Per-observation output of the three-point evaluation.
template <class Real>
struct ObsEval {
  Real lam, Re0, Re1, Re2, r, rho, w;   // at x^k
  Real lamb, Reb0, Reb1, Reb2, wb;      // at the extrapolated iterate xbar^k
  Real gap;                             // F_ij(x^k) - P_ij(c^k|x^(k-1)) - Q_ij(l^k|x^(k-1))
};

// Evaluates one observation at x^k, xbar^k and x^(k-1).
//   pk: camera pack; (l0,l1,l2): landmark position l^k (in MIXED its high part: the camera pass
//   reads no low part); dl = l^k - l^(k-1); u: pixel (internal units);
//   gamma: extrapolation ratio of Eq. nesterov_scalar.
// q^k = l^k - t^k is formed with the camera centre's high and low parts, so that it keeps FP32
// relative accuracy far from the origin.
// xbar: Rbar, dbar = d + gamma dd, qbar = q + gamma (dl - dt) (Eq. nesterov_x).
// x^(k-1): R' = R^k - dR, d' = d - dd, q' = q - (dl - dt); R' p' is formed as R^k p^k - G with
// G = dR p^k + R' e3 (phi . dd) (p' = p^k - e3 (phi . dd)), which the gap below needs anyway.
// The surrogate gap of Eq. DEalpha is written in displacement form: with X = R^k p^k +
// lambda' t^k, Y = lambda' l^k and g' of Eq. g at x^(k-1),
//   |X - g'|^2 + |Y - g'|^2 = |X - Y|^2 / 2 + 2 |(X + Y)/2 - g'|^2,
//   |X - Y|^2 = r^k + |q^k|^2 (lambda' - lambda^k)^2,
//   2 ((X + Y)/2 - g') = dR p^k + R' e3 (phi . dd) + lambda' (dt + dl) = G + lambda' (dt + dl) =: D,
// so gap = [rho(r^k) - rho(r') - w'(r^k - r')]/2 - w' |q^k|^2 (lambda' - lambda^k)^2 / 2
//          - w' |D|^2 / 2, every term of which is formed without cancellation of O(1) values.
template <int LOSS, class Real>
__device__ __forceinline__ void eval_obs(const V4<Real>* __restrict__ pk, Real l0, Real l1, Real l2, Real dl0,
                                         Real dl1, Real dl2, Real u0, Real u1, Real gamma, const LossC<Real>& L,
                                         ObsEval<Real>& o) {
  const V4<Real> a0 = pk[P4_RK + 0], a1 = pk[P4_RK + 1], a2 = pk[P4_RK + 2];
  const V4<Real> g0 = pk[P4_DR + 0], g1 = pk[P4_DR + 1], g2 = pk[P4_DR + 2];
  const V4<Real> b0 = pk[P4_RB + 0], b1 = pk[P4_RB + 1], b2 = pk[P4_RB + 2];
  const V4<Real> dd = pk[P4_DD], d = pk[P4_D];
  const Real s = u0 * u0 + u1 * u1;
  const Real s2 = s * s;
  const Real q0 = (l0 - a0.w) - g0.w;
  const Real q1 = (l1 - a1.w) - g1.w;
  const Real q2 = (l2 - a2.w) - g2.w;
  // ---- x^k
  const Real pz = d.x + d.y * s + d.z * s2;
  const Real Rp0 = a0.x * u0 + a0.y * u1 + a0.z * pz;
  const Real Rp1 = a1.x * u0 + a1.y * u1 + a1.z * pz;
  const Real Rp2 = a2.x * u0 + a2.y * u1 + a2.z * pz;
  const Real qq = q0 * q0 + q1 * q1 + q2 * q2;
  o.lam = fdiv(q0 * Rp0 + q1 * Rp1 + q2 * Rp2, qq);
  o.Re0 = Rp0 - o.lam * q0;
  o.Re1 = Rp1 - o.lam * q1;
  o.Re2 = Rp2 - o.lam * q2;
  o.r = o.Re0 * o.Re0 + o.Re1 * o.Re1 + o.Re2 * o.Re2;
  rho_w<LOSS, Real>(L, o.r, o.rho, o.w);
  // ---- displacements: (l^k - l^(k-1)) - (t^k - t^(k-1)) and phi . dd
  const Real e0 = dl0 - b0.w, e1 = dl1 - b1.w, e2 = dl2 - b2.w;
  const Real phidd = dd.x + dd.y * s + dd.z * s2;
  // ---- xbar^k
  {
    const Real pzb = pz + gamma * phidd;
    const Real qb0 = q0 + gamma * e0, qb1 = q1 + gamma * e1, qb2 = q2 + gamma * e2;
    const Real Rbp0 = b0.x * u0 + b0.y * u1 + b0.z * pzb;
    const Real Rbp1 = b1.x * u0 + b1.y * u1 + b1.z * pzb;
    const Real Rbp2 = b2.x * u0 + b2.y * u1 + b2.z * pzb;
    const Real qqb = qb0 * qb0 + qb1 * qb1 + qb2 * qb2;
    o.lamb = fdiv(qb0 * Rbp0 + qb1 * Rbp1 + qb2 * Rbp2, qqb);
    o.Reb0 = Rbp0 - o.lamb * qb0;
    o.Reb1 = Rbp1 - o.lamb * qb1;
    o.Reb2 = Rbp2 - o.lamb * qb2;
    const Real rb = o.Reb0 * o.Reb0 + o.Reb1 * o.Reb1 + o.Reb2 * o.Reb2;
    Real rhob;
    rho_w<LOSS, Real>(L, rb, rhob, o.wb);
  }
  // ---- x^(k-1) and the surrogate gap
  {
    // R' e3 (the third column of R' = R^k - dR) and G = dR p^k + R' e3 (phi . dd)
    const Real c0z = a0.z - g0.z, c1z = a1.z - g1.z, c2z = a2.z - g2.z;
    const Real G0 = g0.x * u0 + g0.y * u1 + g0.z * pz + c0z * phidd;
    const Real G1 = g1.x * u0 + g1.y * u1 + g1.z * pz + c1z * phidd;
    const Real G2 = g2.x * u0 + g2.y * u1 + g2.z * pz + c2z * phidd;
    const Real qp0 = q0 - e0, qp1 = q1 - e1, qp2 = q2 - e2;
    const Real Rpp0 = Rp0 - G0, Rpp1 = Rp1 - G1, Rpp2 = Rp2 - G2;
    const Real qqp = qp0 * qp0 + qp1 * qp1 + qp2 * qp2;
    const Real lamp = fdiv(qp0 * Rpp0 + qp1 * Rpp1 + qp2 * Rpp2, qqp);
    const Real Rep0 = Rpp0 - lamp * qp0, Rep1 = Rpp1 - lamp * qp1, Rep2 = Rpp2 - lamp * qp2;
    const Real rp = Rep0 * Rep0 + Rep1 * Rep1 + Rep2 * Rep2;
    Real rhop, wp;
    rho_w<LOSS, Real>(L, rp, rhop, wp);
    const Real D0 = G0 + lamp * (b0.w + dl0);
    const Real D1 = G1 + lamp * (b1.w + dl1);
    const Real D2 = G2 + lamp * (b2.w + dl2);
    const Real dlam = lamp - o.lam;
    o.gap = Real(0.5) * (o.rho - rhop - wp * (o.r - rp)) - Real(0.5) * wp * qq * dlam * dlam -
            Real(0.5) * wp * (D0 * D0 + D1 * D1 + D2 * D2);
  }
}

// F_ij(x^k) = rho(|e|^2) / 2 from the camera pack (Eq. Fij).
template <int LOSS, class Real>
__device__ __forceinline__ Real eval_F4(const V4<Real>* __restrict__ pk, Real l0, Real l1, Real l2, Real o0,
                                        Real o1, Real o2, Real u0, Real u1, const LossC<Real>& L) {
  const V4<Real> a0 = pk[P4_RK + 0], a1 = pk[P4_RK + 1], a2 = pk[P4_RK + 2];
  const V4<Real> g0 = pk[P4_DR + 0], g1 = pk[P4_DR + 1], g2 = pk[P4_DR + 2];
  const V4<Real> d = pk[P4_D];
  const Real q0 = (l0 - a0.w) + (o0 - g0.w);
  const Real q1 = (l1 - a1.w) + (o1 - g1.w);
  const Real q2 = (l2 - a2.w) + (o2 - g2.w);
  const Real s = u0 * u0 + u1 * u1;
  const Real pz = d.x + d.y * s + d.z * s * s;
  const Real Rp0 = a0.x * u0 + a0.y * u1 + a0.z * pz;
  const Real Rp1 = a1.x * u0 + a1.y * u1 + a1.z * pz;
  const Real Rp2 = a2.x * u0 + a2.y * u1 + a2.z * pz;
  const Real lam = fdiv(q0 * Rp0 + q1 * Rp1 + q2 * Rp2, q0 * q0 + q1 * q1 + q2 * q2);
  const Real e0 = Rp0 - lam * q0, e1 = Rp1 - lam * q1, e2 = Rp2 - lam * q2;
  Real rho, w;
  rho_w<LOSS, Real>(L, e0 * e0 + e1 * e1 + e2 * e2, rho, w);
  return Real(0.5) * rho;
}

// F_ij(x^k) = rho(|e|^2) / 2 only (Eq. Fij), flat camera layout, q formed by the caller.
template <int LOSS, class Real>
__device__ __forceinline__ Real eval_F(const Real* __restrict__ pk, Real q0, Real q1, Real q2, Real u0, Real u1,
                                       const LossC<Real>& L) {
  const Real s = u0 * u0 + u1 * u1;
  const Real pz = pk[PK_D + 0] + pk[PK_D + 1] * s + pk[PK_D + 2] * s * s;
  const Real Rp0 = pk[PK_R + 0] * u0 + pk[PK_R + 1] * u1 + pk[PK_R + 2] * pz;
  const Real Rp1 = pk[PK_R + 3] * u0 + pk[PK_R + 4] * u1 + pk[PK_R + 5] * pz;
  const Real Rp2 = pk[PK_R + 6] * u0 + pk[PK_R + 7] * u1 + pk[PK_R + 8] * pz;
  const Real lam = (q0 * Rp0 + q1 * Rp1 + q2 * Rp2) / (q0 * q0 + q1 * q1 + q2 * q2);
  const Real e0 = Rp0 - lam * q0, e1 = Rp1 - lam * q1, e2 = Rp2 - lam * q2;
  Real rho, w;
  rho_w<LOSS, Real>(L, e0 * e0 + e1 * e1 + e2 * e2, rho, w);
  return Real(0.5) * rho;
}

// ---------------------------------------------------------------------------
// FP64 small linear algebra for the block solves
// ---------------------------------------------------------------------------

// ProjRot3D (Eq. proj_rot3d): argmin_{R in SO(3)} |R - K|^2 = argmax <R, K>.
// With R(q) of a unit quaternion q = (w, x, y, z), <R(q), K> = q^T N(K) q for the
// symmetric 4x4 N below (expanding the quadratic form entry by entry), so the
// maximiser is R of the eigenvector of N's largest eigenvalue (Horn's method).
// The eigenvector is found with cyclic Jacobi rotations.
template <class T>
__device__ inline void proj_rot3d(const T* __restrict__ K, T* __restrict__ R) {
  T a[4][4];
  a[0][0] = K[0] + K[4] + K[8];
  a[1][1] = K[0] - K[4] - K[8];
  a[2][2] = -K[0] + K[4] - K[8];
  a[3][3] = -K[0] - K[4] + K[8];
  a[0][1] = a[1][0] = K[7] - K[5];
  a[0][2] = a[2][0] = K[2] - K[6];
  a[0][3] = a[3][0] = K[3] - K[1];
  a[1][2] = a[2][1] = K[1] + K[3];
  a[1][3] = a[3][1] = K[2] + K[6];
  a[2][3] = a[3][2] = K[5] + K[7];
  T v[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) v[i][j] = (i == j) ? T(1) : T(0);
  T scale = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]) + fabs(a[3][3]);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = i + 1; j < 4; ++j) scale += T(2) * fabs(a[i][j]);
  for (int sweep = 0; sweep < 20; ++sweep) {
    T off = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = i + 1; j < 4; ++j) off += a[i][j] * a[i][j];
    if (!(off > (sizeof(T) == 4 ? T(1e-13) : T(1e-34)) * scale * scale)) break;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
#pragma unroll
      for (int q = p + 1; q < 4; ++q) {
        const T apq = a[p][q];
        if (apq != T(0)) {
          // rotation in the (p, q) plane that zeroes a[p][q]: t = tan(phi) is the
          // smaller root of t^2 + 2 theta t - 1 = 0, theta = (a_qq - a_pp) / (2 a_pq)
          const T theta = (a[q][q] - a[p][p]) / (T(2) * apq);
          const T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
          const T c = T(1) / sqrt(t * t + T(1));
          const T s = t * c;
          a[p][p] -= t * apq;
          a[q][q] += t * apq;
          a[p][q] = a[q][p] = T(0);
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            if (r != p && r != q) {
              const T arp = a[r][p], arq = a[r][q];
              a[r][p] = a[p][r] = c * arp - s * arq;
              a[r][q] = a[q][r] = s * arp + c * arq;
            }
          }
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const T vrp = v[r][p], vrq = v[r][q];
            v[r][p] = c * vrp - s * vrq;
            v[r][q] = s * vrp + c * vrq;
          }
        }
      }
    }
  }
  T best = a[0][0], w = v[0][0], x = v[1][0], y = v[2][0], z = v[3][0];
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    if (a[k][k] > best) {
      best = a[k][k];
      w = v[0][k];
      x = v[1][k];
      y = v[2][k];
      z = v[3][k];
    }
  }
  const T n = T(1) / sqrt(w * w + x * x + y * y + z * z);
  w *= n;
  x *= n;
  y *= n;
  z *= n;
  R[0] = w * w + x * x - y * y - z * z;
  R[1] = T(2) * (x * y - w * z);
  R[2] = T(2) * (x * z + w * y);
  R[3] = T(2) * (x * y + w * z);
  R[4] = w * w - x * x + y * y - z * z;
  R[5] = T(2) * (y * z - w * x);
  R[6] = T(2) * (x * z - w * y);
  R[7] = T(2) * (y * z + w * x);
  R[8] = w * w - x * x - y * y + z * z;
}

// Exact FP32 -> FP64 widening with integer operations (IEEE-754 binary32 -> binary64:
// exponent rebiased by 1023 - 127, mantissa shifted by 29); FP32 subnormals become signed
// zero. Keeps the conversions of the camera solve off the FP64 unit.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
  const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  const unsigned long long ed = e == 0u ? 0ull : (e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u));
  return __longlong_as_double((long long)(sgn | (ed << 52) | (e == 0u ? 0ull : m)));
}
__device__ __forceinline__ double widen(double d) { return d; }

// FP64 -> FP32 conversions with integer operations on the IEEE-754 encodings (no FP64
// instruction). narrow(d) = the float nearest to d (ties to even); split_df(d) also gives
// lo = the float nearest to d - hi, so that hi + lo carries d to about 2^-48 relative.
// Magnitudes below the FP32 normal range give signed zero, above it infinity; the low part is
// zero for |d| < 2^-74, where the remainder's unit 2^(e-52) falls below the FP32 normal range.
__device__ __forceinline__ void split_df_impl(double d, float& hi, float& lo, bool want_lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned sgn = (unsigned)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ffu) - 1023;
  const unsigned long long mant = b & 0xfffffffffffffull;
  lo = 0.f;
  if (e < -126) {
    hi = __uint_as_float(sgn);
    return;
  }
  if (e > 127) {
    hi = __uint_as_float(sgn | 0x7f800000u | ((e == 1024 && mant) ? 0x400000u : 0u));
    return;
  }
  const unsigned long long sig = mant | (1ull << 52);   // 53-bit significand
  unsigned long long q = sig >> 29;                     // 24 bits
  const unsigned long long rem = sig & ((1ull << 29) - 1ull);
  if (rem > (1ull << 28) || (rem == (1ull << 28) && (q & 1ull))) q += 1ull;
  const long long r = (long long)sig - (long long)(q << 29);   // |r| <= 2^28, units of 2^(e-52)
  int eh = e;
  if (q == (1ull << 24)) {
    q >>= 1;
    eh += 1;
  }
  if (eh > 127) {
    hi = __uint_as_float(sgn | 0x7f800000u);
    return;
  }
  hi = __uint_as_float(sgn | ((unsigned)(eh + 127) << 23) | (unsigned)(q & 0x7fffffull));
  if (want_lo) {
    const int es = e - 52;
    if (es >= -126) {
      const float l = (float)(int)r * __uint_as_float((unsigned)(es + 127) << 23);
      lo = sgn ? -l : l;
    }
  }
}
__device__ __forceinline__ float narrow(double d) {
  float h, l;
  split_df_impl(d, h, l, false);
  return h;
}
__device__ __forceinline__ void split_df(double d, float& hi, float& lo) { split_df_impl(d, hi, lo, true); }

// d in the pass precision: FP32 via narrow, FP64 unchanged; split_real also gives the low
// part (zero in FP64)
template <class Real>
__device__ __forceinline__ Real to_real(double d);
template <>
__device__ __forceinline__ float to_real<float>(double d) { return narrow(d); }
template <>
__device__ __forceinline__ double to_real<double>(double d) { return d; }
__device__ __forceinline__ void split_real(double d, float& hi, float& lo) { split_df(d, hi, lo); }
__device__ __forceinline__ void split_real(double d, double& hi, double& lo) {
  hi = d;
  lo = 0.0;
}

// ---------------------------------------------------------------------------
// Number type of the block solves. The solves are written over a number type T; Num<T>
// supplies its constants, the scalar of the convergence tests, reciprocal square root and
// reciprocal, and conversions. Both precisions solve in T = double.
// ---------------------------------------------------------------------------
template <class T>
struct Num;

template <>
struct Num<double> {
  using S = double;
  static __device__ __forceinline__ double c(float x) { return (double)x; }
  static __device__ __forceinline__ S hi(double x) { return x; }
  static __device__ __forceinline__ bool pos(double x) { return x > 0.0; }
  static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / sqrt(x); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double from(double x) { return x; }
  static __device__ __forceinline__ double to_double(double x) { return x; }
  // squared step below which the rotation iterations stop (the next iterate is exact to rounding)
  static __device__ __forceinline__ S tiny() { return 1e-20; }
  // coefficients of the scaled Newton step X <- hz X + hiz C with C = det(X) X^{-T}
  static __device__ __forceinline__ void newton(const double* X, const double* C, double det, bool scaled,
                                                double& hz, double& hiz) {
    const double idet = 1.0 / det;
    double z = 1.0;
    if (scaled) {
      double nx = 0.0, nc = 0.0;
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        nx += X[a] * X[a];
        nc += C[a] * C[a];
      }
      z = sqrt(sqrt(nc / nx) * idet);
    }
    hz = 0.5 * z;
    hiz = 0.5 * idet / z;
  }
};

// FP32 solves (the MIXED camera solves): constants and conversions on the FP32 pipe (narrow and
// widen use integer operations).
template <>
struct Num<float> {
  using S = float;
  static __device__ __forceinline__ float c(float x) { return x; }
  static __device__ __forceinline__ S hi(float x) { return x; }
  static __device__ __forceinline__ bool pos(float x) { return x > 0.f; }
  static __device__ __forceinline__ float rsqrt(float x) { return 1.f / sqrtf(x); }
  static __device__ __forceinline__ float rcp(float x) { return 1.f / x; }
  static __device__ __forceinline__ float from(double x) { return narrow(x); }
  static __device__ __forceinline__ double to_double(float x) { return widen(x); }
  static __device__ __forceinline__ S tiny() { return 1e-12f; }
  static __device__ __forceinline__ void newton(const float* X, const float* C, float det, bool scaled, float& hz,
                                                float& hiz) {
    const float idet = 1.f / det;
    float z = 1.f;
    if (scaled) {
      float nx = 0.f, nc = 0.f;
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        nx += X[a] * X[a];
        nc += C[a] * C[a];
      }
      z = sqrtf(sqrtf(nc / nx) * idet);
    }
    hz = 0.5f * z;
    hiz = 0.5f * idet / z;
  }
};



// ProjRot3D for det K > 0: the projection onto SO(3) is then the orthogonal polar factor of
// K, computed with Higham's scaled Newton iteration X <- (z X + X^{-T} / z) / 2 with the
// Frobenius-norm scaling z = sqrt(|X^{-1}| / |X|), switched off once the iteration is close.
// The iteration converges quadratically, so once a step changes X by less than 1e-10 the new
// X is the polar factor to about 1e-20. Falls back to the Jacobi method above when det K <= 0
// or the iteration does not settle.
template <class T>
__device__ inline void proj_rot3d_polar(const T* __restrict__ K, T* __restrict__ R) {
  using N = Num<T>;
  using S = typename N::S;
  T X[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) X[a] = K[a];
  bool scaled = true;
  for (int it = 0; it < 40; ++it) {
    T C[9];   // cofactor matrix: X^{-T} = C / det X
    C[0] = X[4] * X[8] - X[5] * X[7];
    C[1] = X[5] * X[6] - X[3] * X[8];
    C[2] = X[3] * X[7] - X[4] * X[6];
    C[3] = X[2] * X[7] - X[1] * X[8];
    C[4] = X[0] * X[8] - X[2] * X[6];
    C[5] = X[1] * X[6] - X[0] * X[7];
    C[6] = X[1] * X[5] - X[2] * X[4];
    C[7] = X[2] * X[3] - X[0] * X[5];
    C[8] = X[0] * X[4] - X[1] * X[3];
    const T det = X[0] * C[0] + X[1] * C[1] + X[2] * C[2];
    if (!N::pos(det)) break;
    T hz, hiz;
    N::newton(X, C, det, scaled, hz, hiz);
    S dif = S(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const T y = hz * X[a] + hiz * C[a];
      const S d = N::hi(y - X[a]);
      dif += d * d;
      X[a] = y;
    }
    if (dif < S(1e-6)) scaled = false;
    if (dif < N::tiny()) {
#pragma unroll
      for (int a = 0; a < 9; ++a) R[a] = X[a];
      return;
    }
  }
  proj_rot3d(K, R);
}

// ProjRot3D(K) for det K > 0 from a rotation Q0 near the answer (the previous R-step's
// rotation or the conditioning rotation R_z). Newton's method on f(Q) = tr(Q^T K) over SO(3):
// with B = Q^T K, f(Q Exp(w)) = tr B + w . b - w^T H w / 2 + O(|w|^3),
//   b = (B21 - B12, B02 - B20, B10 - B01),  H = tr(B) I - (B + B^T) / 2,
// so the step solves H w = b (Cramer's rule) and Q <- Q Cay(w), the rotation of the
// quaternion (1, w/2) (equal to Exp(w) to second order, so the convergence stays quadratic).
// A fixed point has B = Q^T K symmetric; with H positive definite (leading minors checked) and
// det K > 0 it is positive definite, so Q is the polar factor: the maximiser. Once |w| <
// 1e-10 the next iterate is exact to rounding. Returns false (R untouched) if a step fails the
// checks or 8 steps do not settle; the caller then uses proj_rot3d_polar.
template <class T>
__device__ inline bool proj_rot3d_from(const T* __restrict__ K, const T* __restrict__ Q0, T* __restrict__ R) {
  using N = Num<T>;
  using S = typename N::S;
  const T detK = K[0] * (K[4] * K[8] - K[5] * K[7]) - K[1] * (K[3] * K[8] - K[5] * K[6]) +
                 K[2] * (K[3] * K[7] - K[4] * K[6]);
  if (!N::pos(detK)) return false;
  T Q[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) Q[a] = Q0[a];
  for (int it = 0; it < 8; ++it) {
    T B[9];   // Q^T K
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) B[r * 3 + c] = Q[0 * 3 + r] * K[0 * 3 + c] + Q[1 * 3 + r] * K[1 * 3 + c] + Q[2 * 3 + r] * K[2 * 3 + c];
    const T b0 = B[7] - B[5], b1 = B[2] - B[6], b2 = B[3] - B[1];
    const T tr = B[0] + B[4] + B[8];
    const T h00 = tr - B[0], h11 = tr - B[4], h22 = tr - B[8];
    const T h01 = N::c(-0.5f) * (B[1] + B[3]), h02 = N::c(-0.5f) * (B[2] + B[6]), h12 = N::c(-0.5f) * (B[5] + B[7]);
    // Cramer's rule with the leading minors as the positive-definiteness test
    const T m1 = h00 * h11 - h01 * h01;
    const T c00 = h11 * h22 - h12 * h12, c01 = h02 * h12 - h01 * h22, c02 = h01 * h12 - h02 * h11;
    const T c11 = h00 * h22 - h02 * h02, c12 = h01 * h02 - h00 * h12;
    const T det = h00 * c00 + h01 * c01 + h02 * c02;
    if (!N::pos(h00) || !N::pos(m1) || !N::pos(det)) return false;
    const T id = N::rcp(det);
    const T w0 = (c00 * b0 + c01 * b1 + c02 * b2) * id;
    const T w1 = (c01 * b0 + c11 * b1 + c12 * b2) * id;
    const T w2 = (c02 * b0 + c12 * b1 + m1 * b2) * id;
    // Q <- Q Cay(w), quaternion (1, w/2) normalised through 1 / (1 + |w|^2/4)
    const T x = N::c(0.5f) * w0, y = N::c(0.5f) * w1, z = N::c(0.5f) * w2;
    const T xx = x * x, yy = y * y, zz = z * z;
    const T in = N::rcp(N::c(1.0f) + xx + yy + zz);
    T C[9];
    C[0] = (N::c(1.0f) + xx - yy - zz) * in;
    C[1] = N::c(2.0f) * (x * y - z) * in;
    C[2] = N::c(2.0f) * (x * z + y) * in;
    C[3] = N::c(2.0f) * (x * y + z) * in;
    C[4] = (N::c(1.0f) - xx + yy - zz) * in;
    C[5] = N::c(2.0f) * (y * z - x) * in;
    C[6] = N::c(2.0f) * (x * z - y) * in;
    C[7] = N::c(2.0f) * (y * z + x) * in;
    C[8] = (N::c(1.0f) - xx - yy + zz) * in;
    T Qn[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) Qn[r * 3 + c] = Q[r * 3 + 0] * C[0 * 3 + c] + Q[r * 3 + 1] * C[1 * 3 + c] + Q[r * 3 + 2] * C[2 * 3 + c];
#pragma unroll
    for (int a = 0; a < 9; ++a) Q[a] = Qn[a];
    const S ww = N::hi(w0 * w0 + w1 * w1 + w2 * w2);
    if (ww < N::tiny()) {
#pragma unroll
      for (int a = 0; a < 9; ++a) R[a] = Q[a];
      return true;
    }
  }
  return false;
}

// ProjRot3D of a matrix K close to a rotation (the extrapolation R + gamma dR of
// Eq. nesterov_R): for det K > 0 the projection is the orthogonal polar factor of K, reached
// by the Newton-Schulz iteration X <- X (3 I - X^T X) / 2, which converges quadratically when
// |X^T X - I| < 1: once |X^T X - I|_F^2 < 1e-20 one more step reaches the polar factor.
// Falls back to proj_rot3d when K is not close enough or det K <= 0.
template <class T>
__device__ inline void proj_rot3d_near(const T* __restrict__ K, T* __restrict__ R) {
  using N = Num<T>;
  using S = typename N::S;
  const T det = K[0] * (K[4] * K[8] - K[5] * K[7]) - K[1] * (K[3] * K[8] - K[5] * K[6]) +
                K[2] * (K[3] * K[7] - K[4] * K[6]);
  T X[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) X[a] = K[a];
  bool ok = N::pos(det);
  for (int it = 0; it < 8 && ok; ++it) {
    T Sm[9];   // X^T X
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Sm[i * 3 + j] = X[0 * 3 + i] * X[0 * 3 + j] + X[1 * 3 + i] * X[1 * 3 + j] + X[2 * 3 + i] * X[2 * 3 + j];
    S dev = S(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const S dij = N::hi(i == j ? Sm[i * 3 + j] - N::c(1.0f) : Sm[i * 3 + j]);
        dev += dij * dij;
      }
    if (it == 0 && !(dev < S(0.25))) {
      ok = false;
      break;
    }
    T Y[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Y[i * 3 + j] = N::c(0.5f) * (N::c(3.0f) * X[i * 3 + j] -
                                     (X[i * 3 + 0] * Sm[0 * 3 + j] + X[i * 3 + 1] * Sm[1 * 3 + j] +
                                      X[i * 3 + 2] * Sm[2 * 3 + j]));
#pragma unroll
    for (int a = 0; a < 9; ++a) X[a] = Y[a];
    if (dev < N::tiny()) break;
    if (it == 7) ok = false;
  }
  if (ok) {
#pragma unroll
    for (int a = 0; a < 9; ++a) R[a] = X[a];
  } else {
    proj_rot3d(K, R);
  }
}

// ---------------------------------------------------------------------------
// Boundary rotation parameterisation (host and device): axis-angle w <-> R.
// ---------------------------------------------------------------------------

// R = exp([w]x) = I + a [w]x + b [w]x^2 with a = sin(th)/th, b = (1 - cos(th))/th^2 (Rodrigues'
// formula), th = |w|; the series of a and b below 1e-8.
__host__ __device__ inline void rodrigues(const double* w, double* R) {
  const double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  double a, b;
  if (th < 1e-8) {
    a = 1.0 - th * th / 6.0;
    b = 0.5 - th * th / 24.0;
  } else {
    a = sin(th) / th;
    b = (1.0 - cos(th)) / (th * th);
  }
  const double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double k2 = 0.0;
      for (int m = 0; m < 3; ++m) k2 += K[i * 3 + m] * K[m * 3 + j];
      R[i * 3 + j] = (i == j ? 1.0 : 0.0) + a * K[i * 3 + j] + b * k2;
    }
}

// w = log(R): the angle from atan2(|v|, (tr R - 1)/2) with v the axial vector of the
// antisymmetric part; for angles beyond 2 pi / 3 the axis comes from the largest column of
// the symmetric part (R + R^T)/2 - cos(th) I = (1 - cos th) n n^T, its sign from v.
__host__ __device__ inline void rot_log(const double* A, double* w) {
  const double c = (A[0] + A[4] + A[8] - 1.0) / 2.0;
  const double v[3] = {(A[7] - A[5]) / 2.0, (A[2] - A[6]) / 2.0, (A[3] - A[1]) / 2.0};
  const double sn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const double th = atan2(sn, c);
  if (c > -0.5) {
    const double f = sn > 1e-300 ? th / sn : 1.0;
    for (int k = 0; k < 3; ++k) w[k] = v[k] * f;
    return;
  }
  double B[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B[i * 3 + j] = 0.5 * (A[i * 3 + j] + A[j * 3 + i]) - (i == j ? c : 0.0);
  int kk = 0;
  for (int k = 1; k < 3; ++k)
    if (B[k * 4] > B[kk * 4]) kk = k;
  const double a[3] = {B[0 * 3 + kk], B[1 * 3 + kk], B[2 * 3 + kk]};
  const double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  const double sg = (a[0] * v[0] + a[1] * v[1] + a[2] * v[2]) < 0 ? -1.0 : 1.0;
  for (int k = 0; k < 3; ++k) w[k] = sg * a[k] / n * th;
}

}  // namespace daba
