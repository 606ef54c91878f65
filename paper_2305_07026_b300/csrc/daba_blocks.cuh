// daba_blocks.cuh -- Algorithm 1 with coarse blocks (Eq. Ealpha with E' not empty), FP64.
//
// A block holds up to BLK_MAX_CAMS cameras and any set of landmarks. Pairs whose camera and
// landmark share a block (E') keep their exact F_ij in the block surrogate; the others are split
// by the majorizer of Proposition 1. Per iteration:
//   1. the camera pass in block mode (k_cpass_blk): as k_cpass, but an intra pair adds to no
//      statistics, gap or landmark record; it adds F_ij to the camera's F sums;
//   2. the landmark pass in sum mode: every landmark's sums of its inter records (a, b at x̄^k
//      and at x^k, F_ij and the surrogate gap);
//   3. k_blk_solve, one CTA per block: the restart metrics (Eqs. DEalpha, Fak, lFak), one
//      successful Levenberg-Marquardt step on E^alpha(. | x̄^k) from x̄^k, the restart test
//      (Eq. Eak) and, where it fires, the LM step on E^alpha(. | x^k) from x^k.
// LM step: parameters (phi, tau, delta) of each camera (R = R_z Exp(phi), t = t_z + tau,
// d = d_z + delta) and epsilon of each landmark (l = l_z + epsilon). Gauss-Newton model: each
// camera's inter pairs and proximal term from its statistics (cam_lm_model); each landmark's inter
// pairs 2 a I and 2 b, proximal xi I; each intra pair the reweighted Gauss-Newton terms of
// R e = (I - q q^T/|q|^2) R p with w = rho'(|e|^2) at z. The damped system (H + mu diag H) is
// solved through the Schur complement of the cameras (9 per camera, every landmark's 3 x 3 block
// eliminated; dense Cholesky in shared memory); the step is taken if E^alpha decreases
// (surrogate differences term by term), otherwise mu grows tenfold, at most LM_TRIES times.
// Every sum runs in a fixed order, so results do not depend on the schedule.
#pragma once

#include <cooperative_groups.h>

#include "daba_kernels.cuh"

namespace daba {

constexpr int BLK_MAX_CAMS = 512;    // cameras per block (a Schur matrix of 4608 x 4608, 170 MB)
constexpr int BLK_SMEM_CAMS = 16;    // up to this many in every block: the block scratch in shared memory
constexpr int BLK_THREADS = 128;

// landmark sums written by the landmark pass in sum mode (per internal landmark)
enum { LS_AB = 0, LS_BB = 1, LS_AK = 4, LS_BK = 5, LS_F = 8, LS_G = 9, LS_N = 10 };
// per landmark scratch of the block solve: C (packed), C^-1 of the damped system, gradient,
// the solution, the F_ij at z of its intra pairs
enum { BL_C = 0, BL_CI = 6, BL_G = 12, BL_L = 15, BL_FZ = 18, BL_N = 20 };
// per intra pair scratch: B = w Jc^T Jl (9 x 3), B C^-1, and the camera-side terms w Jc^T Jc
// (packed lower 9 x 9) and w Jc^T f
enum { BI_B = 0, BI_BC = 27, BI_A = 54, BI_GC = 99, BI_N = 108 };

// per camera scratch of the block solve: x^k, the conditioning iterate z, the solution, the
// candidate; the statistics at x̄^k and x^k; the LM model (packed lower 9 x 9 and gradient)
struct BlkCam {
  CamT<double> ck, cz, cs, cb;
  double stb[39], stk[39];
  double A[45], g[9];
};

struct BlkArgs {
  int S, ld;   // blocks; row stride of the shared-memory Schur matrix (9 x the most cameras in a
               // block), 0 when the block scratch is in global memory (row stride 9 x the block's cameras)
  const int *cam_ptr, *cams;          // cameras of each block (ascending)
  const int *lm_ptr, *lms;            // landmarks of each block (internal ids, ascending)
  const int *io_ptr, *io_cam, *io_obs;   // per landmark entry: its intra pairs (local camera, observation), by camera
  const int *ci_ptr, *ci_obs, *ci_lm;    // per camera entry: its intra pairs (observation, landmark), by observation
  const int *ci_e, *ci_io;               // ... and the pair's landmark entry and its index in the landmark lists
  BlkCam* g_cam;                         // global scratch (ld = 0): per camera entry
  double* g_vec;                         // ... two vectors of 9 per camera entry (step and right-hand side)
  double* g_S;                           // ... the Schur matrices, block b's at g_soff[b]
  const long long* g_soff;
  // global restart: pass 1 takes the accelerated step and keeps it (cameras in the iteration's
  // cam_alt, landmarks in lsc), with the block's test term blk_g = E(k+1) - Fbar(k) and blk_Ealt =
  // E(k+1); pass 2, after the decision (g_fire), commits the kept step or the MM step. pass 0:
  // the per-block restart in one launch.
  int pass;
  double *blk_g, *blk_Ealt;
  const double2* c_u;
  const int* cam_chunk_ptr;
  const double* part;
  const double* lm_sums;   // LS_N per internal landmark
  double *cam_x, *cam_dx, *cam_Rbar, *cam_Fsum;
  uint8_t* cam_rs;
  const V4<double>* lmrec;   // landmark state of iteration k
  V4<double>* lmrec_out;     // of iteration k + 1
  double *blk_E, *blk_Fbar, *blk_F;
  uint8_t* blk_rs;
  double *lsc, *isc;   // BL_N per internal landmark, BI_N per intra pair
  V4<double>* pack_next;
  LossC<double> L;
  int loss;
};

template <int LOSS>
__device__ __forceinline__ void blk_rho(const LossC<double>& L, double r, double& rho, double& w) {
  rho_w<LOSS, double>(L, r, rho, w);
}
__device__ __forceinline__ void blk_rho_any(int loss, const LossC<double>& L, double r, double& rho, double& w) {
  switch (loss) {
    case LOSS_TRIVIAL: blk_rho<LOSS_TRIVIAL>(L, r, rho, w); break;
    case LOSS_HUBER: blk_rho<LOSS_HUBER>(L, r, rho, w); break;
    case LOSS_CAUCHY: blk_rho<LOSS_CAUCHY>(L, r, rho, w); break;
    default: blk_rho<LOSS_WELSCH>(L, r, rho, w); break;
  }
}

// R e = (I - q q^T/|q|^2) R p and its Jacobian: Jc (3 x 9: phi, tau, delta) and Jl (3 x 3)
__device__ inline void blk_intra_jac(const CamT<double>& c, const double* l, double u0, double u1, double* f,
                                     double Jc[3][9], double Jl[3][3]) {
  const double s = u0 * u0 + u1 * u1;
  const double p[3] = {u0, u1, c.d[0] + c.d[1] * s + c.d[2] * s * s};
  double v[3], q[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    v[r] = c.R[3 * r] * p[0] + c.R[3 * r + 1] * p[1] + c.R[3 * r + 2] * p[2];
    q[r] = l[r] - c.t[r];
  }
  const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
  const double lam = (q[0] * v[0] + q[1] * v[1] + q[2] * v[2]) / qq;
#pragma unroll
  for (int r = 0; r < 3; ++r) f[r] = v[r] - lam * q[r];
  double Pi[3][3], Dq[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Pi[r][k] = (r == k ? 1.0 : 0.0) - q[r] * q[k] / qq;
      Dq[r][k] = (r == k ? -lam : 0.0) - q[r] * (v[k] - 2.0 * lam * q[k]) / qq;
    }
  // d(R Exp(phi) p)/dphi = -R [p]x with [p]x the cross-product matrix of p
  const double px[3][3] = {{0.0, -p[2], p[1]}, {p[2], 0.0, -p[0]}, {-p[1], p[0], 0.0}};
  double Mr[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      Mr[r][k] = -(c.R[3 * r] * px[0][k] + c.R[3 * r + 1] * px[1][k] + c.R[3 * r + 2] * px[2][k]);
  double pe[3];   // Pi R e3
#pragma unroll
  for (int r = 0; r < 3; ++r) pe[r] = Pi[r][0] * c.R[2] + Pi[r][1] * c.R[5] + Pi[r][2] * c.R[8];
  const double ph[3] = {1.0, s, s * s};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Jc[r][k] = Pi[r][0] * Mr[0][k] + Pi[r][1] * Mr[1][k] + Pi[r][2] * Mr[2][k];
      Jc[r][3 + k] = -Dq[r][k];
      Jc[r][6 + k] = pe[r] * ph[k];
      Jl[r][k] = Dq[r][k];
    }
  }
}

// F_ij = rho(|e|^2) / 2 at (camera, landmark)
__device__ inline double blk_F(const CamT<double>& c, const double* l, double u0, double u1, const LossC<double>& L,
                               int loss) {
  const double s = u0 * u0 + u1 * u1;
  const double p[3] = {u0, u1, c.d[0] + c.d[1] * s + c.d[2] * s * s};
  double v[3], q[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    v[r] = c.R[3 * r] * p[0] + c.R[3 * r + 1] * p[1] + c.R[3 * r + 2] * p[2];
    q[r] = l[r] - c.t[r];
  }
  const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
  const double lam = (q[0] * v[0] + q[1] * v[1] + q[2] * v[2]) / qq;
  double r2 = 0.0;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double e = v[r] - lam * q[r];
    r2 += e * e;
  }
  double rho, w;
  blk_rho_any(loss, L, r2, rho, w);
  return 0.5 * rho;
}

// 3 x 3 symmetric (packed xx, yx, yy, zx, zy, zz) inverse and product
__device__ __forceinline__ void sym3_inv(const double* C, double* I) {
  const double a = C[0], b = C[1], c = C[2], d = C[3], e = C[4], f = C[5];
  const double A0 = c * f - e * e, A1 = -(b * f - e * d), A3 = b * e - c * d;
  const double id = 1.0 / (a * A0 + b * A1 + d * A3);
  I[0] = A0 * id;
  I[1] = A1 * id;
  I[2] = (a * f - d * d) * id;
  I[3] = A3 * id;
  I[4] = -(a * e - b * d) * id;
  I[5] = (a * c - b * b) * id;
}
__device__ __forceinline__ void sym3_mul(const double* S, const double* x, double* y) {
  y[0] = S[0] * x[0] + S[1] * x[1] + S[3] * x[2];
  y[1] = S[1] * x[0] + S[2] * x[1] + S[4] * x[2];
  y[2] = S[3] * x[0] + S[4] * x[1] + S[5] * x[2];
}

// landmark position of the conditioning iterate: x^k, or x̄^k = l + gamma (l - l^(k-1))
__device__ __forceinline__ void blk_lpos(const V4<double>* lmrec, int j, double gamma, bool bar, double* l) {
  const V4<double> A = lmrec[2 * (size_t)j], B = lmrec[2 * (size_t)j + 1];
  l[0] = A.x + (bar ? gamma * A.w : 0.0);
  l[1] = A.y + (bar ? gamma * B.x : 0.0);
  l[2] = A.z + (bar ? gamma * B.y : 0.0);
}

// the block's scratch: per camera (C), the step dc, right-hand side rhs and the Cholesky
// diagonal diag (9 per camera), the Schur matrix S (row stride ld); in dynamic shared memory or
// in global memory. A block is solved by one CTA or by a cluster of `cs` CTAs (global scratch):
// rank, thread index in the cluster gt, threads in the cluster GT.
struct BlkWork {
  BlkCam* C;
  double *dc, *rhs, *diag, *S;
  int ld;
  int rank, cs, gt, GT;
};

// static shared memory of a block solve
struct BlkSmem {
  double red[BLK_THREADS];
  double val;
};

// a barrier of the CTA, or of the cluster (release and acquire at cluster scope: the global
// scratch written before it is seen after it by every CTA of the block)
__device__ __forceinline__ void blk_sync(const BlkWork& W) {
  if (W.cs > 1)
    cooperative_groups::this_cluster().sync();
  else
    __syncthreads();
}

// sum over the block's threads: each CTA in thread order (thread 0 adds the 128 partials), then
// the CTAs' sums in rank order (read from each CTA's shared memory); the result on every thread
__device__ __forceinline__ double blk_reduce(BlkSmem& sh, const BlkWork& W, double v) {
  __syncthreads();
  sh.red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < BLK_THREADS; ++k) t += sh.red[k];
    sh.val = t;
  }
  if (W.cs == 1) {
    __syncthreads();
    return 0.0 + sh.val;
  }
  auto cl = cooperative_groups::this_cluster();
  cl.sync();
  double t = 0.0;
  for (int r = 0; r < W.cs; ++r) t += *cl.map_shared_rank(&sh.val, r);
  cl.sync();   // every CTA has read the sums before the next reduction writes them
  return t;
}

// One LM step of block b on E^alpha(. | z), z = x̄^k (bar) or x^k, from z: the cameras' solution
// to W.C[.].cs, the landmarks' to lsc + BL_L (both stay at z if no step is taken).
__device__ inline void blk_lm(const BlkArgs& A, int b, bool bar, double gamma, double xi, BlkSmem& sh,
                              const BlkWork& W) {
  const int tid = threadIdx.x, gt = W.gt, GT = W.GT;
  const int cp0 = A.cam_ptr[b], nc = A.cam_ptr[b + 1] - cp0;
  const int l0 = A.lm_ptr[b], l1 = A.lm_ptr[b + 1];
  const int np = 9 * nc, ld = W.ld;
  const int ao = bar ? LS_AB : LS_AK, bo = bar ? LS_BB : LS_BK;
  BlkCam* C = W.C;
  double* S = W.S;
  // ---- cameras: the model of their inter pairs and proximal term (a thread per camera)
  for (int c = gt; c < nc; c += GT) {
    BlkCam& bc = C[c];
    cam_lm_model(bar ? bc.stb : bc.stk, bc.cz, xi, bc.A, bc.g);
    bc.cs = bc.cz;
  }
  // ---- landmarks: their 3 x 3 block, gradient, couplings B = w Jc^T Jl and F at z of their
  //      intra pairs, and each pair's camera-side terms (summed per camera below)
  for (int e = l0 + gt; e < l1; e += GT) {
    const int j = A.lms[e];
    double* s = A.lsc + (size_t)j * BL_N;
    double lz[3];
    blk_lpos(A.lmrec, j, gamma, bar, lz);
    const double* sm = A.lm_sums + (size_t)j * LS_N;
    const double a2 = 2.0 * sm[ao];
    double Cm[6] = {a2 + xi, 0.0, a2 + xi, 0.0, 0.0, a2 + xi};
    double gl[3] = {2.0 * sm[bo], 2.0 * sm[bo + 1], 2.0 * sm[bo + 2]};
    double Fz = 0.0;
    for (int p = A.io_ptr[e]; p < A.io_ptr[e + 1]; ++p) {
      const double2 u = A.c_u[A.io_obs[p]];
      double f[3], Jc[3][9], Jl[3][3];
      blk_intra_jac(C[A.io_cam[p]].cz, lz, u.x, u.y, f, Jc, Jl);
      double rho, w;
      blk_rho_any(A.loss, A.L, f[0] * f[0] + f[1] * f[1] + f[2] * f[2], rho, w);
      Fz += 0.5 * rho;
      int q = 0;
      for (int r1 = 0; r1 < 3; ++r1)
        for (int c1 = 0; c1 <= r1; ++c1, ++q)
          Cm[q] += w * (Jl[0][r1] * Jl[0][c1] + Jl[1][r1] * Jl[1][c1] + Jl[2][r1] * Jl[2][c1]);
      for (int r1 = 0; r1 < 3; ++r1) gl[r1] += w * (Jl[0][r1] * f[0] + Jl[1][r1] * f[1] + Jl[2][r1] * f[2]);
      double* bi = A.isc + (size_t)p * BI_N;
      for (int i = 0; i < 9; ++i) {
        for (int k = 0; k < 3; ++k) bi[BI_B + 3 * i + k] = w * (Jc[0][i] * Jl[0][k] + Jc[1][i] * Jl[1][k] + Jc[2][i] * Jl[2][k]);
        for (int k = 0; k <= i; ++k)
          bi[BI_A + lt9(i, k)] = w * (Jc[0][i] * Jc[0][k] + Jc[1][i] * Jc[1][k] + Jc[2][i] * Jc[2][k]);
        bi[BI_GC + i] = w * (Jc[0][i] * f[0] + Jc[1][i] * f[1] + Jc[2][i] * f[2]);
      }
    }
    for (int k = 0; k < 6; ++k) s[BL_C + k] = Cm[k];
    for (int k = 0; k < 3; ++k) {
      s[BL_G + k] = gl[k];
      s[BL_L + k] = lz[k];
    }
    s[BL_FZ] = Fz;
  }
  blk_sync(W);
  // ---- each camera's intra pairs added to its model: a thread per (camera, model entry), the
  //      camera's pairs in order
  for (int it = gt; it < nc * 54; it += GT) {
    const int c = it / 54, en = it - 54 * c;
    double v = 0.0;
    for (int q = A.ci_ptr[cp0 + c]; q < A.ci_ptr[cp0 + c + 1]; ++q) v += A.isc[(size_t)A.ci_io[q] * BI_N + BI_A + en];
    if (en < 45)
      C[c].A[en] += v;
    else
      C[c].g[en - 45] += v;
  }
  blk_sync(W);
  double mu = LM_MU0;
  for (int tr = 0; tr < LM_TRIES; ++tr, mu *= 10.0) {
    // ---- damped landmark blocks: C^-1 and B C^-1 of every intra pair
    for (int e = l0 + gt; e < l1; e += GT) {
      double* s = A.lsc + (size_t)A.lms[e] * BL_N;
      double Cm[6];
      for (int k = 0; k < 6; ++k) Cm[k] = s[BL_C + k];
      Cm[0] *= 1.0 + mu;
      Cm[2] *= 1.0 + mu;
      Cm[5] *= 1.0 + mu;
      sym3_inv(Cm, s + BL_CI);
      for (int p = A.io_ptr[e]; p < A.io_ptr[e + 1]; ++p) {
        double* bi = A.isc + (size_t)p * BI_N;
        for (int i = 0; i < 9; ++i) sym3_mul(s + BL_CI, bi + BI_B + 3 * i, bi + BI_BC + 3 * i);
      }
    }
    blk_sync(W);
    // ---- Schur complement S = (A + mu diag A) - sum_j B_j C_j^-1 B_j^T (lower triangle): a
    //      thread per camera pair (a >= b) and row of camera a, over camera a's intra pairs in
    //      order; the landmark's pair with camera b is looked up in its list (ascending cameras)
    const int n_item = nc * (nc + 1) / 2 * 9;
    for (int it = gt; it < n_item; it += GT) {
      const int pi = it / 9, ra = it - 9 * pi;
      int ca = (int)((sqrt(8.0 * pi + 1.0) - 1.0) * 0.5);
      while ((ca + 1) * (ca + 2) / 2 <= pi) ++ca;
      while (ca * (ca + 1) / 2 > pi) --ca;
      const int cbb = pi - ca * (ca + 1) / 2;
      const int nrb = ca == cbb ? ra + 1 : 9;
      double v[9];
#pragma unroll
      for (int rb = 0; rb < 9; ++rb) v[rb] = (ca == cbb && rb <= ra) ? C[ca].A[lt9(ra, rb)] * (ra == rb ? 1.0 + mu : 1.0) : 0.0;
      for (int q = A.ci_ptr[cp0 + ca]; q < A.ci_ptr[cp0 + ca + 1]; ++q) {
        int pb = -1;
        if (ca == cbb) {
          pb = A.ci_io[q];
        } else {
          const int e = A.ci_e[q];
          for (int p = A.io_ptr[e]; p < A.io_ptr[e + 1]; ++p) {
            const int c = A.io_cam[p];
            if (c >= cbb) {
              if (c == cbb) pb = p;
              break;
            }
          }
        }
        if (pb < 0) continue;
        const double* x = A.isc + (size_t)A.ci_io[q] * BI_N + BI_BC + 3 * ra;
        const double x0 = x[0], x1 = x[1], x2 = x[2];
        const double* y = A.isc + (size_t)pb * BI_N + BI_B;
#pragma unroll
        for (int rb = 0; rb < 9; ++rb)
          if (rb < nrb) v[rb] -= x0 * y[3 * rb] + x1 * y[3 * rb + 1] + x2 * y[3 * rb + 2];
      }
      double* Sr = S + (size_t)(9 * ca + ra) * ld + 9 * cbb;
#pragma unroll
      for (int rb = 0; rb < 9; ++rb)
        if (rb < nrb) Sr[rb] = v[rb];
    }
    // ... and its right-hand side -g + sum_j B_j C_j^-1 g_j (a thread per row, camera a's intra pairs in order)
    for (int r = gt; r < np; r += GT) {
      const int ca = r / 9, ra = r - 9 * ca;
      double v = -C[ca].g[ra];
      for (int q = A.ci_ptr[cp0 + ca]; q < A.ci_ptr[cp0 + ca + 1]; ++q) {
        const double* gl = A.lsc + (size_t)A.ci_lm[q] * BL_N + BL_G;
        const double* x = A.isc + (size_t)A.ci_io[q] * BI_N + BI_BC + 3 * ra;
        v += x[0] * gl[0] + x[1] * gl[1] + x[2] * gl[2];
      }
      W.rhs[r] = v;
    }
    blk_sync(W);
    // ---- Cholesky of S in place (column by column: every thread takes the pivot, the column is
    //      scaled, the trailing update a warp per row with its lanes along the row; the pivots'
    //      square roots go to diag, so S[k][k] is only read); a non-positive pivot fails the trial
    const int gw = (gt >> 5), GW = GT >> 5, lane = tid & 31;
    bool ok = true;
    for (int k = 0; k < np; ++k) {
      const double d = S[(size_t)k * ld + k];
      ok = ok && d > 0.0;
      const double dk = sqrt(d > 0.0 ? d : 1.0);
      if (gt == 0) W.diag[k] = dk;
      for (int i = k + 1 + gt; i < np; i += GT) S[(size_t)i * ld + k] /= dk;
      blk_sync(W);
      for (int i = k + 1 + gw; i < np; i += GW) {
        double* Si = S + (size_t)i * ld;
        const double lik = Si[k];
        for (int jj = k + 1 + lane; jj <= i; jj += 32) Si[jj] -= lik * S[(size_t)jj * ld + k];
      }
      blk_sync(W);
    }
    if (!ok) continue;
    // L y = rhs (y to dc), then L^T x = y (x to rhs), then x to dc; column-oriented, by the
    // block's first CTA
    if (W.rank == 0) {
      for (int k = 0; k < np; ++k) {
        const double yk = W.rhs[k] / W.diag[k];
        for (int i = k + 1 + tid; i < np; i += BLK_THREADS) W.rhs[i] -= S[(size_t)i * ld + k] * yk;
        if (tid == 0) W.dc[k] = yk;
        __syncthreads();
      }
      for (int i = np - 1; i >= 0; --i) {
        const double xv = W.dc[i] / W.diag[i];
        const double* Si = S + (size_t)i * ld;
        for (int k = tid; k < i; k += BLK_THREADS) W.dc[k] -= Si[k] * xv;
        if (tid == 0) W.rhs[i] = xv;
        __syncthreads();
      }
      for (int r = tid; r < np; r += BLK_THREADS) W.dc[r] = W.rhs[r];
    }
    blk_sync(W);
    // ---- the candidate: cameras (a thread each), landmarks by back substitution, and the
    //      decrease of E^alpha(. | z) term by term
    double part = 0.0;
    for (int c = gt; c < nc; c += GT) {
      BlkCam& bc = C[c];
      const CamT<double>& cz = bc.cz;
      const double* th = W.dc + 9 * c;
      double Ex[9];
      rodrigues(th, Ex);
      CamT<double> cc;
      for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k)
          cc.R[r * 3 + k] = cz.R[r * 3 + 0] * Ex[0 * 3 + k] + cz.R[r * 3 + 1] * Ex[1 * 3 + k] + cz.R[r * 3 + 2] * Ex[2 * 3 + k];
      for (int k = 0; k < 3; ++k) {
        cc.t[k] = cz.t[k] + th[3 + k];
        cc.d[k] = cz.d[k] + th[6 + k];
      }
      part += cam_phi(bar ? bc.stb : bc.stk, cz, cc, xi);   // inter pairs' P and the proximal term
      bc.cb = cc;   // candidate (cs keeps the accepted solution)
    }
    blk_sync(W);
    for (int e = l0 + gt; e < l1; e += GT) {
      const int j = A.lms[e];
      const double* s = A.lsc + (size_t)j * BL_N;
      double rr[3] = {s[BL_G], s[BL_G + 1], s[BL_G + 2]};
      for (int p = A.io_ptr[e]; p < A.io_ptr[e + 1]; ++p) {
        const double* bi = A.isc + (size_t)p * BI_N + BI_B;
        const double* th = W.dc + 9 * A.io_cam[p];
        for (int k = 0; k < 3; ++k)
          for (int i = 0; i < 9; ++i) rr[k] += bi[3 * i + k] * th[i];
      }
      double dl[3];
      sym3_mul(s + BL_CI, rr, dl);
      double lz[3];
      blk_lpos(A.lmrec, j, gamma, bar, lz);
      const double* sm = A.lm_sums + (size_t)j * LS_N;
      const double dd = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
      part += sm[ao] * dd - 2.0 * (dl[0] * sm[bo] + dl[1] * sm[bo + 1] + dl[2] * sm[bo + 2]) + 0.5 * xi * dd;
      const double lc[3] = {lz[0] - dl[0], lz[1] - dl[1], lz[2] - dl[2]};
      double Fc = 0.0;
      for (int p = A.io_ptr[e]; p < A.io_ptr[e + 1]; ++p) {
        const double2 u = A.c_u[A.io_obs[p]];
        Fc += blk_F(C[A.io_cam[p]].cb, lc, u.x, u.y, A.L, A.loss);
      }
      part += Fc - s[BL_FZ];
    }
    const double dE = blk_reduce(sh, W, part);
    if (dE < 0.0) {   // the step is taken
      for (int e = l0 + gt; e < l1; e += GT) {
        double* s = A.lsc + (size_t)A.lms[e] * BL_N;
        double rr[3] = {s[BL_G], s[BL_G + 1], s[BL_G + 2]};
        for (int p = A.io_ptr[e]; p < A.io_ptr[e + 1]; ++p) {
          const double* bi = A.isc + (size_t)p * BI_N + BI_B;
          const double* th = W.dc + 9 * A.io_cam[p];
          for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 9; ++i) rr[k] += bi[3 * i + k] * th[i];
        }
        double dl[3];
        sym3_mul(s + BL_CI, rr, dl);
        s[BL_L + 0] -= dl[0];
        s[BL_L + 1] -= dl[1];
        s[BL_L + 2] -= dl[2];
      }
      for (int c = gt; c < nc; c += GT) C[c].cs = C[c].cb;
      blk_sync(W);
      return;
    }
  }
  blk_sync(W);
}

// E^alpha(x | x^k) - E^alpha(x^k | x^k) of block b for the solution in C[.].cs and lsc + BL_L
__device__ inline double blk_dE_k(const BlkArgs& A, int b, double xi, BlkSmem& sh, const BlkWork& W) {
  const int gt = W.gt, GT = W.GT;
  const int cp0 = A.cam_ptr[b], nc = A.cam_ptr[b + 1] - cp0;
  const int l0 = A.lm_ptr[b], l1 = A.lm_ptr[b + 1];
  const BlkCam* C = W.C;
  double part = 0.0;
  for (int c = gt; c < nc; c += GT) part += cam_phi(C[c].stk, C[c].ck, C[c].cs, xi);
  for (int e = l0 + gt; e < l1; e += GT) {
    const int j = A.lms[e];
    const double* s = A.lsc + (size_t)j * BL_N;
    double lk[3];
    blk_lpos(A.lmrec, j, 0.0, false, lk);
    const double dl[3] = {s[BL_L] - lk[0], s[BL_L + 1] - lk[1], s[BL_L + 2] - lk[2]};
    const double* sm = A.lm_sums + (size_t)j * LS_N;
    const double dd = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
    part += sm[LS_AK] * dd + 2.0 * (dl[0] * sm[LS_BK] + dl[1] * sm[LS_BK + 1] + dl[2] * sm[LS_BK + 2]) + 0.5 * xi * dd;
    for (int p = A.io_ptr[e]; p < A.io_ptr[e + 1]; ++p) {
      const double2 u = A.c_u[A.io_obs[p]];
      const int c = A.io_cam[p];
      part += blk_F(C[c].cs, s + BL_L, u.x, u.y, A.L, A.loss) - blk_F(C[c].ck, lk, u.x, u.y, A.L, A.loss);
    }
  }
  return blk_reduce(sh, W, part);
}

__global__ void __launch_bounds__(BLK_THREADS) k_blk_solve(BlkArgs A, IterParams P) {
  extern __shared__ __align__(16) double blk_dyn[];   // the block scratch (ld > 0)
  __shared__ BlkSmem sh;
  const int cs = (int)cooperative_groups::this_cluster().num_blocks();
  const int b = blockIdx.x / cs;   // a block per cluster of cs CTAs (cs = 1: a CTA per block)
  const int tid = threadIdx.x;
  const int it = *P.it, first = *P.first;
  const double gamma = P.gam[it], xi = P.xi;
  const int cp0 = A.cam_ptr[b], nc = A.cam_ptr[b + 1] - cp0;
  const int l0 = A.lm_ptr[b], l1 = A.lm_ptr[b + 1];
  BlkWork W;
  W.cs = cs;
  W.rank = (int)(blockIdx.x - (unsigned)b * cs);
  W.gt = W.rank * BLK_THREADS + tid;
  W.GT = cs * BLK_THREADS;
  if (A.ld > 0) {   // shared memory (cs = 1): per camera scratch of the most cameras, dc, rhs, diag, then S
    const int mc = A.ld / 9;
    W.C = reinterpret_cast<BlkCam*>(blk_dyn);
    W.dc = blk_dyn + (size_t)mc * (sizeof(BlkCam) / 8);
    W.rhs = W.dc + A.ld;
    W.diag = W.rhs + A.ld;
    W.S = W.diag + A.ld;
    W.ld = A.ld;
  } else {   // global memory at the block's camera entries and Schur offset
    W.C = A.g_cam + cp0;
    W.dc = A.g_vec + (size_t)27 * cp0;
    W.rhs = W.dc + 9 * nc;
    W.diag = W.rhs + 9 * nc;
    W.S = A.g_S + A.g_soff[b];
    W.ld = 9 * nc;
  }
  const int gt = W.gt, GT = W.GT;
  BlkCam* C = W.C;
  // ---- cameras: x^k, x̄^k, statistics, F sums, displacement (a thread each)
  double part_disp = 0.0, part_Fall = 0.0, part_Fin = 0.0, part_G = 0.0;
  for (int c = gt; c < nc; c += GT) {
    const int cam = A.cams[cp0 + c];
    double pF = 0.0;
    const double* x = A.cam_x + (size_t)cam * CSTRIDE;
    const double* dx = A.cam_dx + (size_t)cam * CSTRIDE;
    CamT<double> ck, cb;
    for (int a = 0; a < 9; ++a) {
      ck.R[a] = x[CS_R + a];
      cb.R[a] = A.cam_Rbar[(size_t)cam * 9 + a];
      part_disp += dx[CS_R + a] * dx[CS_R + a];
    }
    for (int a = 0; a < 3; ++a) {
      ck.t[a] = x[CS_T + a];
      ck.d[a] = x[CS_D + a];
      cb.t[a] = ck.t[a] + gamma * dx[CS_T + a];
      cb.d[a] = ck.d[a] + gamma * dx[CS_D + a];
      part_disp += dx[CS_T + a] * dx[CS_T + a] + dx[CS_D + a] * dx[CS_D + a];
    }
    C[c].ck = ck;
    C[c].cz = cb;   // the accelerated step's conditioning iterate, first
    const int c0 = A.cam_chunk_ptr[cam], c1 = A.cam_chunk_ptr[cam + 1];
    sum_stats<double, double>(A.part, c0, c1, PART_XB, C[c].stb);
    sum_stats<double, double>(A.part, c0, c1, PART_XK, C[c].stk);
    for (int q = c0; q < c1; ++q) {
      pF += A.part[(size_t)q * CP_STRIDE + PART_F];
      part_G += A.part[(size_t)q * CP_STRIDE + PART_G];
      part_Fin += A.part[(size_t)q * CP_STRIDE + PART_FI];
    }
    part_Fall += pF;
    A.cam_Fsum[cam] = pF;   // F_ij(x^k) of the camera's observations (objective trace)
  }
  // ---- landmarks: displacement, gaps and inter F sums
  double part_dl = 0.0, part_Gl = 0.0, part_Fl = 0.0;
  for (int e = l0 + gt; e < l1; e += GT) {
    const int j = A.lms[e];
    const V4<double> LA = A.lmrec[2 * (size_t)j], LB = A.lmrec[2 * (size_t)j + 1];
    part_dl += LA.w * LA.w + LB.x * LB.x + LB.y * LB.y;
    part_Gl += A.lm_sums[(size_t)j * LS_N + LS_G];
    part_Fl += A.lm_sums[(size_t)j * LS_N + LS_F];
  }
  const double disp = blk_reduce(sh, W, part_disp) + blk_reduce(sh, W, part_dl);
  const double Fall = blk_reduce(sh, W, part_Fall), Fin = blk_reduce(sh, W, part_Fin);
  const double G = blk_reduce(sh, W, part_G) + blk_reduce(sh, W, part_Gl);
  const double Fl = blk_reduce(sh, W, part_Fl);
  // Eq. DEalpha, Eq. Fainit, Eq. Fak, Eq. lFak, with E^alpha(x^k | x^k) = sum_E' F + (1/2) sum_E'' F
  const double E0 = Fin + 0.5 * (Fall - Fin) + 0.5 * Fl;
  const double dE = -0.5 * xi * disp + 0.5 * G;
  const double E = first ? E0 : A.blk_E[b];
  const double Fb_prev = first ? E0 : A.blk_Fbar[b];
  const double F = E + dE;
  const double Fbar = (1.0 - P.eta) * Fb_prev + P.eta * F;
  // ---- accelerated step from x̄^k, restart test (Eq. Eak, strict), MM step from x^k where it fires
  bool rs = true;
  double Enext = 0.0;
  if (A.pass == 2) {   // global restart, decided: the MM step in every block, or the kept step
    rs = *P.g_fire != 0;
    if (!rs) {
      for (int c = gt; c < nc; c += GT)
        C[c].cs = *reinterpret_cast<const CamT<double>*>(P.cam_alt + (size_t)A.cams[cp0 + c] * 32);
      Enext = A.blk_Ealt[b];
      blk_sync(W);
    }
  } else if (P.accelerated) {
    blk_lm(A, b, true, gamma, xi, sh, W);
    Enext = F + blk_dE_k(A, b, xi, sh, W);
    if (A.pass == 1) {   // global restart: keep the accelerated step and the block's test term
      for (int c = gt; c < nc; c += GT)
        *reinterpret_cast<CamT<double>*>(P.cam_alt + (size_t)A.cams[cp0 + c] * 32) = C[c].cs;
      if (gt == 0) {
        A.blk_g[b] = Enext - Fbar;
        A.blk_Ealt[b] = Enext;
      }
      return;
    }
    rs = Enext > Fbar;
  }
  if (rs) {
    for (int c = gt; c < nc; c += GT) C[c].cz = C[c].ck;
    blk_sync(W);
    blk_lm(A, b, false, gamma, xi, sh, W);
    Enext = F + blk_dE_k(A, b, xi, sh, W);
  }
  // ---- new state
  for (int e = l0 + gt; e < l1; e += GT) {
    const int j = A.lms[e];
    const double* s = A.lsc + (size_t)j * BL_N;
    const V4<double> LA = A.lmrec[2 * (size_t)j];
    V4<double> nA, nB;
    nA.x = s[BL_L];
    nA.y = s[BL_L + 1];
    nA.z = s[BL_L + 2];
    nA.w = s[BL_L] - LA.x;
    nB.x = s[BL_L + 1] - LA.y;
    nB.y = s[BL_L + 2] - LA.z;
    nB.z = 0.0;
    nB.w = 0.0;
    A.lmrec_out[2 * (size_t)j] = nA;
    A.lmrec_out[2 * (size_t)j + 1] = nB;
  }
  if (gt == 0) {
    A.blk_E[b] = Enext;
    A.blk_Fbar[b] = Fbar;
    A.blk_F[b] = F;
    A.blk_rs[b] = (rs && P.accelerated) ? 1 : 0;
  }
  for (int c = gt; c < nc; c += GT) {
    const int cam = A.cams[cp0 + c];
    const CamT<double>& cs = C[c].cs;
    const CamT<double>& ck = C[c].ck;
    double* x = A.cam_x + (size_t)cam * CSTRIDE;
    double* dx = A.cam_dx + (size_t)cam * CSTRIDE;
    A.cam_rs[cam] = (c == 0 && rs && P.accelerated) ? 1 : 0;   // the block's restart, counted once
    CamT<double> ndx;
    for (int a = 0; a < 9; ++a) {
      ndx.R[a] = cs.R[a] - ck.R[a];
      x[CS_R + a] = cs.R[a];
      dx[CS_R + a] = ndx.R[a];
    }
    for (int a = 0; a < 3; ++a) {
      ndx.t[a] = cs.t[a] - ck.t[a];
      ndx.d[a] = cs.d[a] - ck.d[a];
      x[CS_T + a] = cs.t[a];
      dx[CS_T + a] = ndx.t[a];
      x[CS_D + a] = cs.d[a];
      dx[CS_D + a] = ndx.d[a];
    }
    // the next extrapolation; after a global restart with the momentum reset s^(k+1) = 1, so
    // gamma^(k+1) = 0 (the reduction sets the table to the same after this kernel)
    const double gn = (A.pass == 2 && rs && P.reset_s) ? 0.0 : P.gam[it + 1];
    double K[9], Rb[9];
    for (int a = 0; a < 9; ++a) K[a] = cs.R[a] + gn * ndx.R[a];
    extrap_rotation<double>(K, Rb);
    for (int a = 0; a < 9; ++a) A.cam_Rbar[(size_t)cam * 9 + a] = Rb[a];
    write_pack_t<double>(cs, ndx, Rb, A.pack_next + (size_t)cam * P4N);
  }
}

// The global restart's test over the blocks (Algorithm 1 for the one block made of all): the sum
// of E(k+1) - Fbar(k) over the blocks in a fixed order (lane l takes blocks l, l + 32, ..., then a
// shuffle tree) and the decision.
__global__ void k_blk_fire(int S, const double* __restrict__ blk_g, int* __restrict__ g_fire) {
  double g = 0.0;
  for (int b = threadIdx.x; b < S; b += 32) g += blk_g[b];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) g += __shfl_xor_sync(0xffffffffu, g, off);
  if (threadIdx.x == 0) *g_fire = g > 0.0 ? 1 : 0;
}

}  // namespace daba
