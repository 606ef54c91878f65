// daba_kernels.cuh -- the kernels of one DABA iteration (Algorithm 1, arXiv 2305.07026)
// with one block per camera and one block per landmark.
//
// Per iteration k:
//   1. cpass     (warp/chunk) : camera-sorted observations; evaluates each observation at
//                               x^k, xbar^k and x^(k-1) once, reduces the camera's centred
//                               majorizer statistics (one partial per chunk) and stores the
//                               observation's landmark-side terms as a record in camera order.
//   2. lpass     (CTA/tile)   : per landmark, sums its records and runs the restart metrics,
//                               accelerated solve, restart test and MM re-solve (closed form);
//                               writes the other landmark buffer.
//   3. camsolve  (2 warps per 32 cameras): FP64 camera block solves, the accelerated and the
//                               MM solve side by side, restart test, and the extrapolated
//                               rotation and pack of iteration k+1.
//   4. finalize  (grid)       : F(x^k) trace entry and restart count (deterministic order).
// lpass and camsolve both only need cpass, so they run concurrently (camsolve, the
// latency-bound FP64 path, on the higher-priority stream). Kernel launch order and the
// streams are set by the host runtime (daba_abi.cu).
// cam_prepare builds the pack of the first iteration of a run.
//
// Centred statistics. For a conditioning iterate z (xbar^k or x^k) and a camera c let
// M(c) = [R e1, R e2, d1 R e3, d2 R e3, d3 R e3, t] (3x6) and h = (u1, u2, 1, s, s^2,
// lambda_z) so that R p(d) + lambda_z t = M(c) h. With r0 = R_z p_z + lambda_z t_z - g_z
// = R_z e_z / 2 (from Eq. g) the camera part of the surrogate is, exactly,
//   sum_j P_ij(c|z) = tr(dM H dM^T) + 2 tr(dM B) + const,  dM = M(c) - M(c_z),
//   H = sum_j w h h^T (6x6),  B = sum_j w h r0^T (6x3),
// and for a landmark, with r0' = lambda_z l_z - g_z = -R_z e_z / 2,
//   sum_i Q_ij(l|z) = (sum w lambda^2) |dl|^2 + 2 dl . (sum w lambda r0') + const.
// Both are evaluated relative to the conditioning point, so surrogate differences never
// cancel O(1) quantities.
#pragma once

#include "daba_device.cuh"

namespace daba {

// ---- camera-pass accumulators (registers): Hbar[21] Bbar[18] H[21] B[18] sumF sumGap
enum { CP_HB = 0, CP_BB = 21, CP_H = 39, CP_B = 60, CP_F = 78, CP_G = 79, CP_NACC = 80 };
// ---- chunk partial in memory (pass precision), each statistics set padded to 40 so that
//      it starts on a 16-byte boundary: [Hbar Bbar pad] [H B pad] sumF sumGap pad pad
enum { PART_XB = 0, PART_XK = 40, PART_F = 80, PART_G = 81, PART_FI = 82, CP_STRIDE = 84 };
// (PART_FI: with coarse blocks, the F_ij sum of the chunk's intra-block pairs)
__host__ __device__ constexpr int part_slot(int k) { return k < 39 ? k : (k < 78 ? k + 1 : k + 2); }
// ---- tile partial layout (doubles): sumF restarts pad pad
enum { TP_F = 0, TP_RS = 1, TP_STRIDE = 4 };
// ---- landmark record (two V4): (l[3], delta0) (delta1, delta2, S, E), with l the high part
//      in MIXED, delta = l^k - l^(k-1), S = Fbar^(k-1) - E^(k) the restart slack and E^(k)
//      kept by the FP64 path only; MIXED keeps the low part of l in a separate V4 array.
// ---- camera state (doubles, stride 16): R[9] t[3] d[3] pad
enum { CS_R = 0, CS_T = 9, CS_D = 12, CSTRIDE = 16 };

constexpr int CPASS_WARPS = 1;   // one warp per CTA: 12 resident warps per SM at 156 registers
constexpr int CAMSOLVE_THREADS = 64;   // one camera per active thread
constexpr int LPASS_THREADS = 128;
constexpr int LPASS_UNROLL = 4;   // observations whose records a thread loads before storing any
constexpr int TILE_OBS = 512;     // observations of a small landmark tile
constexpr int TILE_LMS = 128;     // landmarks of a small landmark tile
constexpr int BIG_TILE_OBS = 2048;   // a landmark with more observations gets a tile of its own (max track)
constexpr int MAX_TRACK = BIG_TILE_OBS;

struct IterParams {
  const double* gam;   // gamma^(k) per iteration of the current run segment (+1 look-ahead)
  int* it;             // device iteration counter within the segment
  int* first;          // 1 on the first iteration after the state was set
  double xi, eta;
  double eta1, hxi;    // 1 - eta and xi / 2
  float eta1f, hxif;   // the same in FP32 (no FP64 instruction in the FP32 passes)
  int accelerated;
  int n_alt;
  int* flag;           // error bits: 1 non-finite objective, 2 a bounded wait ran out
  long long wait_ns;   // limit of the landmark pass's first wait on its tile copies (ns)
  // global restart variant (restart_global = 1): one test on the sums of the block metrics.
  // The block kernels take the accelerated update and keep the MM alternative; the reduction
  // decides; the fix-up kernels apply the MM alternative everywhere if the test fired.
  int restart_global;
  int reset_s;         // with restart_global: s <- 1 after a restart (gamma table continued on the device)
  double* g_cam;       // per camera: E(k+1) - Fbar(k) of its accelerated update
  double* g_tile;      // per landmark tile: the sum of the same over its landmarks
  double* cam_alt;     // per camera (32 doubles): MM alternative R t d, its dx, E(k+1), S(k+1)
  int* g_fire;         // 1 if the global test fired in the current iteration
  double* s_dev;       // Nesterov s^(k) on the device (reset_s)
  int fire_given;      // the reduction takes g_fire as decided (coarse blocks) instead of testing
};

template <class Real>
__device__ __forceinline__ Real eta1_of(const IterParams& P);
template <>
__device__ __forceinline__ float eta1_of<float>(const IterParams& P) { return P.eta1f; }
template <>
__device__ __forceinline__ double eta1_of<double>(const IterParams& P) { return P.eta1; }
template <class Real>
__device__ __forceinline__ Real hxi_of(const IterParams& P);
template <>
__device__ __forceinline__ float hxi_of<float>(const IterParams& P) { return P.hxif; }
template <>
__device__ __forceinline__ double hxi_of<double>(const IterParams& P) { return P.hxi; }

__device__ __forceinline__ int tri6(int a, int b) { return a * 6 - (a * (a - 1)) / 2 + (b - a); }

// ---------------------------------------------------------------------------
// 1. camera-sorted pass: one warp per chunk (<= chunk size observations of one camera)
// ---------------------------------------------------------------------------
template <class Real>
__device__ __forceinline__ void accumulate_cam(Real* acc, const ObsEval<Real>& ev, Real u0, Real u1) {
  const Real s = u0 * u0 + u1 * u1;
  Real h[6] = {u0, u1, Real(1), s, s * s, ev.lamb};
  {  // xbar statistics: Hbar += wb h h^T, Bbar += wb h (R e)^T / 2
    Real wh[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) wh[a] = ev.wb * h[a];
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int c = a; c < 6; ++c) acc[CP_HB + tri6(a, c)] += wh[a] * h[c];
    const Real r0[3] = {Real(0.5) * ev.Reb0, Real(0.5) * ev.Reb1, Real(0.5) * ev.Reb2};
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[CP_BB + a * 3 + c] += wh[a] * r0[c];
  }
  h[5] = ev.lam;
  {  // x^k statistics
    Real wh[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) wh[a] = ev.w * h[a];
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int c = a; c < 6; ++c) acc[CP_H + tri6(a, c)] += wh[a] * h[c];
    const Real r0[3] = {Real(0.5) * ev.Re0, Real(0.5) * ev.Re1, Real(0.5) * ev.Re2};
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[CP_B + a * 3 + c] += wh[a] * r0[c];
  }
  acc[CP_F] += Real(0.5) * ev.rho;
  acc[CP_G] += ev.gap;
}

// Per-lane camera statistics of the camera pass and their chunk reduction. FP64: the 80
// accumulators in CP_* order. FP32: the x̄^k and x^k statistics side by side as float2 pairs
// (x: x̄^k, y: x^k), accumulated with the packed FP32 instructions of sm_100+ (__ffma2_rn and
// friends; per component the same rounding as the scalar FMA), so one instruction serves both
// sets. Both store the chunk partial in the layout of PART_*.
template <class Real>
struct CamAcc {
  Real a[CP_NACC];
  Real fi;   // coarse blocks: F_ij of the intra-block pairs
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < CP_NACC; ++k) a[k] = Real(0);
    fi = Real(0);
  }
  __device__ __forceinline__ void add(const ObsEval<Real>& ev, Real u0, Real u1) { accumulate_cam<Real>(a, ev, u0, u1); }
  __device__ __forceinline__ void add_intra(Real F) {
    a[CP_F] += F;
    fi += F;
  }
  __device__ __forceinline__ void reduce_store(int lane, Real* out, bool with_fi = false) {
#pragma unroll
    for (int k = 0; k < CP_NACC; ++k) {
      Real v = a[k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      a[k] = v;
    }
    if (with_fi) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) fi += __shfl_xor_sync(0xffffffffu, fi, off);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < CP_NACC; ++k) out[part_slot(k)] = a[k];
      out[39] = out[79] = out[83] = Real(0);
      out[PART_FI] = with_fi ? fi : Real(0);
    }
  }
};

template <>
struct CamAcc<float> {
  float2 s[39];   // H (21, packed) then B (18); x: at x̄^k, y: at x^k
  float f, g;     // sum F_ij / 2 and the surrogate gap
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < 39; ++k) s[k] = make_float2(0.f, 0.f);
    f = g = 0.f;
  }
  __device__ __forceinline__ void add(const ObsEval<float>& ev, float u0, float u1) {
    const float sq = u0 * u0 + u1 * u1;
    const float h[5] = {u0, u1, 1.f, sq, sq * sq};
    const float2 wv = make_float2(ev.wb, ev.w);
    float2 wh[6], hc[6];
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      hc[a] = make_float2(h[a], h[a]);
      wh[a] = __fmul2_rn(wv, hc[a]);
    }
    hc[5] = make_float2(ev.lamb, ev.lam);
    wh[5] = __fmul2_rn(wv, hc[5]);
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int c = a; c < 6; ++c) s[tri6(a, c)] = __ffma2_rn(wh[a], hc[c], s[tri6(a, c)]);
    const float2 half = make_float2(0.5f, 0.5f);
    const float2 r0[3] = {__fmul2_rn(half, make_float2(ev.Reb0, ev.Re0)), __fmul2_rn(half, make_float2(ev.Reb1, ev.Re1)),
                          __fmul2_rn(half, make_float2(ev.Reb2, ev.Re2))};
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) s[21 + a * 3 + c] = __ffma2_rn(wh[a], r0[c], s[21 + a * 3 + c]);
    f += 0.5f * ev.rho;
    g += ev.gap;
  }
  // Warp reduction of the 40 pairs (the 39 statistics and (f, g)) as a reduce-scatter:
  // over the lane offsets 16, 8 and 4 each lane keeps half of its pairs and adds its partner's
  // copy of them, then offsets 2 and 1 add the last five pairs across the group of four lanes.
  // Each addition pairs the same lanes, in the same order, as a plain butterfly reduction of
  // every pair, so the sums are the same bits; it takes about 300 instead of 700
  // warp-instructions and 10 stores from 8 lanes instead of 84 from lane 0.
  __device__ __forceinline__ void reduce_store(int lane, float* out) {
    float2 u[40];
#pragma unroll
    for (int k = 0; k < 39; ++k) u[k] = s[k];
    u[39] = make_float2(f, g);
    int base = 0;   // first pair index held by this lane after the scatter levels
#pragma unroll
    for (int half = 20, off = 16; half >= 5; half >>= 1, off >>= 1) {
      const bool up = (lane & off) != 0;
      if (up) base += half;
#pragma unroll
      for (int i = 0; i < half; ++i) {
        const float2 keep = up ? u[i + half] : u[i];
        float2 send = up ? u[i] : u[i + half];
        send.x = __shfl_xor_sync(0xffffffffu, send.x, off);
        send.y = __shfl_xor_sync(0xffffffffu, send.y, off);
        u[i] = __fadd2_rn(keep, send);
      }
    }
#pragma unroll
    for (int off = 2; off > 0; off >>= 1)
#pragma unroll
      for (int i = 0; i < 5; ++i)
        u[i] = __fadd2_rn(u[i], make_float2(__shfl_xor_sync(0xffffffffu, u[i].x, off),
                                            __shfl_xor_sync(0xffffffffu, u[i].y, off)));
    if ((lane & 3) == 0) {
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        const int k = base + i;
        if (k < 39) {
          out[PART_XB + k] = u[i].x;
          out[PART_XK + k] = u[i].y;
        } else {
          out[PART_F] = u[i].x;
          out[PART_G] = u[i].y;
          out[39] = out[79] = out[82] = out[83] = 0.f;
        }
      }
    }
  }
};

// asynchronous global -> shared copies (cp.async) used to stage gathered records
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int CPASS_STAGES = 4;   // batches of 32 observations in the ring per warp (two per step)

// Third landmark-side record of an observation: FP64 path (F_ij(x^k), surrogate gap); MIXED
// the gap only (F_ij only enters the FP64 path's per-landmark diagnostics).
template <class Real>
struct RecC;
template <>
struct RecC<float> {
  using type = float;
  static __device__ __forceinline__ float make(float, float gap) { return gap; }
  static __device__ __forceinline__ float F(float) { return 0.f; }
  static __device__ __forceinline__ float gap(float c) { return c; }
};
template <>
struct RecC<double> {
  using type = double2;
  static __device__ __forceinline__ double2 make(double f, double gap) { return make_double2(f, gap); }
  static __device__ __forceinline__ double F(double2 c) { return c.x; }
  static __device__ __forceinline__ double gap(double2 c) { return c.y; }
};

// Per lane and stage: the landmark record (two V4); the pixel and the record position are kept
// in arrays of their own (consecutive lanes in consecutive words, no bank conflicts).
template <class Real, class Real2>
struct CpassStage {
  V4<Real> rec[2];
  Real pad[2];   // 48 B per lane in FP32: eight lanes' 16 B copies fall in distinct banks
};

// Landmark-side record of one observation, stored at c_rpos[o], its position in the landmark
// tiles' processing order (so that the landmark pass streams the records sequentially):
//   rec_a = (wb lamb^2, -wb lamb (Rbar ebar) / 2)   terms of sum_i Q_ij(l | xbar^k)
//   rec_b = (w lam^2, -w lam (R e) / 2)             terms of sum_i Q_ij(l | x^k)
//   rec_c = (F_ij(x^k), surrogate gap), MIXED the gap only (RecC)
// Shared memory of one camera-pass warp: the camera pack, and the staging ring of the landmark
// records, pixels and record positions.
template <class Real, class Real2>
struct CpassWarpSmem {
  V4<Real> pk[P4N];
  CpassStage<Real, Real2> sbuf[CPASS_STAGES][32];
  Real2 su[CPASS_STAGES][32];
  int srp[CPASS_STAGES][32];
};

// Loads of data that the same launch wrote earlier (COH: the persistent kernel, whose phases
// follow one another inside one launch) go to L2 (ld.global.cg), past the SM's incoherent L1
// and read-only caches; the kernels of the graph path read them with plain loads.
template <bool COH, class T>
__device__ __forceinline__ T ld_mut(const T* p) {
  if constexpr (COH) {
    if constexpr (sizeof(T) == 16) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
      T r;
      memcpy(&r, &v, 16);
      return r;
    } else if constexpr (sizeof(T) == 32) {
      const double2 a = __ldcg(reinterpret_cast<const double2*>(p)), b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
      T r;
      memcpy(&r, &a, 16);
      memcpy(reinterpret_cast<char*>(&r) + 16, &b, 16);
      return r;
    } else {
      return __ldcg(p);
    }
  } else {
    return *p;
  }
}

// One chunk of the camera-sorted pass (camera chunk_cam[warp], observations chunk_beg[warp] ..
// chunk_beg[warp + 1]) by one warp; gamma of Eq. nesterov_x for this iteration.
template <int LOSS, class Real, class Real2, bool COH, bool BLK = false>
__device__ __forceinline__ void cpass_chunk(int warp, int lane, CpassWarpSmem<Real, Real2>& sm, Real gamma,
                                            const int* __restrict__ chunk_cam, const int* __restrict__ chunk_beg,
                                            const int* __restrict__ c_lm, const Real2* __restrict__ c_u,
                                            const V4<Real>* __restrict__ pack, const V4<Real>* __restrict__ lmrec,
                                            const LossC<Real>& L, Real* __restrict__ part,
                                            const int* __restrict__ c_rpos, V4<Real>* __restrict__ rec_a,
                                            V4<Real>* __restrict__ rec_b, typename RecC<Real>::type* __restrict__ rec_c,
                                            const uint8_t* __restrict__ c_intra = nullptr) {
  const int cam = chunk_cam[warp];
  const int b = chunk_beg[warp], e = chunk_beg[warp + 1];
  if (lane < P4N) sm.pk[lane] = ld_mut<COH>(pack + (size_t)cam * P4N + lane);
  __syncwarp();
  const V4<Real>* pk = sm.pk;
  CamAcc<Real> acc;
  acc.zero();
  // Pipeline over batches t of 32 observations (one per lane) in a ring of four: the landmark
  // records, pixels and record positions of the next two batches are copied asynchronously
  // (their landmark indices loaded a step earlier) while two batches are evaluated. Each lane
  // only touches its own staging slots.
  const int nb = (e - b + 31) >> 5;
  CpassStage<Real, Real2>(*stg)[32] = sm.sbuf;
  auto issue = [&](int t, int j) {
    const int o = b + 32 * t + lane;
    if (o < e) {
      CpassStage<Real, Real2>& d = stg[t % CPASS_STAGES][lane];
      const V4<Real>* src = lmrec + 2 * (size_t)j;
#pragma unroll
      for (int q = 0; q < (int)(2 * sizeof(V4<Real>) / 16); ++q)
        cp_async16(reinterpret_cast<char*>(d.rec) + 16 * q, reinterpret_cast<const char*>(src) + 16 * q);
      if (sizeof(Real2) == 16)
        cp_async16(&sm.su[t % CPASS_STAGES][lane], c_u + o);
      else
        cp_async8(&sm.su[t % CPASS_STAGES][lane], c_u + o);
      cp_async4(&sm.srp[t % CPASS_STAGES][lane], c_rpos + o);
    }
    cp_async_commit();
  };
  auto index_of = [&](int t) -> int {
    const int o = b + 32 * t + lane;
    return o < e ? c_lm[o] : 0;
  };
  auto process = [&](int t) {
    const int o = b + 32 * t + lane;
    if (o < e) {
      const CpassStage<Real, Real2>& d = stg[t % CPASS_STAGES][lane];
      const V4<Real> r0 = d.rec[0], r1 = d.rec[1];
      const Real2 uu = sm.su[t % CPASS_STAGES][lane];
      ObsEval<Real> ev;
      eval_obs<LOSS, Real>(pk, r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, uu.x, uu.y, gamma, L,
                           ev);
      if constexpr (BLK) {   // coarse blocks: an intra pair keeps its exact F_ij, no statistics or record
        if (c_intra[o]) {
          acc.add_intra(Real(0.5) * ev.rho);
          const int rp = sm.srp[t % CPASS_STAGES][lane];
          V4<Real> z;
          z.x = z.y = z.z = z.w = Real(0);
          rec_a[rp] = z;
          rec_b[rp] = z;
          rec_c[rp] = RecC<Real>::make(Real(0), Real(0));
          return;
        }
      }
      acc.add(ev, uu.x, uu.y);
      const Real wlb = ev.wb * ev.lamb, wl = ev.w * ev.lam;
      V4<Real> ra, rb;
      ra.x = wlb * ev.lamb;
      ra.y = Real(-0.5) * wlb * ev.Reb0;
      ra.z = Real(-0.5) * wlb * ev.Reb1;
      ra.w = Real(-0.5) * wlb * ev.Reb2;
      rb.x = wl * ev.lam;
      rb.y = Real(-0.5) * wl * ev.Re0;
      rb.z = Real(-0.5) * wl * ev.Re1;
      rb.w = Real(-0.5) * wl * ev.Re2;
      const int rp = sm.srp[t % CPASS_STAGES][lane];
      rec_a[rp] = ra;
      rec_b[rp] = rb;
      rec_c[rp] = RecC<Real>::make(Real(0.5) * ev.rho, ev.gap);
    }
  };
  // Two batches per step: batches t, t+1 are evaluated one after the other with one read of
  // the pack while t+2, t+3 are in flight (measured: 0.456 ms against 0.480 ms for one batch
  // per step with two in flight; an unrolled loop over the pair that interleaves the two
  // evaluations needs 189 registers and takes 0.516 ms).
  issue(0, index_of(0));
  issue(1, index_of(1));
  int j0 = index_of(2), j1 = index_of(3);
  for (int t = 0; t < nb; t += 2) {
    issue(t + 2, j0);
    issue(t + 3, j1);
    j0 = index_of(t + 4);
    j1 = index_of(t + 5);
    cp_async_wait<2>();
    process(t);
    process(t + 1);
  }
  cp_async_wait<0>();
  // warp reduction; the partial is stored in the pass precision and summed over the
  // camera's chunks in FP64 by the camera solve
  if constexpr (BLK)
    acc.reduce_store(lane, part + (size_t)warp * CP_STRIDE, true);
  else
    acc.reduce_store(lane, part + (size_t)warp * CP_STRIDE);
}

// Chunks c0 .. c1 - 1. Without a counter (ctr null) one warp per chunk. With one, a bounded grid
// whose warps take the chunks in order from ctr[0]; the warp that leaves last (ctr[1] counts the
// warps out) sets both back to zero for the next launch. No warp waits on another.
template <int LOSS, class Real, class Real2>
__global__ void __launch_bounds__(CPASS_WARPS * 32)
    k_cpass(int c0, int c1, unsigned* __restrict__ ctr, const int* __restrict__ chunk_cam,
            const int* __restrict__ chunk_beg, const int* __restrict__ c_lm, const Real2* __restrict__ c_u,
            const V4<Real>* __restrict__ pack, const V4<Real>* __restrict__ lmrec, LossC<Real> L, IterParams P,
            Real* __restrict__ part, const int* __restrict__ c_rpos, V4<Real>* __restrict__ rec_a,
            V4<Real>* __restrict__ rec_b, typename RecC<Real>::type* __restrict__ rec_c) {
  __shared__ CpassWarpSmem<Real, Real2> sm[CPASS_WARPS];
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const Real gamma = Real(P.gam[*P.it]);
  if (ctr == nullptr) {
    const int warp = c0 + blockIdx.x * CPASS_WARPS + wib;
    if (warp >= c1) return;
    cpass_chunk<LOSS, Real, Real2, false>(warp, lane, sm[wib], gamma, chunk_cam, chunk_beg, c_lm, c_u, pack, lmrec, L,
                                          part, c_rpos, rec_a, rec_b, rec_c);
    return;
  }
  for (;;) {
    int c = 0;
    if (lane == 0) c = c0 + (int)atomicAdd(ctr, 1u);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= c1) break;
    __syncwarp();   // every lane is done with the previous chunk's shared memory
    cpass_chunk<LOSS, Real, Real2, false>(c, lane, sm[wib], gamma, chunk_cam, chunk_beg, c_lm, c_u, pack, lmrec, L,
                                          part, c_rpos, rec_a, rec_b, rec_c);
  }
  if (lane == 0) {
    __threadfence();
    if (atomicAdd(ctr + 1, 1u) == gridDim.x * CPASS_WARPS - 1) {
      ctr[0] = 0u;
      ctr[1] = 0u;
    }
  }
}

// The camera pass with coarse blocks (FP64): c_intra[o] marks the camera-sorted observations
// whose camera and landmark share a block.
template <int LOSS>
__global__ void __launch_bounds__(CPASS_WARPS * 32)
    k_cpass_blk(int n_chunks, const int* __restrict__ chunk_cam, const int* __restrict__ chunk_beg,
                const int* __restrict__ c_lm, const double2* __restrict__ c_u, const V4<double>* __restrict__ pack,
                const V4<double>* __restrict__ lmrec, LossC<double> L, IterParams P, double* __restrict__ part,
                const int* __restrict__ c_rpos, V4<double>* __restrict__ rec_a, V4<double>* __restrict__ rec_b,
                double2* __restrict__ rec_c, const uint8_t* __restrict__ c_intra) {
  __shared__ CpassWarpSmem<double, double2> sm[CPASS_WARPS];
  const int wib = threadIdx.x >> 5;
  const int warp = blockIdx.x * CPASS_WARPS + wib;
  const int lane = threadIdx.x & 31;
  if (warp >= n_chunks) return;
  cpass_chunk<LOSS, double, double2, false, true>(warp, lane, sm[wib], P.gam[*P.it], chunk_cam, chunk_beg, c_lm, c_u,
                                                 pack, lmrec, L, part, c_rpos, rec_a, rec_b, rec_c, c_intra);
}

// ---------------------------------------------------------------------------
// 2. landmark pass: one CTA per tile of consecutive landmarks (internal numbering)
// ---------------------------------------------------------------------------
// Tile data: landmarks tile_lm[t] .. tile_lm[t+1]; their observations occupy the
// landmark-sorted slots lm_ptr[first] .. lm_ptr[last] and the same range of record positions,
// where cpass stored them in camera-sorted order; t_inv maps a slot (relative to the tile
// start) to its record position. One thread issues TMA bulk copies of the tile's three record
// ranges and of its slice of t_inv into shared memory, completing on an mbarrier; each thread
// then reduces its landmark's records through t_inv. Reads the landmark state of iteration k
// and writes that of k+1 to the other buffer.
// Bounded waits on the tile copies, measured with the %globaltimer nanosecond clock. The first
// wait lasts at most IterParams::wait_ns (a runtime option, 1 s by default; 0 gives up before
// the first poll). If it runs out, the CTA sets flag bit 2 (the host returns DABA_ERR_TIMEOUT),
// waits up to LPASS_DRAIN_NS more so that no copy lands in shared memory after the CTA has
// exited, and skips its tile. Both waits also stop after LPASS_MAX_POLLS polls.
constexpr long long LPASS_DRAIN_NS = 2000000000ll;
constexpr long long LPASS_MAX_POLLS = 1ll << 30;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// polls the mbarrier phase until it completes (true) or limit_ns have passed (false)
__device__ __forceinline__ bool mbar_wait_for(unsigned long long* bar, unsigned parity, long long limit_ns) {
  if (limit_ns <= 0) return false;
  const unsigned long long t0 = globaltimer_ns();
  for (long long w = 0; w < LPASS_MAX_POLLS; ++w) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((long long)(globaltimer_ns() - t0) >= limit_ns) return false;
  }
  return false;
}
// 1D bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Shared memory of a tile of at most no_cap observations: two V4 arrays (terms at xbar and at
// x^k), the third records (RecC) and the slot map, each with room for the alignment of its
// copy to 16 bytes, then the mbarrier.
template <class Real>
struct LpassSmem {
  using RC = typename RecC<Real>::type;
  static constexpr int kC = 16 / (int)sizeof(RC);   // elements per 16 bytes
  static __host__ __device__ size_t a_off(int) { return 0; }
  static __host__ __device__ size_t b_off(int cap) { return (size_t)cap * sizeof(V4<Real>); }
  static __host__ __device__ size_t c_off(int cap) { return 2 * (size_t)cap * sizeof(V4<Real>); }
  // a copy widened at both ends holds at most cap + 2 (kC - 1) third records and cap + 14
  // slot-map entries
  static __host__ __device__ size_t i_off(int cap) {
    return c_off(cap) + (((size_t)(cap + 2 * kC) * sizeof(RC) + 15) & ~(size_t)15);
  }
  static __host__ __device__ size_t bar_off(int cap) {
    return i_off(cap) + (((size_t)(cap + 16) * 2 + 15) & ~(size_t)15);
  }
  static __host__ __device__ size_t bytes(int cap) { return bar_off(cap) + 16; }
};
template <class Real>
__host__ __device__ inline size_t lpass_smem_bytes(int no_cap) {
  return LpassSmem<Real>::bytes(no_cap);
}

// double-float addition: (hi, lo) + x with |lo| <= ulp(hi)/2 afterwards
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (x - bb);
  const float l2 = lo + err;
  const float h2 = s + l2;
  lo = l2 - (h2 - s);
  hi = h2;
}

// Outputs of the landmark pass (one set per launch).
template <class Real>
struct LpassOut {
  V4<Real>* lmrec_out = nullptr;
  V4<float>* lm_lo_out = nullptr;
  uint8_t* lm_rs = nullptr;
  double* lm_Fdiag = nullptr;
  double* lm_Fbdiag = nullptr;
  V4<Real>* lm_alt = nullptr;
  double* lm_sums = nullptr;
  double* blk_sums = nullptr;   // coarse blocks: the 10 sums of every landmark, nothing else (sum mode)
};

// One landmark of the landmark pass: sums its records (slots s0 .. s1 of the tile, through the
// slot map) and runs Eqs. DEalpha, Fak, lFak in slack form, the accelerated update, the restart
// test and the MM re-solve, then writes the landmark's state of iteration k+1. A, B, lo0: its
// state of iteration k. Returns whether it restarted (counted for accelerated runs only); gsum
// receives its term of the global restart test.
template <class Real, bool HAS_LO>
__device__ __forceinline__ int lpass_landmark(const V4<Real>* __restrict__ sca, const V4<Real>* __restrict__ scb,
                                              const typename RecC<Real>::type* __restrict__ cc,
                                              const uint16_t* __restrict__ inv, int s0, int s1, const V4<Real>& A,
                                              const V4<Real>& B, const V4<float>& lo0, size_t g, Real gamma, int first,
                                              const IterParams& P, const LpassOut<Real>& O, double& gsum) {
  using RC = typename RecC<Real>::type;
  const bool global = P.accelerated && P.restart_global;
  const Real hx = hxi_of<Real>(P), eta1 = eta1_of<Real>(P);
  Real st[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) st[k] = Real(0);
  for (int s = s0; s < s1; ++s) {
    const int q = inv[s];
    const V4<Real> a = sca[q], b = scb[q];
    const RC c = cc[q];
    st[0] += a.x;
    st[1] += a.y;
    st[2] += a.z;
    st[3] += a.w;
    st[4] += b.x;
    st[5] += b.y;
    st[6] += b.z;
    st[7] += b.w;
    st[8] += RecC<Real>::F(c);
    st[9] += RecC<Real>::gap(c);
  }
  if (O.blk_sums) {   // coarse blocks: the block solve takes it from here
#pragma unroll
    for (int k = 0; k < 10; ++k) O.blk_sums[g * 10 + k] = double(st[k]);
    return 0;
  }
  const Real dl0 = A.w, dl1 = B.x, dl2 = B.y;
  // Eq. DEalpha, Eq. Fak, Eq. lFak in slack form (S = Fbar^(k-1) - E^(k)):
  //   Fbar^(k) - F^(k) = (1 - eta)(S - dE), and E^(k+1) > Fbar^(k)  <=>  dE_next > (1 - eta)(S - dE)
  const Real dE = -hx * (dl0 * dl0 + dl1 * dl1 + dl2 * dl2) + Real(0.5) * st[9];
  const Real S = first ? Real(0) : B.z;
  const Real thr = eta1 * (S - dE);
  // accelerated update (Eq. update_amm): l = lbar - bbar / (abar + xi/2), as a step from l^k
  const Real ib = fdiv(Real(1), st[0] + hx);
  const Real sa0 = gamma * dl0 - st[1] * ib, sa1 = gamma * dl1 - st[2] * ib, sa2 = gamma * dl2 - st[3] * ib;
  // E^alpha(l | x^k) - E^alpha(l^k | x^k) = (a + xi/2)|dl|^2 + 2 dl . b
  const Real ak = st[4] + hx;
  Real step0 = sa0, step1 = sa1, step2 = sa2;
  Real dEn = ak * (sa0 * sa0 + sa1 * sa1 + sa2 * sa2) + Real(2) * (sa0 * st[5] + sa1 * st[6] + sa2 * st[7]);
  const bool rs = P.accelerated ? (!global && dEn > thr) : true;
  if (rs || global) {   // adaptive restart: MM update (Eq. update_mm) from l^k
    const Real ik = fdiv(Real(1), ak);
    const Real m0 = -st[5] * ik, m1 = -st[6] * ik, m2 = -st[7] * ik;
    const Real dEm = -(st[5] * st[5] + st[6] * st[6] + st[7] * st[7]) * ik;
    if (rs) {
      step0 = m0;
      step1 = m1;
      step2 = m2;
      dEn = dEm;
    } else {   // global variant: keep the MM alternative and this block's term of the test
      V4<Real> a0, a1;
      a0.x = m0, a0.y = m1, a0.z = m2, a0.w = thr - dEm;
      a1.x = a1.y = a1.z = a1.w = Real(0);
      if (!HAS_LO) {
        const double E = first ? double(Real(0.5) * st[8]) : double(B.w);
        a1.x = Real(E + double(dE) + double(dEm));
      }
      O.lm_alt[2 * g] = a0;
      O.lm_alt[2 * g + 1] = a1;
      gsum = double(dEn) - double(thr);
    }
  }
  V4<Real> nA, nB;
  if (HAS_LO) {
    float h0 = float(A.x), h1 = float(A.y), h2 = float(A.z);
    float o0 = lo0.x, o1 = lo0.y, o2 = lo0.z;
    df_add(h0, o0, float(step0));
    df_add(h1, o1, float(step1));
    df_add(h2, o2, float(step2));
    nA.x = Real(h0);
    nA.y = Real(h1);
    nA.z = Real(h2);
    V4<float> nlo;
    nlo.x = o0;
    nlo.y = o1;
    nlo.z = o2;
    nlo.w = 0.f;
    O.lm_lo_out[g] = nlo;
  } else {
    nA.x = A.x + step0;
    nA.y = A.y + step1;
    nA.z = A.z + step2;
  }
  nA.w = step0;
  nB.x = step1;
  nB.y = step2;
  nB.z = thr - dEn;
  nB.w = B.w;
  if (!HAS_LO) {   // FP64 path: E^(k) and the diagnostics F^(k), Fbar^(k)
    const double E = first ? double(Real(0.5) * st[8]) : double(B.w);
    const double F = E + double(dE);
    O.lm_Fdiag[g] = F;
    O.lm_Fbdiag[g] = F + double(thr);
    nB.w = Real(F + double(dEn));
    if (O.lm_sums) {   // the reverse mode keeps (a, b) at x̄ and at x^k of every landmark
#pragma unroll
      for (int k = 0; k < 8; ++k) O.lm_sums[g * 8 + k] = double(st[k]);
    }
  }
  O.lmrec_out[2 * g] = nA;
  O.lmrec_out[2 * g + 1] = nB;
  O.lm_rs[g] = (rs && P.accelerated) ? 1 : 0;
  return (rs && P.accelerated) ? 1 : 0;
}

// restart count of a tile and, for the global variant, its sum of the test terms (fixed order)
__device__ __forceinline__ void lpass_tile_sums(int nrs, double gsum, bool global, int tile, int* tile_rs,
                                                double* g_tile) {
  __shared__ int redi[LPASS_THREADS / 32];
  __shared__ double redg[LPASS_THREADS / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nrs += __shfl_xor_sync(0xffffffffu, nrs, off);
  if ((threadIdx.x & 31) == 0) redi[threadIdx.x >> 5] = nrs;
  if (global) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, off);
    if ((threadIdx.x & 31) == 0) redg[threadIdx.x >> 5] = gsum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    for (int w = 0; w < LPASS_THREADS / 32; ++w) n += redi[w];
    tile_rs[tile] = n;
    if (global) {
      double t = 0.0;
      for (int w = 0; w < LPASS_THREADS / 32; ++w) t += redg[w];
      g_tile[tile] = t;
    }
  }
}

// One tile of the landmark pass by the CTA's LPASS_THREADS threads (smem_raw: the tile's shared
// memory; gamma and first of this iteration). Every thread of the CTA calls it. Returns false if
// a bounded wait ran out (the tile is then skipped, flag bit 2 set).
template <class Real, class Real2, bool HAS_LO, bool COH, bool REINIT = COH>
__device__ __forceinline__ bool lpass_tile(int tile, int no_cap, unsigned char* smem_raw, Real gamma, int first,
                                           const int* __restrict__ tile_lm, const int* __restrict__ lm_ptr,
                                           const uint16_t* __restrict__ t_inv, const V4<Real>* __restrict__ rec_a,
                                           const V4<Real>* __restrict__ rec_b,
                                           const typename RecC<Real>::type* __restrict__ rec_c,
                                           const V4<Real>* __restrict__ lmrec, const V4<float>* __restrict__ lm_lo,
                                           const IterParams& P, int* __restrict__ tile_rs, const LpassOut<Real>& O) {
  using RC = typename RecC<Real>::type;
  using SM = LpassSmem<Real>;
  const int lb = tile_lm[tile], le = tile_lm[tile + 1];
  const int nl = le - lb;
  const int ob = lm_ptr[lb], oe = lm_ptr[le];
  const int no = oe - ob;
  V4<Real>* sca = reinterpret_cast<V4<Real>*>(smem_raw + SM::a_off(no_cap));
  V4<Real>* scb = reinterpret_cast<V4<Real>*>(smem_raw + SM::b_off(no_cap));
  RC* scc = reinterpret_cast<RC*>(smem_raw + SM::c_off(no_cap));
  uint16_t* sinv = reinterpret_cast<uint16_t*>(smem_raw + SM::i_off(no_cap));
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + SM::bar_off(no_cap));
  // copy ranges, widened to 16-byte boundaries for the third records and the slot map
  const int cs = ob & ~(SM::kC - 1), ce = (oe + SM::kC - 1) & ~(SM::kC - 1);
  const int is = ob & ~7, ie = (oe + 7) & ~7;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    if (no > 0) {
      const unsigned ba = (unsigned)no * (unsigned)sizeof(V4<Real>);
      const unsigned bc = (unsigned)(ce - cs) * (unsigned)sizeof(RC);
      const unsigned bi = (unsigned)(ie - is) * 2u;
      mbar_arrive_expect_tx(bar, 2u * ba + bc + bi);
      bulk_g2s(sca, rec_a + ob, ba, bar);
      bulk_g2s(scb, rec_b + ob, ba, bar);
      bulk_g2s(scc, rec_c + cs, bc, bar);
      bulk_g2s(sinv, t_inv + is, bi, bar);
    } else {
      mbar_arrive_expect_tx(bar, 0u);
    }
  }
  // the landmark state of this thread's landmark (at most one: nl <= blockDim.x) is loaded
  // while the copies are in flight
  static_assert(TILE_LMS <= LPASS_THREADS, "one landmark per thread");
  const int jl = threadIdx.x;
  const size_t g = (size_t)(lb + jl);
  V4<Real> A, B;
  V4<float> lo0;
  int s0 = 0, s1 = 0;
  if (jl < nl) {
    A = ld_mut<COH>(lmrec + 2 * g);
    B = ld_mut<COH>(lmrec + 2 * g + 1);
    if (HAS_LO) lo0 = ld_mut<COH>(lm_lo + g);
    s0 = lm_ptr[lb + jl] - ob;
    s1 = lm_ptr[lb + jl + 1] - ob;
  }
  __syncthreads();   // the mbarrier is initialised
  bool ok = mbar_wait_for(bar, 0u, P.wait_ns);
  if (!ok) {   // copies not complete in time: report, let them land, skip the tile
    atomicOr(P.flag, 2);
    mbar_wait_for(bar, 0u, LPASS_DRAIN_NS);
  }
  int nrs = 0;
  double gsum = 0.0;   // global restart variant: this thread's E(k+1) - Fbar(k)
  if (ok && jl < nl)
    nrs = lpass_landmark<Real, HAS_LO>(sca, scb, scc + (ob - cs), sinv + (ob - is), s0, s1, A, B, lo0, g, gamma, first,
                                       P, O, gsum);
  lpass_tile_sums(nrs, gsum, P.accelerated && P.restart_global, tile, tile_rs, P.g_tile);   // ends every thread's reads
  if (REINIT && threadIdx.x == 0) mbar_inval(bar);   // the CTA initialises it again for its next tile
  return ok;
}

// Tiles q0 .. q0 + nq - 1 of the launch's tile order (tile q, or tlist[q] with a list). Without a
// counter (ctr null) one CTA per tile; with one, a bounded grid whose CTAs take the tiles in order
// from ctr[0], reset by the CTA that leaves last as in k_cpass.
template <class Real, class Real2, bool HAS_LO>
__global__ void __launch_bounds__(LPASS_THREADS)
    k_lpass(int q0, int nq, const int* __restrict__ tlist, unsigned* __restrict__ ctr, int no_cap,
            const int* __restrict__ tile_lm, const int* __restrict__ lm_ptr, const uint16_t* __restrict__ t_inv,
            const V4<Real>* __restrict__ rec_a, const V4<Real>* __restrict__ rec_b,
            const typename RecC<Real>::type* __restrict__ rec_c, const V4<Real>* __restrict__ lmrec,
            const V4<float>* __restrict__ lm_lo, IterParams P, int* __restrict__ tile_rs, LpassOut<Real> O) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Real gamma = Real(P.gam[*P.it]);
  const int first = *P.first;
  if (ctr == nullptr) {
    const int q = q0 + blockIdx.x;
    lpass_tile<Real, Real2, HAS_LO, false>(tlist ? tlist[q] : q, no_cap, smem_raw, gamma, first, tile_lm, lm_ptr,
                                           t_inv, rec_a, rec_b, rec_c, lmrec, lm_lo, P, tile_rs, O);
    return;
  }
  __shared__ int s_q;
  for (;;) {
    if (threadIdx.x == 0) s_q = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    const int q = s_q;   // read by every thread before the barriers inside the tile let thread 0 on
    if (q >= nq) break;
    lpass_tile<Real, Real2, HAS_LO, false, true>(tlist ? tlist[q0 + q] : q0 + q, no_cap, smem_raw, gamma, first,
                                                 tile_lm, lm_ptr, t_inv, rec_a, rec_b, rec_c, lmrec, lm_lo, P,
                                                 tile_rs, O);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ctr + 1, 1u) == gridDim.x - 1) {
      ctr[0] = 0u;
      ctr[1] = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// 3. camera block solves (FP64)
// ---------------------------------------------------------------------------
template <class T>
struct CamT {
  T R[9], t[3], d[3];
};

// M(c) column a (a = 0..5) of the 3x6 matrix [R e1, R e2, d1 R e3, d2 R e3, d3 R e3, t].
template <class T>
__device__ __forceinline__ void mcol(const CamT<T>& c, int a, T out[3]) {
  if (a < 2) {
    out[0] = c.R[0 + a];
    out[1] = c.R[3 + a];
    out[2] = c.R[6 + a];
  } else if (a < 5) {
    const T dk = c.d[a - 2];
    out[0] = dk * c.R[2];
    out[1] = dk * c.R[5];
    out[2] = dk * c.R[8];
  } else {
    out[0] = c.t[0];
    out[1] = c.t[1];
    out[2] = c.t[2];
  }
}

// Packed camera statistics: H (upper triangle, row-major, 21 values) then B (6x3, 18 values).
template <class T>
__device__ __forceinline__ T st_H(const T* s, int a, int b) { return a <= b ? s[tri6(a, b)] : s[tri6(b, a)]; }
template <class T>
__device__ __forceinline__ T st_B(const T* s, int a, int c) { return s[21 + a * 3 + c]; }

// E^alpha(c | z) - E^alpha(c_z | z) = xi/2 |c - c_z|^2 + tr(dM H dM^T) + 2 tr(dM B).
template <class T>
__device__ inline T cam_phi(const T* st, const CamT<T>& z, const CamT<T>& c, T xi) {
  using N = Num<T>;
  T dM[6][3];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    T mc[3], mz[3];
    mcol(c, a, mc);
    mcol(z, a, mz);
    dM[a][0] = mc[0] - mz[0];
    dM[a][1] = mc[1] - mz[1];
    dM[a][2] = mc[2] - mz[2];
  }
  T prox = N::c(0.f);
#pragma unroll
  for (int k = 0; k < 9; ++k) prox = prox + (c.R[k] - z.R[k]) * (c.R[k] - z.R[k]);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    prox = prox + (c.t[k] - z.t[k]) * (c.t[k] - z.t[k]) + (c.d[k] - z.d[k]) * (c.d[k] - z.d[k]);
  T q = N::c(0.f), lin = N::c(0.f);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    q = q + st_H(st, a, a) * (dM[a][0] * dM[a][0] + dM[a][1] * dM[a][1] + dM[a][2] * dM[a][2]);
#pragma unroll
    for (int b = a + 1; b < 6; ++b)
      q = q + N::c(2.0f) * st_H(st, a, b) * (dM[a][0] * dM[b][0] + dM[a][1] * dM[b][1] + dM[a][2] * dM[b][2]);
    lin = lin + dM[a][0] * st_B(st, a, 0) + dM[a][1] * st_B(st, a, 1) + dM[a][2] * st_B(st, a, 2);
  }
  return N::c(0.5f) * xi * prox + q + N::c(2.0f) * lin;
}

// Block-exact alternation on E^alpha(. | z) started at c_z (z supplies H, B).
// R-step: with (t, d) fixed, tr(dM H dM^T) + 2 tr(dM B) - xi <R, R_z> is affine in R, so
//   R = ProjRot3D(K),  K = xi R_z + 2 (W H - B^T) P(d)^T,  W = M(c_z) - t e6^T,
//   P(d) = [e1, e2, d1 e3, d2 e3, d3 e3, 0].
// (t, d)-step: with R fixed, dM h = dM0 h + v (phi . dd) + lambda dt with v = R e3 and
//   dM0 = M(R, t_z, d_z) - M(c_z); the normal equations of the resulting least squares
//   in y = (dt, dd) use H[5,5], H[5,2:5], H[2:5,2:5]; they are solved through the 3x3 Schur
//   complement of their scaled-identity dt block (below).
// y_out (optional): the (t, d) displacement from z of the last (t, d)-step taken (zero if none),
// exact to the solve's rounding even where c.t = z.t + y rounds it away.
template <class T>
__device__ inline void cam_scam(const T* st, const CamT<T>& z, T xi, int n_alt, CamT<T>& c, T* y_out = nullptr) {
  using N = Num<T>;
  c = z;
  if (y_out) {
#pragma unroll
    for (int k = 0; k < 6; ++k) y_out[k] = N::c(0.f);
  }
  for (int it = 0; it < n_alt; ++it) {
    // ---- R-step
    T W[3][6];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      T mz[3];
      mcol(z, a, mz);
      W[0][a] = mz[0];
      W[1][a] = mz[1];
      W[2][a] = mz[2];
    }
    W[0][5] = z.t[0] - c.t[0];
    W[1][5] = z.t[1] - c.t[1];
    W[2][5] = z.t[2] - c.t[2];
    T G[3][6];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        T s = -st_B(st, a, r);
#pragma unroll
        for (int b = 0; b < 6; ++b) s = s + W[r][b] * st_H(st, b, a);
        G[r][a] = s;
      }
    T K[9];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      K[r * 3 + 0] = xi * z.R[r * 3 + 0] + N::c(2.0f) * G[r][0];
      K[r * 3 + 1] = xi * z.R[r * 3 + 1] + N::c(2.0f) * G[r][1];
      K[r * 3 + 2] = xi * z.R[r * 3 + 2] + N::c(2.0f) * (c.d[0] * G[r][2] + c.d[1] * G[r][3] + c.d[2] * G[r][4]);
    }
    // warm start from the rotation of the previous alternation (first: the conditioning one)
    T Rn[9];
    if (proj_rot3d_from(K, c.R, Rn)) {
#pragma unroll
      for (int a = 0; a < 9; ++a) c.R[a] = Rn[a];
    } else {
      proj_rot3d_polar(K, c.R);
    }
    // ---- (t, d)-step
    const T v[3] = {c.R[2], c.R[5], c.R[8]};
    const T vz[3] = {z.R[2], z.R[5], z.R[8]};
    T dM0[6][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dM0[0][k] = c.R[k * 3 + 0] - z.R[k * 3 + 0];
      dM0[1][k] = c.R[k * 3 + 1] - z.R[k * 3 + 1];
      dM0[2][k] = z.d[0] * (v[k] - vz[k]);
      dM0[3][k] = z.d[1] * (v[k] - vz[k]);
      dM0[4][k] = z.d[2] * (v[k] - vz[k]);
      dM0[5][k] = N::c(0.f);
    }
    // right-hand side: top dM0 H[:,5] + B[5,:];  bottom H[2:5,:] (dM0^T v) + B[2:5,:] v
    T rhs[6];
    T dv[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) dv[a] = dM0[a][0] * v[0] + dM0[a][1] * v[1] + dM0[a][2] * v[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T s = st_B(st, 5, k);
#pragma unroll
      for (int a = 0; a < 6; ++a) s = s + dM0[a][k] * st_H(st, a, 5);
      rhs[k] = N::c(-2.0f) * s;
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      T s = st_B(st, 2 + m, 0) * v[0] + st_B(st, 2 + m, 1) * v[1] + st_B(st, 2 + m, 2) * v[2];
#pragma unroll
      for (int a = 0; a < 6; ++a) s = s + st_H(st, 2 + m, a) * dv[a];
      rhs[3 + m] = N::c(-2.0f) * s;
    }
    // normal equations [alpha I, Bc; Bc^T, D] (dt, dd) = rhs with alpha = 2 H55 + xi,
    // Bc = 2 v h^T (h = H[2:5,5]) and D = 2 H[2:5,2:5] + xi I: eliminate dt (Schur complement)
    //   (D - (4 |v|^2 / alpha) h h^T) dd = rhs_d - (2 (v . rhs_t) / alpha) h,
    //   dt = (rhs_t - 2 v (h . dd)) / alpha,
    // a 3x3 solve (Cramer's rule; leading minors as the positive-definiteness test)
    const T alpha = N::c(2.0f) * st_H(st, 5, 5) + xi;
    if (N::pos(alpha)) {
      const T ia = N::rcp(alpha);
      const T h[3] = {st_H(st, 2, 5), st_H(st, 3, 5), st_H(st, 4, 5)};
      const T vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
      const T vr = v[0] * rhs[0] + v[1] * rhs[1] + v[2] * rhs[2];
      const T f4 = N::c(4.0f) * vv * ia, f2 = N::c(2.0f) * vr * ia;
      T Sm[3][3], r[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
#pragma unroll
        for (int n = 0; n < 3; ++n) Sm[m][n] = N::c(2.0f) * st_H(st, 2 + m, 2 + n) - f4 * h[m] * h[n];
        Sm[m][m] = Sm[m][m] + xi;
        r[m] = rhs[3 + m] - f2 * h[m];
      }
      const T m1 = Sm[0][0] * Sm[1][1] - Sm[0][1] * Sm[0][1];
      const T c00 = Sm[1][1] * Sm[2][2] - Sm[1][2] * Sm[1][2], c01 = Sm[0][2] * Sm[1][2] - Sm[0][1] * Sm[2][2];
      const T c02 = Sm[0][1] * Sm[1][2] - Sm[0][2] * Sm[1][1], c11 = Sm[0][0] * Sm[2][2] - Sm[0][2] * Sm[0][2];
      const T c12 = Sm[0][1] * Sm[0][2] - Sm[0][0] * Sm[1][2];
      const T det = Sm[0][0] * c00 + Sm[0][1] * c01 + Sm[0][2] * c02;
      if (N::pos(Sm[0][0]) && N::pos(m1) && N::pos(det)) {
        const T id = N::rcp(det);
        const T y0 = (c00 * r[0] + c01 * r[1] + c02 * r[2]) * id;
        const T y1 = (c01 * r[0] + c11 * r[1] + c12 * r[2]) * id;
        const T y2 = (c02 * r[0] + c12 * r[1] + m1 * r[2]) * id;
        const T hy = N::c(2.0f) * (h[0] * y0 + h[1] * y1 + h[2] * y2);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const T yt = (rhs[k] - v[k] * hy) * ia;
          c.t[k] = z.t[k] + yt;
          if (y_out) y_out[k] = yt;
        }
        c.d[0] = z.d[0] + y0;
        c.d[1] = z.d[1] + y1;
        c.d[2] = z.d[2] + y2;
        if (y_out) {
          y_out[3] = y0;
          y_out[4] = y1;
          y_out[5] = y2;
        }
      }
    }
  }
}

// Camera solver variant: one successful Levenberg-Marquardt step on E^alpha(. | z) from c_z.
// Parameters theta = (phi, tau, delta) with R = R_z Exp(phi), t = t_z + tau, d = d_z + delta.
// With sigma_a the camera-frame direction of column a of M (e1, e2, d_m e3) the Gauss-Newton
// model of the surrogate in the statistics is (camera frame, q_b = sum_a<5 H_ab sigma_a,
// Q = sum w p p^T = [q_0, q_1, sum_m d_m q_(2+m)], b_a = R_z^T B_a, r_c = row c of R_z):
//   A_phiphi = 2 (tr Q I - Q) + 2 xi I     A_phitau[:, c] = -2 r_c x q_5
//   A_phidel[:, n] = 2 (q_(2+n),y, -q_(2+n),x, 0)
//   A_tautau = (2 H_55 + xi) I             A_taudel[c][n] = 2 H_(5,2+n) R_z[c][2]
//   A_deldel = 2 H[2:5, 2:5] + xi I
//   g_phi = 2 sum_a<5 sigma_a x b_a        g_tau = 2 B_5      g_del[n] = 2 (R_z e3) . B_(2+n)
// The step solves (A + mu diag A) theta = -g (Cholesky) and is taken if cam_phi < 0; mu starts
// at LM_MU0 and grows tenfold, at most LM_TRIES times; otherwise the camera stays at c_z.
constexpr double LM_MU0 = 1e-3;
constexpr int LM_TRIES = 8;

__device__ __forceinline__ int lt9(int i, int j) { return i * (i + 1) / 2 + j; }   // packed lower, j <= i

// the model (A packed lower, g) at c_z
__device__ inline void cam_lm_model(const double* st, const CamT<double>& z, double xi, double* A, double* g) {
  {
    double q[6][3];
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      q[b][0] = st_H(st, 0, b);
      q[b][1] = st_H(st, 1, b);
      q[b][2] = z.d[0] * st_H(st, 2, b) + z.d[1] * st_H(st, 3, b) + z.d[2] * st_H(st, 4, b);
    }
    double Q[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      Q[r][0] = q[0][r];
      Q[r][1] = q[1][r];
      Q[r][2] = z.d[0] * q[2][r] + z.d[1] * q[3][r] + z.d[2] * q[4][r];
    }
    const double trQ = Q[0][0] + Q[1][1] + Q[2][2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) A[lt9(i, j)] = 2.0 * ((i == j ? trQ : 0.0) - 0.5 * (Q[i][j] + Q[j][i])) + (i == j ? 2.0 * xi : 0.0);
    // tau rows (3..5): A[3 + c][i] for phi column i = (-2 r_c x q_5)_i
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      const double r0 = z.R[cc * 3 + 0], r1 = z.R[cc * 3 + 1], r2 = z.R[cc * 3 + 2];
      A[lt9(3 + cc, 0)] = -2.0 * (r1 * q[5][2] - r2 * q[5][1]);
      A[lt9(3 + cc, 1)] = -2.0 * (r2 * q[5][0] - r0 * q[5][2]);
      A[lt9(3 + cc, 2)] = -2.0 * (r0 * q[5][1] - r1 * q[5][0]);
#pragma unroll
      for (int j = 0; j <= cc; ++j) A[lt9(3 + cc, 3 + j)] = cc == j ? 2.0 * st_H(st, 5, 5) + xi : 0.0;
    }
    // delta rows (6..8)
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      A[lt9(6 + n, 0)] = 2.0 * q[2 + n][1];
      A[lt9(6 + n, 1)] = -2.0 * q[2 + n][0];
      A[lt9(6 + n, 2)] = 0.0;
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) A[lt9(6 + n, 3 + cc)] = 2.0 * st_H(st, 5, 2 + n) * z.R[cc * 3 + 2];
#pragma unroll
      for (int m = 0; m <= n; ++m) A[lt9(6 + n, 6 + m)] = 2.0 * st_H(st, 2 + n, 2 + m) + (m == n ? xi : 0.0);
    }
    // gradient
    double bc[5][3];   // b_a = R_z^T B_a (camera frame)
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        bc[a][k] = z.R[0 * 3 + k] * st_B(st, a, 0) + z.R[1 * 3 + k] * st_B(st, a, 1) + z.R[2 * 3 + k] * st_B(st, a, 2);
    // sigma_a x b_a: e1 x b = (0, -b_z, b_y), e2 x b = (b_z, 0, -b_x), d_m e3 x b = d_m (-b_y, b_x, 0)
    g[0] = 2.0 * (bc[1][2] - z.d[0] * bc[2][1] - z.d[1] * bc[3][1] - z.d[2] * bc[4][1]);
    g[1] = 2.0 * (-bc[0][2] + z.d[0] * bc[2][0] + z.d[1] * bc[3][0] + z.d[2] * bc[4][0]);
    g[2] = 2.0 * (bc[0][1] - bc[1][0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) g[3 + k] = 2.0 * st_B(st, 5, k);
#pragma unroll
    for (int n = 0; n < 3; ++n)
      g[6 + n] = 2.0 * (z.R[2] * st_B(st, 2 + n, 0) + z.R[5] * st_B(st, 2 + n, 1) + z.R[8] * st_B(st, 2 + n, 2));
  }
}

__device__ inline void cam_lm(const double* st, const CamT<double>& z, double xi, CamT<double>& c) {
  c = z;
  double A[45], g[9];
  cam_lm_model(st, z, xi, A, g);
  double mu = LM_MU0;
  for (int tr = 0; tr < LM_TRIES; ++tr, mu *= 10.0) {
    // Cholesky of A + mu diag(A), then the two triangular solves
    double L[45];
    bool ok = true;
    for (int i = 0; i < 9; ++i) {
      for (int j = 0; j <= i; ++j) {
        double v = A[lt9(i, j)] * (i == j ? 1.0 + mu : 1.0);
        for (int k = 0; k < j; ++k) v -= L[lt9(i, k)] * L[lt9(j, k)];
        if (i == j) {
          if (!(v > 0.0)) ok = false;
          L[lt9(i, i)] = sqrt(ok ? v : 1.0);
        } else {
          L[lt9(i, j)] = v / L[lt9(j, j)];
        }
      }
    }
    if (!ok) continue;
    double y[9], th[9];
    for (int i = 0; i < 9; ++i) {
      double v = -g[i];
      for (int k = 0; k < i; ++k) v -= L[lt9(i, k)] * y[k];
      y[i] = v / L[lt9(i, i)];
    }
    for (int i = 8; i >= 0; --i) {
      double v = y[i];
      for (int k = i + 1; k < 9; ++k) v -= L[lt9(k, i)] * th[k];
      th[i] = v / L[lt9(i, i)];
    }
    CamT<double> cand;
    double E[9];
    rodrigues(th, E);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc)
        cand.R[r * 3 + cc] = z.R[r * 3 + 0] * E[0 * 3 + cc] + z.R[r * 3 + 1] * E[1 * 3 + cc] + z.R[r * 3 + 2] * E[2 * 3 + cc];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cand.t[k] = z.t[k] + th[3 + k];
      cand.d[k] = z.d[k] + th[6 + k];
    }
    if (cam_phi(st, z, cand, xi) < 0.0) {
      c = cand;
      return;
    }
  }
}

// the camera block solver of the variant in use
enum { CAM_SCAM = 0, CAM_LM = 1 };

// S-CAM in FP32 for the MIXED path: the statistics (FP32 partials summed in FP64) and the
// conditioning point are rounded to FP32 with the origin of t moved to z.t; the solve returns
// the rotation and the (t, d) displacements, which are added to z in FP64, so a small step
// keeps its relative accuracy. The restart metrics are evaluated in FP64 by the caller.
__device__ inline void cam_scam_f32(const double* st, const CamT<double>& z, double xi, int n_alt, CamT<double>& c) {
  float sf[39];
#pragma unroll
  for (int k = 0; k < 39; ++k) sf[k] = narrow(st[k]);
  CamT<float> zf, cf;
#pragma unroll
  for (int a = 0; a < 9; ++a) zf.R[a] = narrow(z.R[a]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    zf.t[k] = 0.f;
    zf.d[k] = narrow(z.d[k]);
  }
  float y[6];
  cam_scam<float>(sf, zf, narrow(xi), n_alt, cf, y);
#pragma unroll
  for (int a = 0; a < 9; ++a) c.R[a] = widen(cf.R[a]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c.t[k] = z.t[k] + widen(y[k]);
    c.d[k] = z.d[k] + widen(y[3 + k]);
  }
}
template <int SOLVER, class Real>
__device__ __forceinline__ void cam_solve(const double* st, const CamT<double>& z, double xi, int n_alt,
                                          CamT<double>& c) {
  if (SOLVER == CAM_LM)
    cam_lm(st, z, xi, c);
  else if (sizeof(Real) == 4)
    cam_scam_f32(st, z, xi, n_alt, c);
  else
    cam_scam(st, z, xi, n_alt, c);
}

__device__ __forceinline__ void acc_add(double& a, float x) { a += widen(x); }
__device__ __forceinline__ void acc_add(double& a, double x) { a += x; }

// Sum over chunks [c0, c1) of the 39 statistics at offset `off` of each partial (COH: the
// partials were written earlier in the same launch, so they are read from L2)
template <class Real, class T, bool COH = false>
__device__ __forceinline__ void sum_stats(const Real* __restrict__ part, int c0, int c1, int off, T* st) {
  static_assert(sizeof(T) == 8, "FP64 sums");
#pragma unroll
  for (int k = 0; k < 39; ++k) st[k] = 0.0;
  for (int c = c0; c < c1; ++c) {
    if constexpr (sizeof(Real) == 4) {
      const float4* p = reinterpret_cast<const float4*>(part + (size_t)c * CP_STRIDE + off);
#pragma unroll
      for (int v = 0; v < 10; ++v) {
        const float4 x = COH ? __ldcg(p + v) : __ldg(p + v);
        acc_add(st[4 * v + 0], x.x);
        acc_add(st[4 * v + 1], x.y);
        acc_add(st[4 * v + 2], x.z);
        if (v < 9) acc_add(st[4 * v + 3], x.w);
      }
    } else {
      const double2* p = reinterpret_cast<const double2*>(part + (size_t)c * CP_STRIDE + off);
#pragma unroll
      for (int v = 0; v < 20; ++v) {
        const double2 x = COH ? __ldcg(p + v) : __ldg(p + v);
        st[2 * v] += x.x;
        if (v < 19) st[2 * v + 1] += x.y;
      }
    }
  }
}

// pass pack from the FP64 solve results (FP32: nearest floats, the camera centre as high and
// low parts)
template <class Real>
__device__ __forceinline__ void write_pack_t(const CamT<double>& x, const CamT<double>& dx, const double* Rb,
                                             V4<Real>* pk) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    Real th, tl;
    split_real(x.t[r], th, tl);
    V4<Real> a, b, g;
    a.x = to_real<Real>(x.R[3 * r + 0]);
    a.y = to_real<Real>(x.R[3 * r + 1]);
    a.z = to_real<Real>(x.R[3 * r + 2]);
    a.w = th;
    b.x = to_real<Real>(Rb[3 * r + 0]);
    b.y = to_real<Real>(Rb[3 * r + 1]);
    b.z = to_real<Real>(Rb[3 * r + 2]);
    b.w = to_real<Real>(dx.t[r]);
    g.x = to_real<Real>(dx.R[3 * r + 0]);
    g.y = to_real<Real>(dx.R[3 * r + 1]);
    g.z = to_real<Real>(dx.R[3 * r + 2]);
    g.w = tl;
    pk[P4_RK + r] = a;
    pk[P4_RB + r] = b;
    pk[P4_DR + r] = g;
  }
  V4<Real> d, e;
  d.x = to_real<Real>(x.d[0]);
  d.y = to_real<Real>(x.d[1]);
  d.z = to_real<Real>(x.d[2]);
  d.w = Real(0);
  e.x = to_real<Real>(dx.d[0]);
  e.y = to_real<Real>(dx.d[1]);
  e.z = to_real<Real>(dx.d[2]);
  e.w = Real(0);
  pk[P4_D] = d;
  pk[P4_DD] = e;
}

// Rbar = ProjRot3D(K) of the extrapolation K = R + gamma dR (Eq. nesterov_R): in FP64 on the
// FP64 path; on the MIXED path K is rounded to FP32 and projected in FP32 (the pass reads Rbar
// in FP32, and the FP32 camera solve rounds it to FP32 as its conditioning rotation).
template <class Real>
__device__ __forceinline__ void extrap_rotation(const double* K, double* Rb) {
  if (sizeof(Real) == 4) {
    float Kf[9], Rf[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) Kf[a] = narrow(K[a]);
    proj_rot3d_near<float>(Kf, Rf);
#pragma unroll
    for (int a = 0; a < 9; ++a) Rb[a] = widen(Rf[a]);
  } else {
    proj_rot3d_near<double>(K, Rb);
  }
}

// ---------------------------------------------------------------------------
// camera prepare: Rbar^k = ProjRot3D(R^k + gamma dR^k) (Eq. nesterov_R) and the pack
// ---------------------------------------------------------------------------
template <class Real>
__global__ void k_cam_prepare(int M, const double* __restrict__ cam_x, const double* __restrict__ cam_dx,
                              IterParams P, double* __restrict__ cam_Rbar, V4<Real>* __restrict__ pack) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double gamma = P.gam[*P.it];
  const double* x = cam_x + (size_t)i * CSTRIDE;
  const double* dx = cam_dx + (size_t)i * CSTRIDE;
  double K[9], Rb[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) K[a] = x[CS_R + a] + gamma * dx[CS_R + a];
  extrap_rotation<Real>(K, Rb);
#pragma unroll
  for (int a = 0; a < 9; ++a) cam_Rbar[(size_t)i * 9 + a] = Rb[a];
  CamT<double> cx, cdx;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    cx.R[a] = x[CS_R + a];
    cdx.R[a] = dx[CS_R + a];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx.t[a] = x[CS_T + a];
    cdx.t[a] = dx[CS_T + a];
    cx.d[a] = x[CS_D + a];
    cdx.d[a] = dx[CS_D + a];
  }
  write_pack_t<Real>(cx, cdx, Rb, pack + (size_t)i * P4N);
}

// Camera block solves in FP64: the statistics summed over the camera's chunks, the
// accelerated S-CAM solve, the restart metrics and test, the MM solve, and the extrapolated
// rotation and pack of iteration k+1.
// The FP32 S-CAM path is held to 5 CTAs per SM (at most 168 registers, a few hundred bytes of
// spills): batches of many small scenes fill more than one wave of CTAs, and 10 instead of 8
// resident warps per SM shorten the second. The FP64 and LM paths would spill heavily and keep 255.
// One group of 32 cameras (cameras i0 + 32 grp .. i0 + 32 grp + 31, those below M) by two warps
// (role 0 and 1, lanes 0..31 each); sh_mm is the group's hand-over buffer in shared memory. Both warps of the CTA
// pass the barrier inside, so every thread of the CTA calls it the same number of times.
template <class Real, int SOLVER, bool COH>
__device__ __forceinline__ void camsolve_group(int grp, int role, int lane, double (*sh_mm)[16], int it, int first,
                                               int i0, int M, const int* __restrict__ cam_chunk_ptr,
                                               const Real* __restrict__ part, double* __restrict__ cam_x,
                                               double* __restrict__ cam_dx, double* __restrict__ cam_Rbar,
                                               const IterParams& P, double* __restrict__ cam_S,
                                               double* __restrict__ cam_E, double* __restrict__ cam_F,
                                               double* __restrict__ cam_Fb, uint8_t* __restrict__ cam_rs,
                                               double* __restrict__ cam_Fsum, V4<Real>* __restrict__ pack_next) {
  // 32 cameras per CTA, two warps: warp 0 takes the accelerated solve (Eq. update_amm) and
  // the restart test, warp 1 the MM solve (Eq. update_mm) of the same cameras; the MM solve is
  // computed whether or not the camera restarts, so that the two FP64 chains run side by side
  // instead of one after the other. Warp 1 hands its solution to warp 0 through shared memory.
  static_assert(CAMSOLVE_THREADS == 64, "two warps per CTA");
  using T = double;
  using N = Num<T>;
  const int i = i0 + grp * 32 + lane;
  const bool valid = i < M;
  const T xi = N::from(P.xi);
  CamT<T> ck, cn;
  T st[39];
  int c0 = 0, c1 = 0;
  double *x = nullptr, *dx = nullptr;
  T dx2 = N::c(0.f), dEn = N::c(0.f);
  if (valid) {
    c0 = cam_chunk_ptr[i];
    c1 = cam_chunk_ptr[i + 1];
    x = cam_x + (size_t)i * CSTRIDE;
    dx = cam_dx + (size_t)i * CSTRIDE;
#pragma unroll
    for (int a = 0; a < 9; ++a) ck.R[a] = N::from(ld_mut<COH>(x + CS_R + a));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ck.t[a] = N::from(ld_mut<COH>(x + CS_T + a));
      ck.d[a] = N::from(ld_mut<COH>(x + CS_D + a));
    }
    if (role == 1 || P.accelerated) {
      // One code path for both warps, so that they fetch the same instructions: warp 1 the MM
      // solve from x^k with the x^k statistics, warp 0 the accelerated solve from xbar^k with
      // the xbar statistics; both then evaluate their solution's decrease with the x^k statistics.
      CamT<T> c0s;
      if (role == 1) {
        c0s = ck;
      } else {
        const T gamma = N::from(P.gam[it]);
#pragma unroll
        for (int a = 0; a < 9; ++a) c0s.R[a] = N::from(ld_mut<COH>(cam_Rbar + (size_t)i * 9 + a));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          c0s.t[a] = ck.t[a] + gamma * N::from(ld_mut<COH>(dx + CS_T + a));
          c0s.d[a] = ck.d[a] + gamma * N::from(ld_mut<COH>(dx + CS_D + a));
        }
      }
      sum_stats<Real, T, COH>(part, c0, c1, role == 1 ? PART_XK : PART_XB, st);
      CamT<T> cs;
      cam_solve<SOLVER, Real>(st, c0s, xi, P.n_alt, cs);
      if (role == 0) sum_stats<Real, T, COH>(part, c0, c1, PART_XK, st);
      const T d = cam_phi(st, ck, cs, xi);   // E^alpha(solution | x^k) - E^alpha(x^k | x^k)
      if (role == 1) {
#pragma unroll
        for (int a = 0; a < 9; ++a) sh_mm[lane][a] = cs.R[a];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          sh_mm[lane][9 + a] = cs.t[a];
          sh_mm[lane][12 + a] = cs.d[a];
        }
        sh_mm[lane][15] = d;
      } else {
        cn = cs;
        dEn = d;
      }
    }
  }
  __syncthreads();
  if (role != 0 || !valid) return;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const T d = N::from(ld_mut<COH>(dx + CS_R + a));
    dx2 = dx2 + d * d;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T dt = N::from(ld_mut<COH>(dx + CS_T + a)), dd = N::from(ld_mut<COH>(dx + CS_D + a));
    dx2 = dx2 + dt * dt + dd * dd;
  }
  T sF = N::c(0.f), sG = N::c(0.f);
  for (int c = c0; c < c1; ++c) {
    acc_add(sF, ld_mut<COH>(part + (size_t)c * CP_STRIDE + PART_F));
    acc_add(sG, ld_mut<COH>(part + (size_t)c * CP_STRIDE + PART_G));
  }
  // Eq. DEalpha and the slack form of Eqs. Fak, lFak (see k_lpass)
  const T dE = N::c(-0.5f) * xi * dx2 + N::c(0.5f) * sG;
  const T S = first ? N::c(0.f) : N::from(ld_mut<COH>(cam_S + i));
  const T thr = N::from(P.eta1) * (S - dE);
  const bool global = P.accelerated && P.restart_global;
  const bool rs = P.accelerated ? (!global && dEn > thr) : true;
  const T E = first ? N::c(0.5f) * sF : N::from(ld_mut<COH>(cam_E + i));
  const T F = E + dE;
  if (global) {   // keep the MM alternative (warp 1's) and this block's term of the global test
    double* alt = P.cam_alt + (size_t)i * 32;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      alt[a] = N::to_double(sh_mm[lane][a]);
      alt[15 + a] = N::to_double(sh_mm[lane][a] - ck.R[a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      alt[9 + a] = N::to_double(sh_mm[lane][9 + a]);
      alt[12 + a] = N::to_double(sh_mm[lane][12 + a]);
      alt[24 + a] = N::to_double(sh_mm[lane][9 + a] - ck.t[a]);
      alt[27 + a] = N::to_double(sh_mm[lane][12 + a] - ck.d[a]);
    }
    alt[30] = N::to_double(F + sh_mm[lane][15]);
    alt[31] = N::to_double(thr - sh_mm[lane][15]);
    P.g_cam[i] = N::to_double(dEn - thr);
  }
  if (rs) {   // restart: the MM solution of warp 1
#pragma unroll
    for (int a = 0; a < 9; ++a) cn.R[a] = sh_mm[lane][a];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cn.t[a] = sh_mm[lane][9 + a];
      cn.d[a] = sh_mm[lane][12 + a];
    }
    dEn = sh_mm[lane][15];
  }
  cam_Fsum[i] = N::to_double(sF);   // sum of F_ij(x^k) over the camera's observations (objective trace)
  cam_F[i] = N::to_double(F);
  cam_Fb[i] = N::to_double(F + thr);
  cam_E[i] = N::to_double(F + dEn);
  cam_S[i] = N::to_double(thr - dEn);
  cam_rs[i] = (rs && P.accelerated) ? 1 : 0;
  CamT<T> ndx;
#pragma unroll
  for (int a = 0; a < 9; ++a) ndx.R[a] = cn.R[a] - ck.R[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ndx.t[a] = cn.t[a] - ck.t[a];
    ndx.d[a] = cn.d[a] - ck.d[a];
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    x[CS_R + a] = N::to_double(cn.R[a]);
    dx[CS_R + a] = N::to_double(ndx.R[a]);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    x[CS_T + a] = N::to_double(cn.t[a]);
    dx[CS_T + a] = N::to_double(ndx.t[a]);
    x[CS_D + a] = N::to_double(cn.d[a]);
    dx[CS_D + a] = N::to_double(ndx.d[a]);
  }
  // extrapolation of iteration k+1 (Eq. nesterov_R) and its pass pack
  const T gn = N::from(P.gam[it + 1]);
  T K[9], Rb[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) K[a] = cn.R[a] + gn * ndx.R[a];
  extrap_rotation<Real>(K, Rb);
#pragma unroll
  for (int a = 0; a < 9; ++a) cam_Rbar[(size_t)i * 9 + a] = N::to_double(Rb[a]);
  write_pack_t<Real>(cn, ndx, Rb, pack_next + (size_t)i * P4N);
}

template <class Real, int SOLVER>
__global__ void __launch_bounds__(CAMSOLVE_THREADS, (sizeof(Real) == 4 && SOLVER == CAM_SCAM) ? 5 : 1)
    k_camsolve(int i0, int M, const int* __restrict__ cam_chunk_ptr, const Real* __restrict__ part,
               double* __restrict__ cam_x, double* __restrict__ cam_dx, double* __restrict__ cam_Rbar, IterParams P,
               double* __restrict__ cam_S, double* __restrict__ cam_E, double* __restrict__ cam_F,
               double* __restrict__ cam_Fb, uint8_t* __restrict__ cam_rs, double* __restrict__ cam_Fsum,
               V4<Real>* __restrict__ pack_next) {
  // cameras i0 .. M - 1, 32 per CTA
  __shared__ double sh_mm[32][16];   // MM solution R(9) t(3) d(3) and its dEn
  camsolve_group<Real, SOLVER, false>(blockIdx.x, threadIdx.x >> 5, threadIdx.x & 31, sh_mm, *P.it, *P.first, i0, M,
                                      cam_chunk_ptr, part, cam_x, cam_dx, cam_Rbar, P, cam_S, cam_E, cam_F, cam_Fb,
                                      cam_rs, cam_Fsum, pack_next);
}

// ---------------------------------------------------------------------------
// 4. reduction of one iteration: F(x^k) = sum over cameras of their F_ij sums (FP64) and
//    the restart count. Every block reduces a fixed slice; the last block to finish (a
//    ticket counter, no waiting) combines the block results in block order.
// ---------------------------------------------------------------------------
constexpr int FIN_BLOCKS = 64;
constexpr int FIN_THREADS = 256;

__device__ __forceinline__ void block_sum2(double& f, long long& n, double* sf, long long* sn) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    f += __shfl_xor_sync(0xffffffffu, f, off);
    n += __shfl_xor_sync(0xffffffffu, n, off);
  }
  if ((threadIdx.x & 31) == 0) {
    sf[threadIdx.x >> 5] = f;
    sn[threadIdx.x >> 5] = n;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    f = 0.0;
    n = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      f += sf[w];
      n += sn[w];
    }
  }
}

// s^(k+1) = (sqrt(4 s^2 + 1) + 1) / 2 (Eq. nesterov_scalar) with every operation rounded
// separately (no contraction), as the host computes the table of a run
__device__ __forceinline__ double nesterov_next(double s) {
  return __dmul_rn(__dadd_rn(sqrt(__dadd_rn(__dmul_rn(__dmul_rn(4.0, s), s), 1.0)), 1.0), 0.5);
}

__global__ void __launch_bounds__(FIN_THREADS)
    k_finalize(int M, const double* __restrict__ cam_Fsum, const uint8_t* __restrict__ cam_rs, int n_tiles,
               const int* __restrict__ tile_rs, int n_blocks, double s2, IterParams P, double* __restrict__ blk,
               unsigned int* __restrict__ ticket, double* __restrict__ trace, int* __restrict__ restarts,
               int* __restrict__ flag) {
  __shared__ double sf[FIN_THREADS / 32];
  __shared__ long long sn[FIN_THREADS / 32];
  __shared__ bool last;
  double f = 0.0;
  long long n = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
    f += cam_Fsum[i];
    n += cam_rs[i];
  }
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += stride) n += tile_rs[t];
  block_sum2(f, n, sf, sn);
  const bool global = P.accelerated && P.restart_global;
  double g = 0.0;
  if (global && !P.fire_given) {   // global restart variant: sum over every block of E(k+1) - Fbar(k)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) g += P.g_cam[i];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += stride) g += P.g_tile[t];
    __syncthreads();   // thread 0 has read the first sums out of sf / sn
    long long dummy = 0;
    block_sum2(g, dummy, sf, sn);
  }
  if (threadIdx.x == 0) {
    blk[3 * blockIdx.x] = f;
    blk[3 * blockIdx.x + 1] = (double)n;
    blk[3 * blockIdx.x + 2] = g;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  // the last block's first warp combines the block results: lane l takes blocks l, l + 32, ...
  // in order, then a fixed shuffle tree (the same order on every run)
  __threadfence();
  double ft = 0.0, nt = 0.0, gt = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) {
    ft += ((volatile double*)blk)[3 * b];
    nt += ((volatile double*)blk)[3 * b + 1];
    if (global) gt += ((volatile double*)blk)[3 * b + 2];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ft += __shfl_xor_sync(0xffffffffu, ft, off);
    nt += __shfl_xor_sync(0xffffffffu, nt, off);
    gt += __shfl_xor_sync(0xffffffffu, gt, off);
  }
  if (threadIdx.x == 0) {
    const int k = *P.it;
    trace[k] = ft * s2;
    if (global) {
      // the test of Algorithm 1 for the block made of everything: sum E(k+1) > sum Fbar(k)
      const int fire = P.fire_given ? *P.g_fire : (gt > 0.0 ? 1 : 0);
      *P.g_fire = fire;
      restarts[k] = fire ? n_blocks : 0;
      if (P.reset_s) {   // Eq. nesterov_scalar continued on the device, s <- 1 after a restart
        const double s1 = fire ? 1.0 : nesterov_next(*P.s_dev);
        const double s2n = nesterov_next(s1), s3n = nesterov_next(s2n);
        *P.s_dev = s1;
        const_cast<double*>(P.gam)[k + 1] = __ddiv_rn(__dsub_rn(s1, 1.0), s2n);
        const_cast<double*>(P.gam)[k + 2] = __ddiv_rn(__dsub_rn(s2n, 1.0), s3n);
      }
    } else {
      restarts[k] = (int)nt;
    }
    if (!isfinite(ft)) atomicOr(flag, 1);
    *P.it = k + 1;
    *P.first = 0;
    *ticket = 0u;
  }
}

// ---------------------------------------------------------------------------
// 5. persistent path: the iterations of a run in one cooperative launch (MIXED, Algorithm 1 with
//    per-block restart and S-CAM). Every CTA is resident; grid barriers separate the camera
//    pass, the camera solves and landmark tiles, and the reduction. Data written earlier in the
//    launch is read through L2 (COH loads; TMA and cp.async.cg read L2 already).
// ---------------------------------------------------------------------------
constexpr int PERS_THREADS = 128;                    // 4 camera-pass warps / 2 camera-solve groups / 1 tile
constexpr long long GRID_BAR_NS = 2000000000ll;     // a grid barrier gives up after 2 s (flag bit 4)

__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }

// Barrier over the grid of a cooperative launch: thread 0 of each CTA arrives on a counter; the
// last arrival resets it and advances the generation, the others poll the generation, at most
// GRID_BAR_NS (then flag bit 4 is set and the CTA goes on, so the launch always ends).
__device__ __forceinline__ void grid_barrier(unsigned* count, unsigned* gen, int* flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = *(volatile unsigned*)gen;
    __threadfence();
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      while (*(volatile unsigned*)gen == g) {
        if ((long long)(globaltimer_ns() - t0) >= GRID_BAR_NS) {
          atomicOr(flag, 4);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

struct PersArgs {
  int M, n_chunks, n_tiles, tile_obs, n_small;   // tiles [0, n_small) hold up to tile_obs observations, the rest one long track
  const int *chunk_cam, *chunk_beg, *c_lm, *c_rpos, *cam_chunk_ptr, *tile_lm, *lm_ptr;
  const float2* c_u;
  const uint16_t* t_inv;
  V4<float>*pack[2];
  V4<float>*lmrec[2];
  V4<float>*lmlo[2];
  float* part;
  V4<float>*rec_a;
  V4<float>*rec_b;
  float* rec_c;
  double *cam_x, *cam_dx, *cam_Rbar, *cam_S, *cam_E, *cam_F, *cam_Fb, *cam_Fsum;
  uint8_t *cam_rs, *lm_rs;
  int* tile_rs;
  double *fin_blk, *trace;
  int* restarts;
  unsigned *bar_count, *bar_gen;
  double s2;   // s_norm^2
};

template <int LOSS>
__global__ void __launch_bounds__(PERS_THREADS, 3)
    k_run_persistent(PersArgs A, IterParams P, LossC<float> L, int n_iter, int par0) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sf[PERS_THREADS / 32], sf2[PERS_THREADS / 32];
  __shared__ long long sn[PERS_THREADS / 32], sn2[PERS_THREADS / 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int G = gridDim.x;
  const int first0 = *P.first;
  const int n_cs = (A.M + 63) / 64;   // camera-solve items: two groups of 32 cameras
  for (int j = 0; j < n_iter; ++j) {
    const int par = (par0 + j) & 1;
    const float gamma = float(P.gam[j]);
    const int first = j == 0 ? first0 : 0;
    // ---- camera pass: the grid's warps take the chunks
    {
      CpassWarpSmem<float, float2>* cw = reinterpret_cast<CpassWarpSmem<float, float2>*>(smem) + wib;
      for (int w = blockIdx.x * 4 + wib; w < A.n_chunks; w += G * 4)
        cpass_chunk<LOSS, float, float2, true>(w, lane, *cw, gamma, A.chunk_cam, A.chunk_beg, A.c_lm, A.c_u,
                                               A.pack[par], A.lmrec[par], L, A.part, A.c_rpos, A.rec_a, A.rec_b,
                                               A.rec_c);
    }
    fence_proxy_async_global();   // the records written above are read by bulk copies (async proxy)
    grid_barrier(A.bar_count, A.bar_gen, P.flag);
    fence_proxy_async_global();
    // ---- camera solves (items 0 .. n_cs) and landmark tiles (the rest), strided over the CTAs
    {
      LpassOut<float> O;
      O.lmrec_out = A.lmrec[par ^ 1];
      O.lm_lo_out = A.lmlo[par ^ 1];
      O.lm_rs = A.lm_rs;
      O.lm_Fdiag = nullptr;
      O.lm_Fbdiag = nullptr;
      O.lm_alt = nullptr;
      O.lm_sums = nullptr;
      for (int item = blockIdx.x; item < n_cs + A.n_tiles; item += G) {
        if (item < n_cs) {
          double(*sh)[16] = reinterpret_cast<double(*)[16]>(smem) + (wib >> 1) * 32;
          camsolve_group<float, CAM_SCAM, true>(2 * item + (wib >> 1), wib & 1, lane, sh, j, first, 0, A.M,
                                                A.cam_chunk_ptr, A.part, A.cam_x, A.cam_dx, A.cam_Rbar, P, A.cam_S,
                                                A.cam_E, A.cam_F, A.cam_Fb, A.cam_rs, A.cam_Fsum, A.pack[par ^ 1]);
          __syncthreads();   // the hand-over buffers are read before the next item reuses the memory
        } else {
          const int tile = item - n_cs;
          lpass_tile<float, float2, true, true>(tile, tile < A.n_small ? A.tile_obs : BIG_TILE_OBS, smem, gamma, first,
                                                A.tile_lm, A.lm_ptr, A.t_inv, A.rec_a, A.rec_b, A.rec_c, A.lmrec[par], A.lmlo[par], P,
                                                A.tile_rs, O);
        }
      }
    }
    grid_barrier(A.bar_count, A.bar_gen, P.flag);
    // ---- reduction: F(x^k) and the restart count in the order of k_finalize (FIN_BLOCKS blocks
    // of FIN_THREADS threads: each of these threads computes two of them, and the warp trees run
    // over the same lanes, so the trace has the same bits as on the graph path)
    static_assert(FIN_THREADS == 2 * PERS_THREADS, "two reduction threads per thread");
    for (int fb = blockIdx.x; fb < FIN_BLOCKS; fb += G) {   // the reduction block fb of k_finalize
      double f[2] = {0.0, 0.0};
      long long n[2] = {0, 0};
      const int stride = FIN_BLOCKS * FIN_THREADS;
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int vt = threadIdx.x + v * PERS_THREADS;   // the k_finalize thread emulated
        for (int i = fb * FIN_THREADS + vt; i < A.M; i += stride) {
          f[v] += ld_mut<true>(A.cam_Fsum + i);
          n[v] += ld_mut<true>(A.cam_rs + i);
        }
        for (int t = fb * FIN_THREADS + vt; t < A.n_tiles; t += stride) n[v] += ld_mut<true>(A.tile_rs + t);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          f[v] += __shfl_xor_sync(0xffffffffu, f[v], off);
          n[v] += __shfl_xor_sync(0xffffffffu, n[v], off);
        }
      }
      if (lane == 0) {   // warp results of the emulated warps wib and wib + 4
        sf[wib] = f[0];
        sn[wib] = n[0];
        sf2[wib] = f[1];
        sn2[wib] = n[1];
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double ft = 0.0;
        long long nt = 0;
        for (int w = 0; w < FIN_THREADS / 32; ++w) {
          ft += w < 4 ? sf[w] : sf2[w - 4];
          nt += w < 4 ? sn[w] : sn2[w - 4];
        }
        A.fin_blk[3 * fb] = ft;
        A.fin_blk[3 * fb + 1] = (double)nt;
      }
      __syncthreads();   // sf / sn are read before the next block's warps write them
    }
    grid_barrier(A.bar_count, A.bar_gen, P.flag);
    if (blockIdx.x == 0 && threadIdx.x < 32) {
      double ft = 0.0, nt = 0.0;
      for (int b = threadIdx.x; b < FIN_BLOCKS; b += 32) {
        ft += ld_mut<true>(A.fin_blk + 3 * b);
        nt += ld_mut<true>(A.fin_blk + 3 * b + 1);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        ft += __shfl_xor_sync(0xffffffffu, ft, off);
        nt += __shfl_xor_sync(0xffffffffu, nt, off);
      }
      if (threadIdx.x == 0) {
        A.trace[j] = ft * A.s2;
        A.restarts[j] = (int)nt;
        if (!isfinite(ft)) atomicOr(P.flag, 1);
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *P.it = n_iter;
    *P.first = 0;
  }
}

// Global restart variant, after the reduction: when the test fired, every camera takes the MM
// alternative kept by the camera solve, with its restart metrics, the extrapolated rotation of
// iteration k+1 and the pass pack (gamma^(k+1) read after the reduction advanced the counter;
// 0 after a momentum reset).
template <class Real>
__global__ void k_fix_cams(int M, IterParams P, double* __restrict__ cam_x, double* __restrict__ cam_dx,
                           double* __restrict__ cam_Rbar, double* __restrict__ cam_S, double* __restrict__ cam_E,
                           uint8_t* __restrict__ cam_rs, V4<Real>* __restrict__ pack_next) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M || !*P.g_fire) return;
  const double* a = P.cam_alt + (size_t)i * 32;
  CamT<double> cn, ndx;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    cn.R[q] = a[q];
    ndx.R[q] = a[15 + q];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    cn.t[q] = a[9 + q];
    cn.d[q] = a[12 + q];
    ndx.t[q] = a[24 + q];
    ndx.d[q] = a[27 + q];
  }
  double* x = cam_x + (size_t)i * CSTRIDE;
  double* dx = cam_dx + (size_t)i * CSTRIDE;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    x[CS_R + q] = cn.R[q];
    dx[CS_R + q] = ndx.R[q];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    x[CS_T + q] = cn.t[q];
    dx[CS_T + q] = ndx.t[q];
    x[CS_D + q] = cn.d[q];
    dx[CS_D + q] = ndx.d[q];
  }
  cam_E[i] = a[30];
  cam_S[i] = a[31];
  cam_rs[i] = 1;
  const double gn = P.gam[*P.it];
  double K[9], Rb[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) K[q] = cn.R[q] + gn * ndx.R[q];
  extrap_rotation<Real>(K, Rb);
#pragma unroll
  for (int q = 0; q < 9; ++q) cam_Rbar[(size_t)i * 9 + q] = Rb[q];
  write_pack_t<Real>(cn, ndx, Rb, pack_next + (size_t)i * P4N);
}

// Global restart variant: when the test fired, every landmark takes its MM alternative, stepped
// from l^k as the landmark pass steps (double-float in MIXED).
template <class Real, bool HAS_LO>
__global__ void k_fix_lms(int N, IterParams P, const V4<Real>* __restrict__ lmrec, const V4<float>* __restrict__ lm_lo,
                          const V4<Real>* __restrict__ lm_alt, V4<Real>* __restrict__ lmrec_out,
                          V4<float>* __restrict__ lm_lo_out, uint8_t* __restrict__ lm_rs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N || !*P.g_fire) return;
  const size_t g = (size_t)j;
  const V4<Real> A = lmrec[2 * g];
  const V4<Real> a0 = lm_alt[2 * g], a1 = lm_alt[2 * g + 1];
  V4<Real> nA, nB = lmrec_out[2 * g + 1];
  if (HAS_LO) {
    const V4<float> lo0 = lm_lo[g];
    float h0 = float(A.x), h1 = float(A.y), h2 = float(A.z);
    float o0 = lo0.x, o1 = lo0.y, o2 = lo0.z;
    df_add(h0, o0, float(a0.x));
    df_add(h1, o1, float(a0.y));
    df_add(h2, o2, float(a0.z));
    nA.x = Real(h0);
    nA.y = Real(h1);
    nA.z = Real(h2);
    V4<float> nlo;
    nlo.x = o0;
    nlo.y = o1;
    nlo.z = o2;
    nlo.w = 0.f;
    lm_lo_out[g] = nlo;
  } else {
    nA.x = A.x + a0.x;
    nA.y = A.y + a0.y;
    nA.z = A.z + a0.z;
    nB.w = a1.x;
  }
  nA.w = a0.x;
  nB.x = a0.y;
  nB.y = a0.z;
  nB.z = a0.w;
  lmrec_out[2 * g] = nA;
  lmrec_out[2 * g + 1] = nB;
  lm_rs[g] = 1;
}

// ---------------------------------------------------------------------------
// objective F(x^k) only (Eq. Fobj): camera-sorted chunks, landmark position from its
// high and low parts; one partial per chunk
// ---------------------------------------------------------------------------
template <int LOSS, class Real, class Real2, bool HAS_LO>
__global__ void __launch_bounds__(CPASS_WARPS * 32)
    k_objective(int n_chunks, const int* __restrict__ chunk_cam, const int* __restrict__ chunk_beg,
                const int* __restrict__ c_lm, const Real2* __restrict__ c_u, const V4<Real>* __restrict__ pack,
                const V4<Real>* __restrict__ lmrec, const V4<float>* __restrict__ lm_lo, LossC<Real> L,
                Real* __restrict__ chunk_f) {
  __shared__ V4<Real> spk[CPASS_WARPS][P4N];
  const int wib = threadIdx.x >> 5;
  const int warp = blockIdx.x * CPASS_WARPS + wib;
  const int lane = threadIdx.x & 31;
  if (warp >= n_chunks) return;
  const int cam = chunk_cam[warp];
  const int b = chunk_beg[warp], e = chunk_beg[warp + 1];
  if (lane < P4N) spk[wib][lane] = pack[(size_t)cam * P4N + lane];
  __syncwarp();
  Real f = Real(0);
  for (int o = b + lane; o < e; o += 32) {
    const int j = c_lm[o];
    const Real2 uu = c_u[o];
    const V4<Real> A = lmrec[2 * (size_t)j];
    Real o0 = Real(0), o1 = Real(0), o2 = Real(0);
    if (HAS_LO) {
      const V4<float> lo = lm_lo[j];
      o0 = Real(lo.x);
      o1 = Real(lo.y);
      o2 = Real(lo.z);
    }
    f += eval_F4<LOSS, Real>(spk[wib], A.x, A.y, A.z, o0, o1, o2, uu.x, uu.y, L);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
  if (lane == 0) chunk_f[warp] = f;
}

// FP64 sum of n values (one block, fixed order) times s2 into *out
template <class Real>
__global__ void k_sum(int n, const Real* __restrict__ v, double s2, double* __restrict__ out) {
  __shared__ double red[32];
  double f = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) f += double(v[t]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    double ft = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) ft += red[w];
    *out = ft * s2;
  }
}

// F per segment of chunks (a batch of independent scenes: one block per scene, its chunks
// summed in FP64 in a fixed order) times s2 into out[scene]
template <class Real>
__global__ void k_segment_sum(const int* __restrict__ seg_ptr, const Real* __restrict__ v, double s2,
                              double* __restrict__ out) {
  __shared__ double red[32];
  const int b = seg_ptr[blockIdx.x], e = seg_ptr[blockIdx.x + 1];
  double f = 0.0;
  for (int t = b + threadIdx.x; t < e; t += blockDim.x) f += widen(v[t]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    double ft = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) ft += red[w];
    out[blockIdx.x] = ft * s2;
  }
}

}  // namespace daba
