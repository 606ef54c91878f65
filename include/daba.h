/*
 * daba.h -- C ABI of the B300 (sm_103a) implementation of one accelerated
 * majorization-minimization iteration of DABA (Decentralized and Accelerated
 * Bundle Adjustment, arXiv 2305.07026) and the loop of Algorithm 1 around it.
 *
 * Problem (Sec. 2, Problem 1): minimise F(x) = sum_{(i,j) in E} rho(|e_ij|^2)/2
 * over cameras c_i = (R_i, t_i, d_i) and landmarks l_j, with the reprojection
 * error e_ij of Sec. 3 (Eq. error) and a robust loss rho satisfying
 * Assumption 1 (App. B). Each call below is one piece of Algorithm 1 (Sec. 6):
 * every camera and every landmark is its own block, so every reprojection pair
 * is split by the majorizer of Proposition 1 into P_ij(c_i|x^k) + Q_ij(l_j|x^k)
 * (Eq. Ealpha with E' empty), the blocks are solved independently (Eqs.
 * update_amm / update_mm), and Nesterov extrapolation (Eq. nesterov_x) runs
 * with the per-block adaptive restart of Sec. 5 (Eqs. DEalpha-Eak).
 *
 * Conventions shared by every entry point
 *  - Pointers are caller-owned. Unless stated otherwise an array argument may be
 *    host memory or device memory of the context's GPU; the library detects
 *    which with cudaPointerGetAttributes and copies host arrays through its own
 *    device buffers (pageable or pinned host memory both work).
 *  - All GPU work is ordered on the cudaStream_t passed as `stream` (NULL means
 *    the legacy default stream). Calls return after the work is enqueued, except
 *    where a host output is written, which waits for that stream.
 *  - Errors are returned as daba_status; a failing call leaves the iterate,
 *    the restart metrics and the observations unchanged, and
 *    daba_last_error() returns a one-line reason. No exception crosses the ABI.
 *  - A context is not thread-safe; use one per host thread.
 *
 * Units. Pixels are measured from the principal point. Internally every pixel
 * quantity is divided by s_norm (options.pixel_scale, 0 = median focal length
 * of the first state set): an exact reparameterisation, so objective values
 * returned by the library are in pixel^2.
 */
#ifndef DABA_H_
#define DABA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DABA_OK = 0,
  DABA_ERR_ARG = 1,         /* invalid size, option or null pointer */
  DABA_ERR_INDEX = 2,       /* observation index out of range */
  DABA_ERR_DEGENERATE = 3,  /* |l_j - t_i| <= epsilon for an observed pair (Assumption 2) */
  DABA_ERR_NONFINITE = 4,   /* non-finite input value, or the iterate became non-finite */
  DABA_ERR_CUDA = 5,        /* a CUDA runtime call failed */
  DABA_ERR_OOM = 6,         /* device allocation failed */
  DABA_ERR_STATE = 7,       /* call out of order (e.g. run before observations and state are set) */
  DABA_ERR_TIMEOUT = 8      /* a bounded wait inside a kernel ran out (see daba_set_wait_limit) */
} daba_status;

/* Robust losses of Assumption 1 (App. B); `loss_scale_px` is c below, in pixels.
 * TRIVIAL rho(s)=s; HUBER s if s<=c^2 else 2c sqrt(s)-c^2; CAUCHY c^2 log(1+s/c^2);
 * WELSCH c^2 (1-exp(-s/c^2)). */
typedef enum { DABA_LOSS_TRIVIAL = 0, DABA_LOSS_HUBER = 1, DABA_LOSS_CAUCHY = 2, DABA_LOSS_WELSCH = 3 } daba_loss;

/* DABA_FP64: every quantity in FP64.
 * DABA_MIXED: per-observation residuals, weights and majorizer terms in FP32; the
 * per-camera sums across warps, the camera state and the camera restart metrics in FP64;
 * the camera subproblem solve (S-CAM) and the extrapolated rotation in FP32 on displacements
 * from the FP64 state; landmark solves and metrics in FP32 with double-float positions. */
typedef enum { DABA_FP64 = 0, DABA_MIXED = 1 } daba_precision;

typedef struct {
  daba_loss loss;
  double loss_scale_px;   /* loss scale c in pixels (ignored for TRIVIAL) */
  double xi;              /* proximal weight xi > 0 of Eq. Ealpha, internal units (default 1e-10) */
  double eta;             /* 0 < eta <= 1 of Eq. lFak (default 0.5) */
  int accelerated;        /* 1: DABA (Algorithm 1); 0: DUBA, always the MM update (Sec. 7.2) */
  int cam_alternations;   /* R-step / (t,d)-step alternations of the camera block solve (default 2) */
  double pixel_scale;     /* s_norm in pixels; 0 = median focal length of the first state set */
  daba_precision prec;
  /* work schedule (0 = default; results do not depend on it except for the order of FP
   * sums): observations per camera-pass chunk (32..65536, default 2048), observations per
   * landmark tile (32..2048, default 512) and landmarks per tile (1..128, default 128). */
  int32_t chunk_obs;
  int32_t tile_obs;
  int32_t tile_lms;
  /* restart test (method variant; default DABA_RESTART_BLOCK, Algorithm 1): with
   * DABA_RESTART_GLOBAL one test decides for all blocks, sum_alpha E^alpha(k+1) >
   * sum_alpha Fbar^alpha(k) (the test of Algorithm 1 for the single block made of every camera
   * and landmark, whose metrics are the sums because Eqs. Fak, lFak, Eak are linear); when it
   * fires every block takes its MM update (Eq. update_mm). momentum_reset = 1 (global only)
   * also restarts Nesterov's scalar: s^(k+1) = 1 after an iteration whose test fired. */
  int32_t restart_mode;
  int32_t momentum_reset;
  /* camera block solver (method variant; default DABA_CAM_SCAM): DABA_CAM_SCAM runs
   * cam_alternations block-exact alternations (R-step: ProjRot3D, (t, d)-step: normal
   * equations); DABA_CAM_LM takes one successful Levenberg-Marquardt step (Sec. 7.1 reports one
   * successful inner LM step per subproblem) on the Gauss-Newton model in R_z Exp(phi), t, d,
   * damping 1e-3 x diag, raised tenfold up to 8 times, the step kept only if E^alpha(. | z)
   * decreases. */
  int32_t cam_solver;
} daba_options;

typedef enum { DABA_CAM_SCAM = 0, DABA_CAM_LM = 1 } daba_cam_solver;

typedef enum { DABA_RESTART_BLOCK = 0, DABA_RESTART_GLOBAL = 1 } daba_restart_mode;

typedef struct daba_ctx daba_ctx;

/* Fills `opt` with the defaults listed above (Huber, c = 1 px, MIXED). */
void daba_default_options(daba_options* opt);

/* Creates a context for M cameras, N landmarks and nnz observations and allocates
 * all device memory it will use (O(M + N + nnz)) on the current CUDA device.
 * M >= 1, N >= 1, 1 <= nnz < 2^31. On success *out owns the memory until
 * daba_destroy. */
daba_status daba_create(int32_t M, int32_t N, int64_t nnz, const daba_options* opt, daba_ctx** out);

/* Sets the observation list E (Problem 1): cam_idx[k] in [0, M), lm_idx[k] in [0, N),
 * uv[2k], uv[2k+1] the observed distorted pixel u_ij (Sec. 3) relative to the
 * principal point, row-major nnz x 2. The library sorts the observations stably
 * by camera and by landmark (ties keep input order) and builds its CSR offsets
 * and work schedules (setup, not part of an iteration). Resets the iteration
 * count and the restart metrics. At most 2048 observations per landmark (DABA_ERR_ARG otherwise). */
daba_status daba_set_observations(daba_ctx* ctx, const int32_t* cam_idx, const int32_t* lm_idx,
                                  const double* uv, void* stream);

/* Sets the iterate x^(0) = x^(-1) (Algorithm 1, initialisation) and resets s^(0) = 1
 * and the restart metrics (Eq. Fainit).
 * cams: M x 9 row-major [w(3), t(3), f, k1, k2]: w is the axis-angle vector of the
 *   camera-to-world rotation R_i (a point l has camera-frame coordinates
 *   R_i^T (l - t_i)), t_i the camera centre, f the focal length in pixels, k1, k2
 *   the radial undistortion coefficients on |u|/f, i.e. the undistorted ray is
 *   [u/f, 1 + k1 |u/f|^2 + k2 |u/f|^4] (Eq. reprojection1 with d = (f, k1/f, k2/f^3)).
 * lms: N x 3 row-major landmark positions. Returns DABA_ERR_NONFINITE on NaN/Inf. */
daba_status daba_set_state(daba_ctx* ctx, const double* cams, const double* lms, void* stream);

/* Runs `iters` >= 0 iterations of Algorithm 1 from the current iterate x^k.
 * obj_trace (iters + 1 doubles, host or device, may be NULL): F(x^k), ...,
 *   F(x^(k+iters)) in pixel^2 (Eq. Fobj). F(x^(k+iters)) needs one extra objective pass,
 *   which is skipped when obj_trace is NULL.
 * restarts (iters int32, host or device, may be NULL): number of blocks whose
 *   adaptive restart fired in each iteration (Algorithm 1, restart test).
 * Requires observations and state to be set (DABA_ERR_STATE otherwise). Returns
 * DABA_ERR_NONFINITE if the objective became non-finite and DABA_ERR_TIMEOUT if a landmark-pass
 * wait on its tile copies ran out (daba_set_wait_limit). Any failure after the first launch puts
 * back the entry state: the iterate x^k, x^(k-1), s^k, k, the restart metrics and the per-block
 * diagnostics of daba_get_block_metrics are then those from before the call. To do so the call
 * copies that state (device to device, on `stream`) before its first launch; a run of one
 * iteration copies only the camera part, because it does not overwrite the landmark buffer of x^k.
 * Waits for the stream before returning (the status needs the device's answer). */
daba_status daba_run(daba_ctx* ctx, int32_t iters, double* obj_trace, int32_t* restarts, void* stream);

/* Objective F(x^k) of the current iterate in pixel^2 (Eq. Fobj), written to *out
 * (host or device double). */
daba_status daba_objective(daba_ctx* ctx, double* out, void* stream);

/* F(x^k) (Eq. Fobj, pixel^2) and its gradient w.r.t. the boundary parameters, by adjoint
 * kernels of the per-observation gradients of Eq. DFij (App. D):
 *   F:      1 double;
 *   g_cams: M x 9, d F / d [w(3), t(3), f, k1, k2] of daba_set_state (the rotation part is
 *           w.r.t. the axis-angle vector of norm <= pi that daba_get_state returns);
 *   g_lms:  N x 3, d F / d l_j;
 *   g_uv:   nnz x 2, d F / d u_ij (input observation order).
 * Each output may be NULL, host or device memory. Evaluated in the context's precision
 * (MIXED: FP32 per observation, FP64 per-camera and per-landmark sums). Uses the library's
 * scratch buffers: do not overlap with daba_run on another stream. */
daba_status daba_objective_grad(daba_ctx* ctx, double* F, double* g_cams, double* g_lms, double* g_uv,
                                void* stream);

/* Reverse-mode derivative of K >= 1 iterations of Algorithm 1 (Eqs. nesterov_scalar,
 * nesterov_x, nesterov_R, the majorizer of Proposition 1, the closed-form landmark update and
 * S-CAM, or with cam_solver = DABA_CAM_LM the LM step, for the cameras) from the state last set
 * by daba_set_state (x^0 = x^(-1)).
 * With y = <seed_cams, cams_K> + <seed_lms, lms_K> for the boundary state (cams_K, lms_K)
 * after K iterations (the layout of daba_get_state), writes
 *   g_cams: M x 9, dy / d cams_0 (the layout of daba_set_state);
 *   g_lms:  N x 3, dy / d lms_0;
 *   g_uv:   nnz x 2, dy / d u_ij (input observation order).
 * The per-block restart decisions, and with the LM solver the damping trial each camera's step
 * took (or that it took none), are piecewise constant and are held at those of the forward run. Runs the K iterations itself (leaving the state at x^K, as daba_run(K)
 * would), keeps the state every 10 iterations and, per segment of 10 iterations from the last,
 * runs the segment again keeping each iteration's state, camera statistics, landmark sums and
 * decisions; it costs about two forward runs plus the adjoint kernels and holds about K/10 + 11
 * copies of the state and 10 of the per-iteration data (about 64 B per landmark). Seeds and
 * outputs: host or device memory; outputs may be NULL. A MIXED context differentiates its own
 * trajectory: its forward run keeps all K + 1 iterates (widened to FP64) and every iteration's
 * restart decisions; then, per iteration from the last, an FP64 context that it owns (same
 * observations and pixel unit, created on first use, kept until destroy) re-forms that
 * iteration's statistics in FP64 at the MIXED iterate and runs the FP64 adjoint kernels with the
 * MIXED decisions. It needs pixels set from host memory (DABA_ERR_STATE otherwise) and holds
 * K + 1 FP64 states. With momentum_reset, the Nesterov scalars the device continued (s = 1 after
 * a global restart) are read back after every forward iteration and replayed with the restart
 * decisions. DABA_ERR_STATE if iterations have run since the state was set. */
daba_status daba_unrolled_grad(daba_ctx* ctx, int32_t K, const double* seed_cams, const double* seed_lms,
                               double* g_cams, double* g_lms, double* g_uv, void* stream);

/* Replaces the observed pixels (nnz x 2, input observation order, host or device) without
 * re-sorting: the observation list stays that of daba_set_observations. Requires the state to
 * be set (the internal unit s is fixed by then). DABA_ERR_NONFINITE on NaN/Inf. */
daba_status daba_set_pixels(daba_ctx* ctx, const double* uv, void* stream);

/* Copies the current iterate x^k out in the boundary layout of daba_set_state
 * (either pointer may be NULL to skip it). */
daba_status daba_get_state(daba_ctx* ctx, double* cams, double* lms, void* stream);

/* Per-block restart metrics after the last iteration (each pointer may be NULL):
 *   F_cam[M], F_lm[N]        F^alpha(k) of Eq. Fak (pixel^2) of the last iteration k,
 *   Fbar_cam[M], Fbar_lm[N]  Fbar^alpha(k) of Eq. lFak (pixel^2),
 *   rs_cam[M], rs_lm[N]      1 where the restart test fired in that iteration.
 * F and Fbar of landmarks are reported only for DABA_FP64 (DABA_ERR_STATE otherwise). */
daba_status daba_get_block_metrics(daba_ctx* ctx, double* F_cam, double* Fbar_cam, double* F_lm,
                                   double* Fbar_lm, uint8_t* rs_cam, uint8_t* rs_lm, void* stream);

/* The sort orders and CSR offsets built by daba_set_observations (each may be NULL):
 *   cam_order[nnz]: input indices sorted stably by camera; cam_ptr[M+1] its offsets;
 *   lm_order[nnz]:  input indices sorted stably by landmark; lm_ptr[N+1] its offsets. */
daba_status daba_get_sort(daba_ctx* ctx, int32_t* cam_order, int32_t* cam_ptr, int32_t* lm_order,
                          int32_t* lm_ptr, void* stream);

/* Declares the problem a batch of independent scenes: cameras [cam_begin[s], cam_begin[s+1])
 * form scene s (cam_begin[0] = 0, cam_begin[n_scenes] = M, non-decreasing; host array of
 * n_scenes + 1 int32), and each landmark belongs to the scene of the cameras observing it
 * (DABA_ERR_ARG if a landmark is observed from two scenes). With every camera and landmark a
 * block of its own (Sec. 5), blocks of different scenes share no term, and the Nesterov
 * scalars (Eq. nesterov_scalar) depend only on k, so one daba_run iteration over the batch is
 * one iteration of Algorithm 1 for every scene at once; results equal those of separate runs
 * with the same pixel_scale. Call after daba_set_observations (which clears the partition).
 * DABA_ERR_STATE before observations are set. */
daba_status daba_set_scenes(daba_ctx* ctx, int32_t n_scenes, const int32_t* cam_begin);

/* F(x^k) of every scene of the batch (Eq. Fobj over the scene's observations), pixel^2, into
 * out[n_scenes] (host or device doubles). DABA_ERR_STATE without a scene partition. */
daba_status daba_scene_objectives(daba_ctx* ctx, double* out, void* stream);

/* Checkpoint of the full method state (x^k, x^k - x^(k-1), s^k, k and the per-block
 * restart metrics; with coarse blocks also E^alpha, Fbar^alpha, F^alpha and the restart flag of
 * every block, and a fingerprint of the partition) into a host buffer. With buf == NULL only
 * *bytes is set to the required size. Importing it into a context with the same sizes, options,
 * observations and partition resumes bit-identically (DABA_ERR_ARG for another partition). */
daba_status daba_export_checkpoint(daba_ctx* ctx, void* buf, size_t* bytes);
daba_status daba_import_checkpoint(daba_ctx* ctx, const void* buf, size_t bytes);

/* Device-time breakdown of the last daba_run (milliseconds, summed over its
 * iterations) for the kernels of one iteration, in the order:
 * [0] camera prepare of the first iteration (extrapolation, Eq. nesterov_x), [1] camera-sorted observation pass,
 * [2] landmark-sorted observation pass + landmark solves, [3] camera solves + next extrapolation, [4] reduction.
 * Timing is recorded only when enabled with daba_set_timing(ctx, 1): a run of at most 256
 * iterations is then its own graph with an event-record node around every kernel (the nodes
 * lengthen each iteration by some tens of microseconds), a longer run is launched directly with
 * events. Results do not depend on it. */
daba_status daba_set_timing(daba_ctx* ctx, int enable);
daba_status daba_get_timing(daba_ctx* ctx, double* ms5);

/* Limit of the landmark pass's first wait on its tile copies (the bulk copies into shared
 * memory complete on an mbarrier that the CTA polls against the %globaltimer clock), in
 * nanoseconds; default 1e9 (1 s). When the limit runs out the CTA records it, waits up to 2 s more
 * for its copies to land, skips its tile and daba_run returns DABA_ERR_TIMEOUT with the entry
 * state restored; the context stays usable. 0 gives up before the first poll, which makes every
 * landmark pass report a timeout (a test of that path). DABA_ERR_ARG if first_wait_ns < 0. */
daba_status daba_set_wait_limit(daba_ctx* ctx, int64_t first_wait_ns);

/* Coarse blocks (Sec. 4, Eq. Ealpha with E' not empty; FP64 contexts):
 * block b holds the cameras i with cam_block[i] = b (at most 512 per block, none allowed) and the
 * landmarks j with lm_block[j] = b (host or device int32 arrays of M and N entries, block ids in
 * [0, n_blocks), 1 <= n_blocks <= M + N). A reprojection pair whose camera and landmark share a
 * block keeps its exact F_ij in the block's surrogate; every other pair is split by the majorizer
 * of Proposition 1 into P_ij (camera's block) and Q_ij (landmark's block). Each iteration of
 * Algorithm 1 then takes, per block, one successful Levenberg-Marquardt step on
 * E^alpha(. | xbar^k) from xbar^k (Sec. 7.1 reports one successful inner LM step per
 * subproblem), the per-block restart test of Eq. Eak, and where it fires the LM step on
 * E^alpha(. | x^k) from x^k. With restart_mode = DABA_RESTART_GLOBAL one test on the sums over
 * the blocks decides for all of them (every block's accelerated step is kept, the test runs, then
 * every block commits its kept step or takes the MM step), with momentum_reset also s <- 1. LM step: R = R_z Exp(phi), t = t_z + tau, d = d_z + delta,
 * l = l_z + epsilon; Gauss-Newton model of the block surrogate (the intra pairs reweighted with
 * w = rho'(|e|^2) at z, the proximal term to second order); damping 1e-3 x diag, raised tenfold
 * up to 8 times; taken only if E^alpha(. | z) decreases. The damped system is solved through the
 * Schur complement of the block's cameras (9 per camera; every landmark's 3 x 3 block
 * eliminated), with a dense Cholesky factorisation, by one CTA per block (scratch in shared memory
 * up to 16 cameras, in global memory above) or by a thread-block cluster per block over global
 * scratch (daba_set_block_ctas; about (9 n_c)^3 / 3 FP64 multiply-adds per damping trial). The restart metrics of Eqs. DEalpha-Eak are per block
 * (daba_get_partition_metrics); the restart count of daba_run counts the blocks that hold a
 * camera. A camera may observe each landmark of its block at most once (DABA_ERR_ARG otherwise,
 * as for a block id out of range or a block of more than 512 cameras). Call after
 * daba_set_observations (which clears the partition); n_blocks = 0 returns to one block per
 * camera and per landmark (the arrays are then ignored). The device scratch grows with the
 * partition: 888 bytes per intra pair, 248 per landmark, and with global scratch 1752 bytes per
 * camera plus (9 n_c)^2 x 8 bytes per block. Checkpoints carry the partition's block metrics;
 * the unrolled gradient is not available while a partition is set. */
daba_status daba_set_partition(daba_ctx* ctx, int32_t n_blocks, const int32_t* cam_block, const int32_t* lm_block);

/* How the next daba_set_partition spreads a block over CTAs (Algorithm 1 with coarse blocks, its
 * results the same up to the rounding order of the block's sums): 0 (default) automatic: one CTA
 * per block, its scratch in shared memory, when every block has at most 16 cameras and there are
 * more than n_SM / 2 blocks, else a thread-block cluster of up to 16 CTAs per block (as many as
 * keep the grid within two CTAs per SM) over global scratch; 1: one CTA per block (shared
 * scratch up to 16 cameras, global above); 2..16: a cluster of at most that many CTAs per block
 * over global scratch (the largest of 16, 8, 4, 2 not above it that the device can place).
 * DABA_ERR_ARG outside 0..16. Takes effect at the next daba_set_partition. */
daba_status daba_set_block_ctas(daba_ctx* ctx, int32_t ctas);

/* Per-block metrics of the last iteration with a partition (each pointer may be NULL, n_blocks
 * entries, host or device): F^alpha(k) (Eq. Fak) and Fbar^alpha(k) (Eq. lFak) in pixel^2 and the
 * restart flag. DABA_ERR_STATE without a partition. */
daba_status daba_get_partition_metrics(daba_ctx* ctx, double* F_blk, double* Fbar_blk, uint8_t* rs_blk, void* stream);

/* Persistent path (enable = 1): daba_run then launches, after the prepare kernel of its first
 * iteration, all its iterations (up to 1024 per launch) as ONE cooperative kernel whose CTAs
 * are all resident and loop over the work of every iteration, with grid-wide barriers (bounded
 * by a 2 s clock limit each; a run-out gives DABA_ERR_TIMEOUT) between the camera pass, the
 * camera solves with the landmark tiles, and the reduction; a batch of scenes set with
 * daba_set_scenes then runs all its iterations in one launch. The iterates, per-block metrics and
 * objective trace are the same bits as on the default path (CUDA graphs of the separate
 * kernels). The default path is the faster one on B300: one kernel must hold the largest register
 * footprint of the three phases (168 registers, 3 CTAs of 128 threads per SM), which starves the
 * landmark pass of the CTAs that keep its copies in flight (512-scene batch, 100 iterations:
 * 70.4 ms persistent against 38.0 ms; 26M-observation scene: 1.28 against 0.76 ms per
 * iteration). MIXED contexts with per-block restart and S-CAM only (DABA_ERR_ARG otherwise);
 * per-kernel timing does not apply. */
daba_status daba_set_persistent(daba_ctx* ctx, int enable);

/* Range schedule of each iteration (a schedule option like chunk_obs: the iterates, metrics and
 * objective trace are the same bits with it and without it; no paper counterpart). The cameras
 * are cut into `ranges` ranges of about equal observation counts (camera order; a camera is never
 * split, so heavy cameras can leave fewer ranges). The camera pass runs range by range; the camera
 * solves of a range start as soon as its chunks are done, beside the camera passes of the later
 * ranges, and the landmark tiles whose observing cameras all lie in ranges 0 .. r start when the
 * camera passes of those ranges are done.
 *   ranges       1 (one range) .. 64
 *   cpass_warps  resident warps per SM of each camera-pass launch (0: one CTA per chunk)
 *   lpass_ctas   resident CTAs per SM of each landmark-pass launch of small tiles (0: one per tile)
 *   prio[3]      stream-priority rank, 0 (highest) to 2, of the camera passes, the camera solves
 *                and the landmark passes
 * Defaults for problems of at least 2^20 observations: 2 ranges, or 6 when the camera solves
 * (32 cameras per CTA) need more CTAs than 5 per SM, ranks (1, 0, 1), no bounds; 1 range below. It applies to the graph path (runs without per-kernel timing) of contexts with
 * the per-block restart, no coarse blocks and the persistent path off, and is ignored elsewhere;
 * the ranges are recomputed when the observations change. DABA_ERR_ARG for a value out of range. */
typedef struct {
  int32_t ranges;
  int32_t cpass_warps;
  int32_t lpass_ctas;
  int32_t prio[3];
} daba_pipeline;
daba_status daba_set_pipeline(daba_ctx* ctx, const daba_pipeline* p);

/* Number of kernel launches the library issued in the last daba_run. */
int64_t daba_last_launch_count(const daba_ctx* ctx);

/* Device memory of a context (Sec. 7, memory and communication: the paper reports the most
 * memory a device uses). *bytes = the bytes of the device buffers the context holds now (its
 * own, plus those of the FP64 context it creates for the reverse mode of a MIXED context);
 * *peak = the most it has held at once (with such an FP64 context, the sum of both peaks, an
 * upper bound). Counts the library's own allocations, not the CUDA runtime's memory for
 * graphs, streams and module code. Buffers are allocated by daba_create (sized by M, N and
 * nnz) and by the calls that first need more (daba_set_partition and
 * daba_unrolled_grad); daba_run allocates none. Either pointer may be NULL (not both:
 * DABA_ERR_ARG, as for a NULL context). Host pointers; no GPU work. */
daba_status daba_device_bytes(const daba_ctx* ctx, int64_t* bytes, int64_t* peak);

/* The objective in pixel^2 of caller-provided device arrays (the value daba_objective returns
 * for a context holding the same cameras, landmarks and observations), allocating no device
 * memory. The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (a framework whose memory pool owns the device, a real-time loop that must not
 * allocate, a plugin limited to the buffers it is handed).
 *   cams (M x 9), lms (N x 3), cam_idx, lm_idx (nnz), uv (nnz x 2): as in daba_set_state and
 *   daba_set_observations, but all of them, and `out` (one double), must be managed memory or
 *   device memory of the current device (device memory of another GPU is DABA_ERR_ARG).
 *   loss is a daba_loss value; pixel_scale > 0 is the internal unit in pixels (the result
 *   depends on it only through rounding).
 * Its scratch is one file-scope __device__ array of about 2.4 MB that every GPU which loads
 * the library holds until the process exits; it limits M to 16384 (DABA_ERR_ARG beyond that,
 * as for other invalid sizes, options or host pointers). The first call on a device looks up
 * that array's address with cudaGetSymbolAddress, so make the first call before any stream
 * capture. All calls share the array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller. Observation indices out of range, or a
 * landmark at a camera centre, make *out NaN instead of returning an error
 * (the call does not wait for the GPU). Returns DABA_ERR_CUDA if a launch fails. */
daba_status daba_objective_noalloc(int32_t M, int32_t N, int64_t nnz, const double* cams, const double* lms,
                                   const int32_t* cam_idx, const int32_t* lm_idx, const double* uv, int32_t loss,
                                   double loss_scale_px, double pixel_scale, double* out, void* stream);

/* One-line description of the last error of this context (never NULL). */
const char* daba_last_error(const daba_ctx* ctx);

/* Frees the context and all its device memory. NULL is a no-op. */
void daba_destroy(daba_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DABA_H_ */
