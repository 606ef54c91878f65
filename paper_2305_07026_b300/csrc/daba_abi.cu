// daba_abi.cu -- host runtime and C ABI (include/daba.h) of the DABA iteration library.
//
// Setup (daba_set_observations) sorts the observations stably by camera and by
// landmark on the host, builds the CSR offsets, the camera chunks of the
// camera-sorted pass and the landmark tiles of the landmark-sorted pass, and
// uploads them. daba_run then enqueues, per iteration of Algorithm 1, the five
// kernels of daba_kernels.cuh on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/daba.h"
#include "daba_kernels.cuh"
#include "daba_state.cuh"
#include "daba_adjoint.cuh"
#include "daba_blocks.cuh"

using namespace daba;

namespace {

constexpr int CHUNK_OBS = 2048;   // camera-sorted pass: default observations per warp chunk
constexpr int GSEG = 1024;        // iterations per run segment (device gamma / trace buffers)
constexpr int LREC = 8;           // landmark record: two V4 (l[3], delta0), (delta1, delta2, S, E)
constexpr int GRAPH_ITERS = 8;    // iterations per captured graph (even: keeps the buffer parity)
constexpr int RUN_GRAPH_MAX = 256;   // a run of at most this many iterations is one graph launch
constexpr int64_t PIPE_MIN_NNZ = 1 << 20;   // two-range schedule by default from this many observations
constexpr int PIPE_MAX_RANGES = 64;
constexpr int PIPE_POOL = 8;   // streams per kernel role of the range schedule
constexpr uint64_t CKPT_MAGIC = 0x44414241434b5033ull;   // "DABACKP3"

}  // namespace

struct daba_ctx {
  int M = 0, N = 0;
  int64_t nnz = 0;
  daba_options opt{};
  std::string err;
  int dev = 0;
  // sizes of the schedules
  int n_chunks = 0, n_tiles = 0, max_chunks = 0, max_tiles = 0;
  int tile_class_end[2] = {0, 0};   // tiles [0, e0): small, [e0, e1): one long-track landmark each
  bool obs_set = false, state_set = false, checked = false;
  double s_norm = 0.0, u_scale_uploaded = -1.0;
  bool h_uv_stale = false;   // pixels last set from device memory (the host copy is older)
  double s_k = 1.0;   // Nesterov s^(k)
  int64_t k = 0;      // iteration index
  bool timing = false;
  long long wait_ns = 1000000000ll;   // landmark pass: limit of the first wait on the tile copies
  double tms[5] = {0, 0, 0, 0, 0};
  int64_t launches = 0;
  // host copies (setup data and boundary state)
  std::vector<int32_t> h_cam_idx, h_lm_idx;
  std::vector<double> h_uv;
  std::vector<int32_t> h_c_order, h_cam_ptr, h_l_order, h_lm_ptr, h_t_order;
  std::vector<int32_t> h_li_order;          // observations sorted by internal landmark id
  std::vector<int32_t> h_ci_order;          // observations in the device's camera order
  std::vector<int32_t> h_lperm, h_linv;     // internal -> external landmark id and inverse
  // device buffers
  void *c_lm = nullptr, *c_u = nullptr;
  void *chunk_cam = nullptr, *chunk_beg = nullptr, *cam_chunk_ptr = nullptr;
  void *lm_ptr = nullptr, *tile_lm = nullptr, *c_rpos = nullptr, *t_inv = nullptr;
  void *rec_a = nullptr, *rec_b = nullptr, *rec_c = nullptr;   // landmark-side records in camera order
  void *cam_x = nullptr, *cam_dx = nullptr, *cam_Rbar = nullptr, *pack2[2] = {nullptr, nullptr};
  void *cam_S = nullptr, *cam_E = nullptr, *cam_F = nullptr, *cam_Fb = nullptr, *cam_rs = nullptr;
  void *lmrec2[2] = {nullptr, nullptr}, *lm_lo2[2] = {nullptr, nullptr};   // double-buffered landmark state
  void *lm_rs = nullptr, *lm_Fd = nullptr, *lm_Fbd = nullptr;
  void *chunk_part = nullptr, *chunk_f = nullptr, *tile_rs = nullptr, *cam_Fsum = nullptr;
  void *fin_blk = nullptr, *fin_ticket = nullptr;
  void *d_gam = nullptr, *d_it = nullptr, *d_first = nullptr, *d_flag = nullptr, *d_trace = nullptr,
       *d_rs = nullptr, *d_obj = nullptr;
  // state I/O: staging of boundary-layout state, external -> internal landmark id, checks
  void *st_cam = nullptr, *st_lm = nullptr, *d_linv = nullptr, *d_chk = nullptr, *d_bad = nullptr;
  // device copies of the camera order (device position -> input index) and of the internal ->
  // external landmark map (gradient outputs, pixel updates)
  void *d_ci_order = nullptr, *d_lperm = nullptr;
  std::vector<std::pair<void*, size_t>> allocs;   // device buffers of this context and their sizes
  size_t dev_bytes = 0, dev_peak = 0;              // bytes they hold now, and the most held at once
  std::vector<cudaEvent_t> events;
  cudaStream_t s_hi = nullptr, s_lo = nullptr;   // camera pass + solves (high priority), landmark pass
  cudaEvent_t ev_fork = nullptr, ev_hi = nullptr, ev_lo = nullptr;
  // CUDA graphs of GRAPH_ITERS and of 1 iteration(s) starting at an even / odd k (the double
  // buffers alternate with k), captured on s_cap at the first untimed run
  cudaStream_t s_cap = nullptr;
  cudaEvent_t ev_cap0 = nullptr, ev_cap1 = nullptr;
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [GRAPH_ITERS or 1][k & 1]
  int64_t graph_nl[2] = {0, 0};                                                // kernel launches per graph
  // a whole run (the first-iteration prepare and n iterations) as one graph, per start parity;
  // recaptured when a run of another length comes, or with timing switched on or off (the
  // timing graph also holds the per-kernel event records)
  cudaGraphExec_t run_graph[2] = {nullptr, nullptr};
  int run_graph_n[2] = {0, 0};
  int64_t run_graph_nl[2] = {0, 0};
  bool run_graph_timing[2] = {false, false};
  // a batch of independent scenes: camera ranges, chunk ranges per scene (device), outputs
  int n_scenes = 1;
  std::vector<int32_t> h_scene_cam;
  void *d_scene_chunk = nullptr, *d_scene_f = nullptr;
  // reverse mode (daba_unrolled_grad), allocated at first use: adjoints of x^(k+1), x^k, x^(k-1)
  // (cameras, landmarks), of the two conditioning points, of the statistics, of the pixels,
  // and copies of the iteration state
  void *adj_c[3] = {nullptr, nullptr, nullptr}, *adj_l[3] = {nullptr, nullptr, nullptr};
  void *zb_c[2] = {nullptr, nullptr}, *zb_l[2] = {nullptr, nullptr};
  void *st_bar = nullptr, *ab_bar = nullptr, *g_u = nullptr;
  std::vector<void*> slots;
  std::vector<void*> itslots;         // per iteration of a segment: statistics, landmark sums, decisions
  void* lm_sums_out = nullptr;        // set while the segment sweep runs: the landmark pass's (a, b) sums
  // global restart variant (allocated when restart_mode is global): per-block terms of the test,
  // the MM alternatives, the decision and the device Nesterov scalar
  void *g_cam = nullptr, *g_tile = nullptr, *cam_alt = nullptr, *lm_alt = nullptr, *g_fire = nullptr,
       *s_dev = nullptr;
  // the entry state of daba_run, put back when the run fails
  void* bk = nullptr;
  // reverse mode of a MIXED context: an FP64 context with the same observations and unit that
  // replays each iteration from the MIXED iterate (created at first use, refreshed when the
  // observations or pixels change: obs_version), and the MIXED run's restart decisions
  daba_ctx* shadow = nullptr;
  int64_t obs_version = 0, shadow_version = -1;
  void* mx_dec = nullptr;
  size_t mx_dec_bytes = 0;
  // persistent path (daba_set_persistent): a run's iterations in one cooperative launch
  bool persistent = false;
  void* d_gbar = nullptr;   // grid-barrier counter and generation
  // coarse blocks (daba_set_partition): up to BLK_MAX_CAMS cameras and any landmarks per block,
  // FP64; the buffers grow with the partition (blk_cap: bytes held per buffer)
  int n_blocks = 0;
  int blk_ld = 0;        // 9 x the most cameras in one block with the scratch in shared memory, else 0
  size_t blk_smem = 0;   // dynamic shared memory of the block solve
  int blk_cs = 1;        // CTAs per block (a thread-block cluster when above 1; global scratch only)
  int blk_pref = 0;      // daba_set_block_ctas: 0 automatic, 1 one CTA per block, 2..16 a cluster
  uint64_t blk_hash = 0;   // FNV-1a of the partition (n_blocks, cam_block, lm_block): checkpoints carry it
  int blk_ncam = 0;        // blocks that hold a camera (the restart count of an iteration)
  void *blk_g = nullptr, *blk_Ealt = nullptr;   // global restart over blocks: test terms, kept E(k+1)
  void *blk_ci_e = nullptr, *blk_ci_io = nullptr, *blk_gcam = nullptr, *blk_gvec = nullptr, *blk_gS = nullptr,
       *blk_soff = nullptr;
  void *c_intra = nullptr, *blk_cam_ptr = nullptr, *blk_cams = nullptr, *blk_lm_ptr = nullptr, *blk_lms = nullptr,
       *blk_io_ptr = nullptr, *blk_io_cam = nullptr, *blk_io_obs = nullptr, *blk_ci_ptr = nullptr,
       *blk_ci_obs = nullptr, *blk_ci_lm = nullptr, *blk_sums = nullptr, *blk_lsc = nullptr, *blk_isc = nullptr,
       *blk_E = nullptr, *blk_Fbar = nullptr, *blk_F = nullptr, *blk_rs = nullptr, *blk_bk = nullptr;
  std::vector<std::pair<void*, size_t>> blk_cap;
  // range schedule (daba_set_pipeline): the R ranges in use (1: the one-range iteration), their
  // camera and chunk bounds, the landmark tiles in launch order (per class r, the tiles whose
  // observing cameras all lie in ranges <= r, some in range r: small tiles, then one-landmark
  // tiles, pipe_nt of each) and each class's lowest observing range, the counters of the bounded
  // grids, stream pools per role (camera pass, camera solves, landmark pass) and events per range
  daba_pipeline pipe{};
  int pipe_R = 1;
  std::vector<int> pipe_cam, pipe_chunk, pipe_nt, pipe_minr;
  void *d_tlist = nullptr, *d_ctr = nullptr;
  cudaStream_t s_pool[3][PIPE_POOL] = {};
  std::vector<cudaEvent_t> ev_rng;   // 3 per range: camera pass, camera solves, landmark pass done
  int n_sm = 0;
  std::vector<int32_t> h_tile_lm, h_lmi_ptr, h_cam_chunk_ptr;
};

namespace {

daba_status fail(daba_ctx* c, daba_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(ctx, DABA_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

daba_status dalloc(daba_ctx* ctx, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(ctx, DABA_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  ctx->allocs.emplace_back(*p, bytes);
  ctx->dev_bytes += bytes;
  ctx->dev_peak = std::max(ctx->dev_peak, ctx->dev_bytes);
  return DABA_OK;
}

// *p holds at least `bytes` afterwards; a smaller buffer is freed and replaced (contents dropped)
daba_status dgrow(daba_ctx* ctx, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  auto& cap = ctx->blk_cap;
  auto it = std::find_if(cap.begin(), cap.end(), [&](const std::pair<void*, size_t>& c) { return c.first == *p; });
  if (*p && it != cap.end() && it->second >= bytes) return DABA_OK;
  if (*p) {
    if (it != cap.end()) cap.erase(it);
    auto a = std::find_if(ctx->allocs.begin(), ctx->allocs.end(),
                          [&](const std::pair<void*, size_t>& x) { return x.first == *p; });
    if (a != ctx->allocs.end()) {
      ctx->dev_bytes -= a->second;
      ctx->allocs.erase(a);
    }
    cudaFree(*p);
    *p = nullptr;
  }
  daba_status s = dalloc(ctx, p, bytes);
  if (s == DABA_OK) cap.emplace_back(*p, bytes);
  return s;
}

// copy `bytes` from a host or device source into host memory
daba_status fetch(daba_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (is_device_ptr(src)) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  } else {
    std::memcpy(dst, src, bytes);
  }
  return DABA_OK;
}

// copy host data to a host or device destination
daba_status deliver(daba_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (is_device_ptr(dst)) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  } else {
    std::memcpy(dst, src, bytes);
  }
  return DABA_OK;
}

bool is_mixed(const daba_ctx* c) { return c->opt.prec == DABA_MIXED; }

// buffers of iteration k (the landmark state and the camera pack alternate between two)
inline void* pack_at(const daba_ctx* c, int64_t k) { return c->pack2[k & 1]; }
inline void* lmrec_at(const daba_ctx* c, int64_t k) { return c->lmrec2[k & 1]; }
inline void* lmlo_at(const daba_ctx* c, int64_t k) { return c->lm_lo2[k & 1]; }

// internal (device) index of external landmark j (identity until observations are set)
inline size_t lm_internal(const daba_ctx* c, int j) { return c->h_linv.empty() ? (size_t)j : (size_t)c->h_linv[j]; }
size_t real_sz(const daba_ctx* c) { return is_mixed(c) ? sizeof(float) : sizeof(double); }

// stable counting sort of 0..n-1 by key in [0, K): order and CSR offsets
void counting_sort(const std::vector<int32_t>& key, int K, std::vector<int32_t>& order, std::vector<int32_t>& ptr) {
  const int64_t n = (int64_t)key.size();
  ptr.assign(K + 1, 0);
  for (int64_t i = 0; i < n; ++i) ptr[key[i] + 1]++;
  for (int k = 0; k < K; ++k) ptr[k + 1] += ptr[k];
  std::vector<int32_t> pos(ptr.begin(), ptr.end() - 1);
  order.resize(n);
  for (int64_t i = 0; i < n; ++i) order[pos[key[i]]++] = (int32_t)i;
}

template <class Real, class Real2>
void upload_u(daba_ctx* ctx, cudaStream_t st, cudaError_t* err) {
  const double s = ctx->s_norm;
  std::vector<Real2> cu(ctx->nnz);
  for (int64_t o = 0; o < ctx->nnz; ++o) {
    const int32_t i = ctx->h_ci_order[o];
    cu[o].x = Real(ctx->h_uv[2 * (size_t)i] / s);
    cu[o].y = Real(ctx->h_uv[2 * (size_t)i + 1] / s);
  }
  *err = cudaMemcpyAsync(ctx->c_u, cu.data(), cu.size() * sizeof(Real2), cudaMemcpyHostToDevice, st);
  if (*err == cudaSuccess) *err = cudaStreamSynchronize(st);
}

daba_status ensure_u(daba_ctx* ctx, cudaStream_t st) {
  if (ctx->u_scale_uploaded == ctx->s_norm) return DABA_OK;
  if (ctx->h_uv_stale) return fail(ctx, DABA_ERR_STATE, "pixels set from device memory cannot be re-scaled");
  cudaError_t e;
  if (is_mixed(ctx))
    upload_u<float, float2>(ctx, st, &e);
  else
    upload_u<double, double2>(ctx, st, &e);
  if (e != cudaSuccess) return fail(ctx, DABA_ERR_CUDA, "uploading pixels: %s", cudaGetErrorString(e));
  ctx->u_scale_uploaded = ctx->s_norm;
  return DABA_OK;
}

// Assumption 2 check of the current iterate on the device (once per state set)
daba_status check_degenerate(daba_ctx* ctx, cudaStream_t st) {
  if (ctx->checked) return DABA_OK;
  k_chk_init<<<1, 32, 0, st>>>((int*)ctx->d_chk, (unsigned long long*)ctx->d_bad);
  if (is_mixed(ctx))
    k_check_degenerate<float, true><<<ctx->n_chunks, 256, 0, st>>>(
        (const int*)ctx->chunk_cam, (const int*)ctx->chunk_beg, (const int*)ctx->c_lm, (const double*)ctx->cam_x,
        (const V4<float>*)lmrec_at(ctx, ctx->k), (const V4<float>*)lmlo_at(ctx, ctx->k),
        (unsigned long long*)ctx->d_bad);
  else
    k_check_degenerate<double, false><<<ctx->n_chunks, 256, 0, st>>>(
        (const int*)ctx->chunk_cam, (const int*)ctx->chunk_beg, (const int*)ctx->c_lm, (const double*)ctx->cam_x,
        (const V4<double>*)lmrec_at(ctx, ctx->k), nullptr, (unsigned long long*)ctx->d_bad);
  CK(cudaGetLastError());
  unsigned long long bad = 0;
  CK(cudaMemcpyAsync(&bad, ctx->d_bad, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad != ~0ull) {
    const int32_t o = ctx->h_ci_order[(size_t)bad];   // input index of that observation
    return fail(ctx, DABA_ERR_DEGENERATE, "observation %d: landmark %d coincides with camera %d centre", o,
                ctx->h_lm_idx[o], ctx->h_cam_idx[o]);
  }
  ctx->checked = true;
  return DABA_OK;
}

template <class Real>
LossC<Real> loss_consts(const daba_ctx* ctx) {
  const double c = ctx->opt.loss == DABA_LOSS_TRIVIAL ? 1.0 : ctx->opt.loss_scale_px / ctx->s_norm;
  LossC<Real> L;
  L.c = Real(c);
  L.c2 = Real(c * c);
  L.inv_c2 = Real(1.0 / (c * c));
  return L;
}

IterParams iter_params(daba_ctx* ctx) {
  IterParams P;
  P.gam = (const double*)ctx->d_gam;
  P.it = (int*)ctx->d_it;
  P.first = (int*)ctx->d_first;
  P.xi = ctx->opt.xi;
  P.eta = ctx->opt.eta;
  P.eta1 = 1.0 - ctx->opt.eta;
  P.hxi = 0.5 * ctx->opt.xi;
  P.eta1f = (float)P.eta1;
  P.hxif = (float)P.hxi;
  P.accelerated = ctx->opt.accelerated;
  P.n_alt = ctx->opt.cam_alternations;
  P.flag = (int*)ctx->d_flag;
  P.wait_ns = ctx->wait_ns;
  P.restart_global = ctx->opt.restart_mode == DABA_RESTART_GLOBAL ? 1 : 0;
  P.reset_s = ctx->opt.momentum_reset;
  P.g_cam = (double*)ctx->g_cam;
  P.g_tile = (double*)ctx->g_tile;
  P.cam_alt = (double*)ctx->cam_alt;
  P.g_fire = (int*)ctx->g_fire;
  P.s_dev = (double*)ctx->s_dev;
  P.fire_given = 0;
  return P;
}

// Kernel ranges of one launch: the camera pass takes chunks c0 .. c1 - 1 (c1 < 0: all), with a
// bounded grid of `grid` one-warp CTAs when ctr is set.
struct PassRange {
  int c0 = 0, c1 = -1;
  unsigned* ctr = nullptr;
  int grid = 0;
};

template <int LOSS, class Real, class Real2, bool HAS_LO>
cudaError_t launch_passes(daba_ctx* ctx, cudaStream_t st, int which, int64_t k, PassRange r = PassRange()) {
  const LossC<Real> L = loss_consts<Real>(ctx);
  const IterParams P = iter_params(ctx);
  const int threads = CPASS_WARPS * 32;
  const int c1 = r.c1 < 0 ? ctx->n_chunks : r.c1;
  int blocks = (c1 - r.c0 + CPASS_WARPS - 1) / CPASS_WARPS;
  if (blocks <= 0) return cudaSuccess;
  if (which == 1) {
    if (r.ctr) blocks = std::min(blocks, r.grid);
    k_cpass<LOSS, Real, Real2><<<blocks, threads, 0, st>>>(
        r.c0, c1, r.ctr, (const int*)ctx->chunk_cam, (const int*)ctx->chunk_beg, (const int*)ctx->c_lm,
        (const Real2*)ctx->c_u, (const V4<Real>*)pack_at(ctx, k), (const V4<Real>*)lmrec_at(ctx, k), L, P,
        (Real*)ctx->chunk_part, (const int*)ctx->c_rpos, (V4<Real>*)ctx->rec_a, (V4<Real>*)ctx->rec_b,
        (typename RecC<Real>::type*)ctx->rec_c);
  } else if (which == 6) {
    k_objective<LOSS, Real, Real2, HAS_LO><<<blocks, threads, 0, st>>>(
        ctx->n_chunks, (const int*)ctx->chunk_cam, (const int*)ctx->chunk_beg, (const int*)ctx->c_lm,
        (const Real2*)ctx->c_u, (const V4<Real>*)pack_at(ctx, k), (const V4<Real>*)lmrec_at(ctx, k),
        (const V4<float>*)lmlo_at(ctx, k), L, (Real*)ctx->chunk_f);
  }
  return cudaGetLastError();
}

template <class Real, class Real2, bool HAS_LO>
cudaError_t launch_by_loss(daba_ctx* ctx, cudaStream_t st, int which, int64_t k, PassRange r) {
  switch (ctx->opt.loss) {
    case DABA_LOSS_TRIVIAL: return launch_passes<LOSS_TRIVIAL, Real, Real2, HAS_LO>(ctx, st, which, k, r);
    case DABA_LOSS_HUBER: return launch_passes<LOSS_HUBER, Real, Real2, HAS_LO>(ctx, st, which, k, r);
    case DABA_LOSS_CAUCHY: return launch_passes<LOSS_CAUCHY, Real, Real2, HAS_LO>(ctx, st, which, k, r);
    default: return launch_passes<LOSS_WELSCH, Real, Real2, HAS_LO>(ctx, st, which, k, r);
  }
}

cudaError_t launch_pass(daba_ctx* ctx, cudaStream_t st, int which, int64_t k, PassRange r = PassRange()) {
  ctx->launches++;
  if (is_mixed(ctx)) return launch_by_loss<float, float2, true>(ctx, st, which, k, r);
  return launch_by_loss<double, double2, false>(ctx, st, which, k, r);
}

// Tiles of one landmark-pass launch: positions q[c] .. q[c] + n[c] - 1 of the tile order (tlist, or
// the tiles themselves when it is null) for the small (c = 0) and one-landmark (c = 1) tiles; the
// small tiles with a bounded grid of `grid` CTAs when ctr is set.
struct TileRange {
  const int* tlist = nullptr;
  int q[2] = {0, 0}, n[2] = {-1, -1};   // n < 0: every tile of the class
  unsigned* ctr = nullptr;
  int grid = 0;
};

// landmark pass: small tiles, then the one-landmark tiles of long tracks
template <class Real, class Real2, bool HAS_LO>
cudaError_t launch_lpass_t(daba_ctx* ctx, cudaStream_t st, int64_t k, const TileRange& r) {
  const IterParams P = iter_params(ctx);
  LpassOut<Real> O;
  O.lmrec_out = (V4<Real>*)lmrec_at(ctx, k + 1);
  O.lm_lo_out = (V4<float>*)lmlo_at(ctx, k + 1);
  O.lm_rs = (uint8_t*)ctx->lm_rs;
  O.lm_Fdiag = (double*)ctx->lm_Fd;
  O.lm_Fbdiag = (double*)ctx->lm_Fbd;
  O.lm_alt = (V4<Real>*)ctx->lm_alt;
  O.lm_sums = (double*)ctx->lm_sums_out;
  O.blk_sums = ctx->n_blocks > 0 ? (double*)ctx->blk_sums : nullptr;
  const int caps[2] = {ctx->opt.tile_obs, BIG_TILE_OBS};
  int t0 = 0;
  for (int c = 0; c < 2; ++c) {
    const int q0 = r.n[c] < 0 ? t0 : r.q[c];
    const int nt = r.n[c] < 0 ? ctx->tile_class_end[c] - t0 : r.n[c];
    if (nt > 0) {
      unsigned* ctr = c == 0 ? r.ctr : nullptr;
      const int grid = ctr ? std::min(nt, r.grid) : nt;
      k_lpass<Real, Real2, HAS_LO><<<grid, LPASS_THREADS, lpass_smem_bytes<Real>(caps[c]), st>>>(
          q0, nt, r.tlist, ctr, caps[c], (const int*)ctx->tile_lm, (const int*)ctx->lm_ptr,
          (const uint16_t*)ctx->t_inv, (const V4<Real>*)ctx->rec_a, (const V4<Real>*)ctx->rec_b,
          (const typename RecC<Real>::type*)ctx->rec_c, (const V4<Real>*)lmrec_at(ctx, k),
          (const V4<float>*)lmlo_at(ctx, k), P, (int*)ctx->tile_rs, O);
      ctx->launches++;
    }
    t0 = ctx->tile_class_end[c];
  }
  return cudaGetLastError();
}

cudaError_t launch_lpass(daba_ctx* ctx, cudaStream_t st, int64_t k, const TileRange& r = TileRange()) {
  if (is_mixed(ctx)) return launch_lpass_t<float, float2, true>(ctx, st, k, r);
  return launch_lpass_t<double, double2, false>(ctx, st, k, r);
}

cudaError_t launch_prepare(daba_ctx* ctx, cudaStream_t st, int64_t k) {
  ctx->launches++;
  const IterParams P = iter_params(ctx);
  const int blocks = (ctx->M + 127) / 128;
  if (is_mixed(ctx))
    k_cam_prepare<float><<<blocks, 128, 0, st>>>(ctx->M, (const double*)ctx->cam_x, (const double*)ctx->cam_dx, P,
                                                 (double*)ctx->cam_Rbar, (V4<float>*)pack_at(ctx, k));
  else
    k_cam_prepare<double><<<blocks, 128, 0, st>>>(ctx->M, (const double*)ctx->cam_x, (const double*)ctx->cam_dx, P,
                                                  (double*)ctx->cam_Rbar, (V4<double>*)pack_at(ctx, k));
  return cudaGetLastError();
}

// camera solves of cameras i0 .. i1 - 1 (i1 < 0: all)
template <int SOLVER>
cudaError_t launch_camsolve_t(daba_ctx* ctx, cudaStream_t st, int64_t k, int i0, int i1) {
  if (i1 < 0) i1 = ctx->M;
  if (i1 <= i0) return cudaSuccess;
  ctx->launches++;
  const IterParams P = iter_params(ctx);
  const int blocks = (i1 - i0 + 31) / 32;   // 32 cameras per CTA (two warps)
  if (is_mixed(ctx))
    k_camsolve<float, SOLVER><<<blocks, CAMSOLVE_THREADS, 0, st>>>(i0, i1, (const int*)ctx->cam_chunk_ptr, (const float*)ctx->chunk_part,
                                             (double*)ctx->cam_x, (double*)ctx->cam_dx, (double*)ctx->cam_Rbar, P,
                                             (double*)ctx->cam_S, (double*)ctx->cam_E, (double*)ctx->cam_F,
                                             (double*)ctx->cam_Fb, (uint8_t*)ctx->cam_rs, (double*)ctx->cam_Fsum,
                                             (V4<float>*)pack_at(ctx, k + 1));
  else
    k_camsolve<double, SOLVER><<<blocks, CAMSOLVE_THREADS, 0, st>>>(i0, i1, (const int*)ctx->cam_chunk_ptr,
                                              (const double*)ctx->chunk_part, (double*)ctx->cam_x,
                                              (double*)ctx->cam_dx, (double*)ctx->cam_Rbar, P, (double*)ctx->cam_S,
                                              (double*)ctx->cam_E, (double*)ctx->cam_F, (double*)ctx->cam_Fb,
                                              (uint8_t*)ctx->cam_rs, (double*)ctx->cam_Fsum,
                                              (V4<double>*)pack_at(ctx, k + 1));
  return cudaGetLastError();
}

cudaError_t launch_camsolve(daba_ctx* ctx, cudaStream_t st, int64_t k, int i0 = 0, int i1 = -1) {
  if (ctx->opt.cam_solver == DABA_CAM_LM) return launch_camsolve_t<CAM_LM>(ctx, st, k, i0, i1);
  return launch_camsolve_t<CAM_SCAM>(ctx, st, k, i0, i1);
}

// fire_given: the global restart was decided over coarse blocks (g_fire), counted as n_restart
// blocks when it fired
cudaError_t launch_finalize(daba_ctx* ctx, cudaStream_t st, bool fire_given = false, int n_restart = -1) {
  ctx->launches++;
  IterParams P = iter_params(ctx);
  P.fire_given = fire_given ? 1 : 0;
  k_finalize<<<FIN_BLOCKS, FIN_THREADS, 0, st>>>(ctx->M, (const double*)ctx->cam_Fsum, (const uint8_t*)ctx->cam_rs,
                                                  ctx->n_tiles, (const int*)ctx->tile_rs,
                                                  n_restart >= 0 ? n_restart : ctx->M + ctx->N,
                                                  ctx->s_norm * ctx->s_norm, P,
                                                  (double*)ctx->fin_blk, (unsigned int*)ctx->fin_ticket,
                                                  (double*)ctx->d_trace, (int*)ctx->d_rs, (int*)ctx->d_flag);
  return cudaGetLastError();
}

// coarse blocks: one iteration k (direct launches on st): the camera pass in block mode, the
// landmark pass in sum mode, the block solves, the reduction
template <int LOSS>
cudaError_t launch_blk_iter_t(daba_ctx* ctx, cudaStream_t st, int64_t k) {
  const IterParams P = iter_params(ctx);
  const LossC<double> L = loss_consts<double>(ctx);
  cudaError_t e;
  if (ctx->n_chunks > 0) {
    k_cpass_blk<LOSS><<<ctx->n_chunks, CPASS_WARPS * 32, 0, st>>>(
        ctx->n_chunks, (const int*)ctx->chunk_cam, (const int*)ctx->chunk_beg, (const int*)ctx->c_lm,
        (const double2*)ctx->c_u, (const V4<double>*)pack_at(ctx, k), (const V4<double>*)lmrec_at(ctx, k), L, P,
        (double*)ctx->chunk_part, (const int*)ctx->c_rpos, (V4<double>*)ctx->rec_a, (V4<double>*)ctx->rec_b,
        (double2*)ctx->rec_c, (const uint8_t*)ctx->c_intra);
    ctx->launches++;
  }
  if ((e = launch_lpass(ctx, st, k)) != cudaSuccess) return e;   // sum mode while blk_sums is set
  BlkArgs A;
  A.S = ctx->n_blocks;
  A.ld = ctx->blk_ld;
  A.cam_ptr = (const int*)ctx->blk_cam_ptr;
  A.cams = (const int*)ctx->blk_cams;
  A.lm_ptr = (const int*)ctx->blk_lm_ptr;
  A.lms = (const int*)ctx->blk_lms;
  A.io_ptr = (const int*)ctx->blk_io_ptr;
  A.io_cam = (const int*)ctx->blk_io_cam;
  A.io_obs = (const int*)ctx->blk_io_obs;
  A.ci_ptr = (const int*)ctx->blk_ci_ptr;
  A.ci_obs = (const int*)ctx->blk_ci_obs;
  A.ci_lm = (const int*)ctx->blk_ci_lm;
  A.ci_e = (const int*)ctx->blk_ci_e;
  A.ci_io = (const int*)ctx->blk_ci_io;
  A.g_cam = (BlkCam*)ctx->blk_gcam;
  A.g_vec = (double*)ctx->blk_gvec;
  A.g_S = (double*)ctx->blk_gS;
  A.g_soff = (const long long*)ctx->blk_soff;
  A.c_u = (const double2*)ctx->c_u;
  A.cam_chunk_ptr = (const int*)ctx->cam_chunk_ptr;
  A.part = (const double*)ctx->chunk_part;
  A.lm_sums = (const double*)ctx->blk_sums;
  A.cam_x = (double*)ctx->cam_x;
  A.cam_dx = (double*)ctx->cam_dx;
  A.cam_Rbar = (double*)ctx->cam_Rbar;
  A.cam_Fsum = (double*)ctx->cam_Fsum;
  A.cam_rs = (uint8_t*)ctx->cam_rs;
  A.lmrec = (const V4<double>*)lmrec_at(ctx, k);
  A.lmrec_out = (V4<double>*)lmrec_at(ctx, k + 1);
  A.blk_E = (double*)ctx->blk_E;
  A.blk_Fbar = (double*)ctx->blk_Fbar;
  A.blk_F = (double*)ctx->blk_F;
  A.blk_rs = (uint8_t*)ctx->blk_rs;
  A.lsc = (double*)ctx->blk_lsc;
  A.isc = (double*)ctx->blk_isc;
  A.pack_next = (V4<double>*)pack_at(ctx, k + 1);
  A.L = L;
  A.loss = LOSS;
  A.blk_g = (double*)ctx->blk_g;
  A.blk_Ealt = (double*)ctx->blk_Ealt;
  auto solve = [&](int pass) -> cudaError_t {
    A.pass = pass;
    ctx->launches++;
    if (ctx->blk_cs > 1) {   // a cluster of blk_cs CTAs per block
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(ctx->n_blocks * ctx->blk_cs));
      cfg.blockDim = dim3(BLK_THREADS);
      cfg.dynamicSmemBytes = ctx->blk_smem;
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)ctx->blk_cs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, k_blk_solve, A, P);
    }
    k_blk_solve<<<ctx->n_blocks, BLK_THREADS, ctx->blk_smem, st>>>(A, P);
    return cudaGetLastError();
  };
  if (ctx->opt.accelerated && ctx->opt.restart_mode == DABA_RESTART_GLOBAL) {
    // global restart: every block's accelerated step kept, the test over the blocks, then the
    // MM step everywhere or the kept steps committed; the reduction takes the decision
    if ((e = solve(1)) != cudaSuccess) return e;
    k_blk_fire<<<1, 32, 0, st>>>(ctx->n_blocks, (const double*)ctx->blk_g, (int*)ctx->g_fire);
    ctx->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = solve(2)) != cudaSuccess) return e;
    return launch_finalize(ctx, st, true, ctx->blk_ncam);
  }
  if ((e = solve(0)) != cudaSuccess) return e;
  return launch_finalize(ctx, st);
}

cudaError_t launch_blk_iter(daba_ctx* ctx, cudaStream_t st, int64_t k) {
  switch (ctx->opt.loss) {
    case DABA_LOSS_TRIVIAL: return launch_blk_iter_t<LOSS_TRIVIAL>(ctx, st, k);
    case DABA_LOSS_HUBER: return launch_blk_iter_t<LOSS_HUBER>(ctx, st, k);
    case DABA_LOSS_CAUCHY: return launch_blk_iter_t<LOSS_CAUCHY>(ctx, st, k);
    default: return launch_blk_iter_t<LOSS_WELSCH>(ctx, st, k);
  }
}

// persistent path: n iterations from iteration index k0 as one cooperative launch on st (after
// the prepare kernel of the run's first iteration)
size_t pers_smem(const daba_ctx* ctx) {
  const bool big = ctx->tile_class_end[1] > ctx->tile_class_end[0];
  size_t b = std::max((size_t)4 * sizeof(CpassWarpSmem<float, float2>), (size_t)2 * 32 * 16 * sizeof(double));
  b = std::max(b, lpass_smem_bytes<float>(ctx->opt.tile_obs));
  if (big) b = std::max(b, lpass_smem_bytes<float>(BIG_TILE_OBS));
  return b;
}

template <int LOSS>
cudaError_t launch_persistent_t(daba_ctx* ctx, cudaStream_t st, int64_t k0, int n) {
  auto kern = k_run_persistent<LOSS>;
  const size_t smem = pers_smem(ctx);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, n_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PERS_THREADS, smem)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->dev)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  PersArgs A;
  A.M = ctx->M;
  A.n_chunks = ctx->n_chunks;
  A.n_tiles = ctx->tile_class_end[1];
  A.tile_obs = ctx->opt.tile_obs;
  A.n_small = ctx->tile_class_end[0];
  A.chunk_cam = (const int*)ctx->chunk_cam;
  A.chunk_beg = (const int*)ctx->chunk_beg;
  A.c_lm = (const int*)ctx->c_lm;
  A.c_rpos = (const int*)ctx->c_rpos;
  A.cam_chunk_ptr = (const int*)ctx->cam_chunk_ptr;
  A.tile_lm = (const int*)ctx->tile_lm;
  A.lm_ptr = (const int*)ctx->lm_ptr;
  A.c_u = (const float2*)ctx->c_u;
  A.t_inv = (const uint16_t*)ctx->t_inv;
  for (int q = 0; q < 2; ++q) {
    A.pack[q] = (V4<float>*)ctx->pack2[q];
    A.lmrec[q] = (V4<float>*)ctx->lmrec2[q];
    A.lmlo[q] = (V4<float>*)ctx->lm_lo2[q];
  }
  A.part = (float*)ctx->chunk_part;
  A.rec_a = (V4<float>*)ctx->rec_a;
  A.rec_b = (V4<float>*)ctx->rec_b;
  A.rec_c = (float*)ctx->rec_c;
  A.cam_x = (double*)ctx->cam_x;
  A.cam_dx = (double*)ctx->cam_dx;
  A.cam_Rbar = (double*)ctx->cam_Rbar;
  A.cam_S = (double*)ctx->cam_S;
  A.cam_E = (double*)ctx->cam_E;
  A.cam_F = (double*)ctx->cam_F;
  A.cam_Fb = (double*)ctx->cam_Fb;
  A.cam_Fsum = (double*)ctx->cam_Fsum;
  A.cam_rs = (uint8_t*)ctx->cam_rs;
  A.lm_rs = (uint8_t*)ctx->lm_rs;
  A.tile_rs = (int*)ctx->tile_rs;
  A.fin_blk = (double*)ctx->fin_blk;
  A.trace = (double*)ctx->d_trace;
  A.restarts = (int*)ctx->d_rs;
  A.bar_count = (unsigned*)ctx->d_gbar;
  A.bar_gen = (unsigned*)ctx->d_gbar + 1;
  A.s2 = ctx->s_norm * ctx->s_norm;
  IterParams P = iter_params(ctx);
  LossC<float> L = loss_consts<float>(ctx);
  int n_iter = n, par0 = (int)(k0 & 1);
  if ((e = cudaMemsetAsync(ctx->d_gbar, 0, 8, st)) != cudaSuccess) return e;
  void* args[] = {&A, &P, &L, &n_iter, &par0};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(per_sm * n_sm), dim3(PERS_THREADS), args, smem, st);
  ctx->launches++;
  return e;
}

cudaError_t launch_persistent(daba_ctx* ctx, cudaStream_t st, int64_t k0, int n) {
  switch (ctx->opt.loss) {
    case DABA_LOSS_TRIVIAL: return launch_persistent_t<LOSS_TRIVIAL>(ctx, st, k0, n);
    case DABA_LOSS_HUBER: return launch_persistent_t<LOSS_HUBER>(ctx, st, k0, n);
    case DABA_LOSS_CAUCHY: return launch_persistent_t<LOSS_CAUCHY>(ctx, st, k0, n);
    default: return launch_persistent_t<LOSS_WELSCH>(ctx, st, k0, n);
  }
}

// global restart variant: apply the MM alternatives when the reduction's test fired (the
// kernels return at once otherwise)
cudaError_t launch_fixups(daba_ctx* ctx, cudaStream_t st, int64_t k) {
  if (!(ctx->opt.accelerated && ctx->opt.restart_mode == DABA_RESTART_GLOBAL)) return cudaSuccess;
  const IterParams P = iter_params(ctx);
  const int M = ctx->M, N = ctx->N;
  if (is_mixed(ctx)) {
    k_fix_cams<float><<<(M + 127) / 128, 128, 0, st>>>(M, P, (double*)ctx->cam_x, (double*)ctx->cam_dx,
                                                       (double*)ctx->cam_Rbar, (double*)ctx->cam_S, (double*)ctx->cam_E,
                                                       (uint8_t*)ctx->cam_rs, (V4<float>*)pack_at(ctx, k + 1));
    k_fix_lms<float, true><<<(N + 255) / 256, 256, 0, st>>>(
        N, P, (const V4<float>*)lmrec_at(ctx, k), (const V4<float>*)lmlo_at(ctx, k), (const V4<float>*)ctx->lm_alt,
        (V4<float>*)lmrec_at(ctx, k + 1), (V4<float>*)lmlo_at(ctx, k + 1), (uint8_t*)ctx->lm_rs);
  } else {
    k_fix_cams<double><<<(M + 127) / 128, 128, 0, st>>>(M, P, (double*)ctx->cam_x, (double*)ctx->cam_dx,
                                                        (double*)ctx->cam_Rbar, (double*)ctx->cam_S,
                                                        (double*)ctx->cam_E, (uint8_t*)ctx->cam_rs,
                                                        (V4<double>*)pack_at(ctx, k + 1));
    k_fix_lms<double, false><<<(N + 255) / 256, 256, 0, st>>>(
        N, P, (const V4<double>*)lmrec_at(ctx, k), nullptr, (const V4<double>*)ctx->lm_alt,
        (V4<double>*)lmrec_at(ctx, k + 1), nullptr, (uint8_t*)ctx->lm_rs);
  }
  ctx->launches += 2;
  return cudaGetLastError();
}

// F(x^k) of the current state into d_obj (device double): per-tile sums and their
// reduction. With prepare, the pack is first rebuilt from the state (gamma entry 0 is
// read; it does not affect F).
daba_status enqueue_objective(daba_ctx* ctx, cudaStream_t st, bool prepare) {
  if (prepare) {
    CK(cudaMemsetAsync(ctx->d_it, 0, sizeof(int), st));
    CK(cudaMemsetAsync(ctx->d_gam, 0, sizeof(double), st));
    CK(launch_prepare(ctx, st, ctx->k));
  }
  CK(launch_pass(ctx, st, 6, ctx->k));
  ctx->launches++;
  if (is_mixed(ctx))
    k_sum<float><<<1, 1024, 0, st>>>(ctx->n_chunks, (const float*)ctx->chunk_f, ctx->s_norm * ctx->s_norm,
                                     (double*)ctx->d_obj);
  else
    k_sum<double><<<1, 1024, 0, st>>>(ctx->n_chunks, (const double*)ctx->chunk_f, ctx->s_norm * ctx->s_norm,
                                      (double*)ctx->d_obj);
  CK(cudaGetLastError());
  return DABA_OK;
}

// A timing event record: inside a stream capture an event-record node of the graph (a plain
// cudaEventRecord there would only mark a dependency; the external flag is refused outside a
// capture), outside one an ordinary record.
cudaError_t rec_time(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t q = cudaStreamIsCapturing(s, &cs);
  if (q != cudaSuccess) return q;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                             : cudaEventRecord(e, s);
}

cudaEvent_t ev(daba_ctx* ctx, size_t i) {
  while (ctx->events.size() <= i) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    ctx->events.push_back(e);
  }
  return ctx->events[i];
}

void pipe_streams_free(daba_ctx* ctx) {
  for (auto& pool : ctx->s_pool)
    for (cudaStream_t& q : pool) {
      if (q) {
        cudaStreamSynchronize(q);
        cudaStreamDestroy(q);
      }
      q = nullptr;
    }
  for (cudaEvent_t e : ctx->ev_rng)
    if (e) cudaEventDestroy(e);
  ctx->ev_rng.clear();
}

// The ranges of the range schedule for the current observations (daba_set_pipeline): camera
// bounds at the first cameras whose observations start at or after r nnz / R (a camera is never
// split; empty ranges are dropped), the landmark tiles grouped by the last range observing them.
daba_status pipe_cut(daba_ctx* ctx, cudaStream_t st) {
  ctx->pipe_R = 1;
  const int R = ctx->pipe.ranges;
  if (R <= 1 || ctx->h_tile_lm.empty()) return DABA_OK;
  const int M = ctx->M;
  std::vector<int> cb{0};
  int i = 0;
  for (int r = 1; r < R; ++r) {
    const double at = (double)r * (double)ctx->nnz / R;
    while (i < M && (double)ctx->h_cam_ptr[i] < at) ++i;
    if (i > cb.back() && i < M && ctx->h_cam_chunk_ptr[i] > ctx->h_cam_chunk_ptr[cb.back()]) cb.push_back(i);
  }
  if (ctx->h_cam_chunk_ptr[M] <= ctx->h_cam_chunk_ptr[cb.back()]) cb.pop_back();   // no chunks after the last bound
  cb.push_back(M);
  const int Rn = (int)cb.size() - 1;
  if (Rn <= 1) return DABA_OK;
  std::vector<int> rng_of(M);
  for (int r = 0; r < Rn; ++r)
    for (int c = cb[r]; c < cb[r + 1]; ++c) rng_of[c] = r;
  // per tile the lowest and the highest range of its observing cameras
  const int n_tiles = ctx->n_tiles;
  std::vector<int> tlo(n_tiles), thi(n_tiles);
  for (int t = 0; t < n_tiles; ++t) {
    int lo = Rn, hi = 0;
    const int ob = ctx->h_lmi_ptr[ctx->h_tile_lm[t]], oe = ctx->h_lmi_ptr[ctx->h_tile_lm[t + 1]];
    for (int o = ob; o < oe; ++o) {
      const int r = rng_of[ctx->h_cam_idx[ctx->h_li_order[o]]];
      lo = std::min(lo, r);
      hi = std::max(hi, r);
    }
    tlo[t] = oe > ob ? lo : 0;
    thi[t] = oe > ob ? hi : 0;
  }
  std::vector<int32_t> tl;
  tl.reserve(n_tiles);
  std::vector<int> nt(2 * Rn, 0), minr(Rn);
  for (int r = 0; r < Rn; ++r) {
    minr[r] = r;
    for (int c = 0; c < 2; ++c) {
      const int t0 = c == 0 ? 0 : ctx->tile_class_end[0], t1 = ctx->tile_class_end[c];
      for (int t = t0; t < t1; ++t)
        if (thi[t] == r) {
          tl.push_back(t);
          ++nt[2 * r + c];
          minr[r] = std::min(minr[r], tlo[t]);
        }
    }
  }
  CK(cudaMemcpyAsync(ctx->d_tlist, tl.data(), tl.size() * 4, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  ctx->pipe_cam = cb;
  ctx->pipe_chunk.resize(Rn + 1);
  for (int r = 0; r <= Rn; ++r) ctx->pipe_chunk[r] = ctx->h_cam_chunk_ptr[cb[r]];
  ctx->pipe_nt = nt;
  ctx->pipe_minr = minr;
  ctx->pipe_R = Rn;
  return DABA_OK;
}

void drop_graphs(daba_ctx* ctx) {
  for (auto& row : ctx->graph)
    for (cudaGraphExec_t& g : row) {
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
  for (int p = 0; p < 2; ++p) {
    if (ctx->run_graph[p]) cudaGraphExecDestroy(ctx->run_graph[p]);
    ctx->run_graph[p] = nullptr;
    ctx->run_graph_n[p] = 0;
  }
}

#define CE(call)                             \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return e_;        \
  } while (0)

// The range schedule applies (daba_set_pipeline): more than one range and the iteration is the
// default one (per-block restart, no coarse blocks, no per-kernel timing).
bool pipe_active(const daba_ctx* ctx) {
  return ctx->pipe_R > 1 && !ctx->timing && ctx->n_blocks == 0 && !ctx->persistent &&
         ctx->opt.restart_mode == DABA_RESTART_BLOCK;
}

// One iteration k on the range schedule, with pools of PIPE_POOL streams per role:
//   camera pass of range r (after the fork) --> camera solves of range r
//   camera passes of ranges minr[r] .. r -----> landmark tiles of class r
// then st waits for every camera solve and landmark launch and runs the reduction. Every kernel
// reads and writes what it does in the one-range order, and each camera solve and landmark tile
// waits for the camera-pass chunks it reads, so the results are the same bits.
cudaError_t enqueue_iter_ranges(daba_ctx* ctx, cudaStream_t st, int64_t kk) {
  const int R = ctx->pipe_R;
  while ((int)ctx->ev_rng.size() < 3 * R) {
    cudaEvent_t e = nullptr;
    CE(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->ev_rng.push_back(e);
  }
  cudaEvent_t* E = ctx->ev_rng.data();
  unsigned* ctr = (unsigned*)ctx->d_ctr;
  CE(cudaEventRecord(ctx->ev_fork, st));
  for (int r = 0; r < R; ++r) {   // camera passes
    cudaStream_t q = ctx->s_pool[0][r % PIPE_POOL];
    if (r < PIPE_POOL) CE(cudaStreamWaitEvent(q, ctx->ev_fork, 0));
    PassRange pr;
    pr.c0 = ctx->pipe_chunk[r];
    pr.c1 = ctx->pipe_chunk[r + 1];
    if (ctx->pipe.cpass_warps > 0) {
      pr.ctr = ctr + 4 * r;
      pr.grid = ctx->pipe.cpass_warps * ctx->n_sm / CPASS_WARPS;
    }
    CE(launch_pass(ctx, q, 1, kk, pr));
    CE(cudaEventRecord(E[3 * r], q));
  }
  for (int r = 0; r < R; ++r) {   // camera solves
    cudaStream_t q = ctx->s_pool[1][r % PIPE_POOL];
    CE(cudaStreamWaitEvent(q, E[3 * r], 0));
    CE(launch_camsolve(ctx, q, kk, ctx->pipe_cam[r], ctx->pipe_cam[r + 1]));
    CE(cudaEventRecord(E[3 * r + 1], q));
  }
  int q0 = 0;
  for (int r = 0; r < R; ++r) {   // landmark tiles by class
    cudaStream_t q = ctx->s_pool[2][r % PIPE_POOL];
    for (int c = ctx->pipe_minr[r]; c <= r; ++c) CE(cudaStreamWaitEvent(q, E[3 * c], 0));
    TileRange tr;
    tr.tlist = (const int*)ctx->d_tlist;
    tr.q[0] = q0;
    tr.n[0] = ctx->pipe_nt[2 * r];
    tr.q[1] = q0 + tr.n[0];
    tr.n[1] = ctx->pipe_nt[2 * r + 1];
    q0 = tr.q[1] + tr.n[1];
    if (ctx->pipe.lpass_ctas > 0) {
      tr.ctr = ctr + 4 * r + 2;
      tr.grid = ctx->pipe.lpass_ctas * ctx->n_sm;
    }
    CE(launch_lpass(ctx, q, kk, tr));
    CE(cudaEventRecord(E[3 * r + 2], q));
  }
  for (int r = 0; r < R; ++r) {
    CE(cudaStreamWaitEvent(st, E[3 * r + 1], 0));
    CE(cudaStreamWaitEvent(st, E[3 * r + 2], 0));
  }
  CE(launch_finalize(ctx, st));
  return cudaSuccess;
}

// Enqueues n iterations of Algorithm 1 starting at an iteration of parity k0 & 1 on stream st
// (the camera pass, then the landmark pass and the camera solves on two priority streams,
// joined before the reduction; or the range schedule); with timing, records the per-kernel
// events from index evi.
cudaError_t enqueue_iters(daba_ctx* ctx, cudaStream_t st, int64_t k0, int n, size_t evi) {
  for (int j = 0; j < n; ++j) {
    const int64_t kk = k0 + j;
    if (pipe_active(ctx)) {
      CE(enqueue_iter_ranges(ctx, st, kk));
      continue;
    }
    CE(cudaEventRecord(ctx->ev_fork, st));
    CE(cudaStreamWaitEvent(ctx->s_hi, ctx->ev_fork, 0));
    if (ctx->timing) CE(rec_time(ev(ctx, evi + 0), ctx->s_hi));
    CE(launch_pass(ctx, ctx->s_hi, 1, kk));
    if (ctx->timing) CE(rec_time(ev(ctx, evi + 1), ctx->s_hi));
    CE(cudaEventRecord(ctx->ev_hi, ctx->s_hi));
    CE(cudaStreamWaitEvent(ctx->s_lo, ctx->ev_hi, 0));
    // The camera solves go on the high-priority stream and are enqueued before the landmark
    // pass: with direct launches the priority decides which kernel's CTAs the SMs take first; in
    // a graph the priority made no measurable difference and the order of the nodes did. Measured (ms per
    // iteration, graph / direct): 0.729 / 0.746 on the tourism workload and 0.367 / 0.388 on the
    // 512-scene batch, against 0.757 / 0.748 and 0.421 / 0.386 with the landmark pass enqueued
    // first, and 0.78 / 0.43 direct with the landmark pass on the high-priority stream.
    CE(launch_camsolve(ctx, ctx->s_hi, kk));
    if (ctx->timing) CE(rec_time(ev(ctx, evi + 2), ctx->s_hi));
    CE(cudaEventRecord(ctx->ev_hi, ctx->s_hi));
    if (ctx->timing) CE(rec_time(ev(ctx, evi + 3), ctx->s_lo));
    CE(launch_lpass(ctx, ctx->s_lo, kk));
    if (ctx->timing) CE(rec_time(ev(ctx, evi + 4), ctx->s_lo));
    CE(cudaEventRecord(ctx->ev_lo, ctx->s_lo));
    CE(cudaStreamWaitEvent(st, ctx->ev_hi, 0));
    CE(cudaStreamWaitEvent(st, ctx->ev_lo, 0));
    if (ctx->timing) CE(rec_time(ev(ctx, evi + 5), st));
    CE(launch_finalize(ctx, st));
    CE(launch_fixups(ctx, st, kk));
    if (ctx->timing) CE(rec_time(ev(ctx, evi + 6), st));
    if (ctx->timing) evi += 7;
  }
  return cudaSuccess;
}
#undef CE

// Graph instantiation: on the range schedule the kernel nodes keep the priorities of the
// streams they were captured on (otherwise a graph ignores them).
cudaError_t instantiate(const daba_ctx* ctx, cudaGraphExec_t* exec, cudaGraph_t g) {
  return cudaGraphInstantiateWithFlags(exec, g, pipe_active(ctx) ? cudaGraphInstantiateFlagUseNodePriority : 0);
}

// Captures the four iteration graphs (GRAPH_ITERS and 1 iterations, even and odd start) on
// s_cap; their launch counts go to graph_nl.
daba_status ensure_graphs(daba_ctx* ctx) {
  if (ctx->graph[0][0]) return DABA_OK;
  const bool timing = ctx->timing;
  ctx->timing = false;
  for (int gi = 0; gi < 2; ++gi)
    for (int par = 0; par < 2; ++par) {
      const int64_t l0 = ctx->launches;
      cudaError_t e = cudaStreamBeginCapture(ctx->s_cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t e1 = enqueue_iters(ctx, ctx->s_cap, par, gi == 0 ? GRAPH_ITERS : 1, 0);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(ctx->s_cap, &g);
        e = e1 != cudaSuccess ? e1 : e2;
        if (e == cudaSuccess) e = instantiate(ctx, &ctx->graph[gi][par], g);
        if (g) cudaGraphDestroy(g);
      }
      ctx->graph_nl[gi] = ctx->launches - l0;
      ctx->launches = l0;
      if (e != cudaSuccess) {
        cudaGetLastError();
        drop_graphs(ctx);
        ctx->timing = timing;
        return fail(ctx, DABA_ERR_CUDA, "capturing the iteration graph: %s", cudaGetErrorString(e));
      }
    }
  ctx->timing = timing;
  return DABA_OK;
}

// The graph of a whole run of n iterations from an iteration of the current parity: the
// prepare kernel, then the n iterations (captured once per parity, length and timing mode).
// With timing the graph records the per-kernel events of the run (event 0 and 1 around the
// prepare kernel, then 7 per iteration, as the direct launches do).
daba_status ensure_run_graph(daba_ctx* ctx, int n) {
  const int par = (int)(ctx->k & 1);
  const bool timing = ctx->timing;
  if (ctx->run_graph[par] && ctx->run_graph_n[par] == n && ctx->run_graph_timing[par] == timing) return DABA_OK;
  if (ctx->run_graph[par]) cudaGraphExecDestroy(ctx->run_graph[par]);
  ctx->run_graph[par] = nullptr;
  ctx->run_graph_n[par] = 0;
  if (timing) ev(ctx, 2 + 7 * (size_t)n);   // every event the capture records exists before it
  const int64_t l0 = ctx->launches;
  cudaError_t e = cudaStreamBeginCapture(ctx->s_cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = timing ? rec_time(ev(ctx, 0), ctx->s_cap) : cudaSuccess;
    if (e1 == cudaSuccess) e1 = launch_prepare(ctx, ctx->s_cap, ctx->k);
    if (e1 == cudaSuccess && timing) e1 = rec_time(ev(ctx, 1), ctx->s_cap);
    if (e1 == cudaSuccess) e1 = enqueue_iters(ctx, ctx->s_cap, ctx->k, n, timing ? 2 : 0);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(ctx->s_cap, &g);
    e = e1 != cudaSuccess ? e1 : e2;
    if (e == cudaSuccess) e = instantiate(ctx, &ctx->run_graph[par], g);
    if (g) cudaGraphDestroy(g);
  }
  ctx->run_graph_nl[par] = ctx->launches - l0;
  ctx->launches = l0;
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->run_graph[par] = nullptr;
    return fail(ctx, DABA_ERR_CUDA, "capturing the run graph: %s", cudaGetErrorString(e));
  }
  ctx->run_graph_n[par] = n;
  ctx->run_graph_timing[par] = timing;
  return DABA_OK;
}

template <int LOSS, class Real, class Real2, bool HAS_LO>
cudaError_t launch_grad_t(daba_ctx* ctx, cudaStream_t st) {
  const LossC<Real> L = loss_consts<Real>(ctx);
  if (ctx->n_chunks == 0) return cudaSuccess;
  k_grad_obs<LOSS, Real, Real2, HAS_LO><<<ctx->n_chunks, 32, 0, st>>>(
      ctx->n_chunks, (const int*)ctx->chunk_cam, (const int*)ctx->chunk_beg, (const int*)ctx->c_lm,
      (const Real2*)ctx->c_u, (const int*)ctx->c_rpos, (const int*)ctx->d_ci_order, (const V4<Real>*)pack_at(ctx, ctx->k),
      (const V4<Real>*)lmrec_at(ctx, ctx->k), (const V4<float>*)lmlo_at(ctx, ctx->k), L, ctx->s_norm,
      (Real*)ctx->chunk_part, (V4<Real>*)ctx->rec_a, (double2*)ctx->rec_b);
  return cudaGetLastError();
}

template <class Real, class Real2, bool HAS_LO>
cudaError_t launch_grad_by_loss(daba_ctx* ctx, cudaStream_t st) {
  switch (ctx->opt.loss) {
    case DABA_LOSS_TRIVIAL: return launch_grad_t<LOSS_TRIVIAL, Real, Real2, HAS_LO>(ctx, st);
    case DABA_LOSS_HUBER: return launch_grad_t<LOSS_HUBER, Real, Real2, HAS_LO>(ctx, st);
    case DABA_LOSS_CAUCHY: return launch_grad_t<LOSS_CAUCHY, Real, Real2, HAS_LO>(ctx, st);
    default: return launch_grad_t<LOSS_WELSCH, Real, Real2, HAS_LO>(ctx, st);
  }
}

// ---- reverse mode -----------------------------------------------------------
constexpr int ADJ_CKPT = 10;   // iterations between the states kept by the forward sweep

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// A copy of everything an iteration reads besides the fixed setup: the camera state, its
// restart slack and accumulated E, the landmark records and the first-iteration flag.
struct SlotLayout {
  size_t x, dx, S, E, lm, first, bytes;
};
SlotLayout slot_layout(const daba_ctx* c) {
  SlotLayout L;
  size_t o = 0;
  L.x = o;
  o = align256(o + (size_t)c->M * CSTRIDE * 8);
  L.dx = o;
  o = align256(o + (size_t)c->M * CSTRIDE * 8);
  L.S = o;
  o = align256(o + (size_t)c->M * 8);
  L.E = o;
  o = align256(o + (size_t)c->M * 8);
  L.lm = o;
  o = align256(o + (size_t)c->N * LREC * 8);
  L.first = o;
  o = align256(o + 16);
  L.bytes = o;
  return L;
}

// What the adjoint of one iteration reads besides the state: the chunk partials of the camera
// statistics, the landmarks' (a, b) sums at x̄ and x^k, and the restart decisions.
struct ItLayout {
  size_t part, sums, rs_cam, rs_lm, bytes;
};
ItLayout it_layout(const daba_ctx* c) {
  ItLayout L;
  size_t o = 0;
  L.part = o;
  o = align256(o + (size_t)c->max_chunks * CP_STRIDE * 8);
  L.sums = o;
  o = align256(o + (size_t)c->N * 8 * 8);
  L.rs_cam = o;
  o = align256(o + (size_t)c->M);
  L.rs_lm = o;
  o = align256(o + (size_t)c->N);
  L.bytes = o;
  return L;
}

daba_status ensure_adjoint(daba_ctx* ctx, size_t n_slots) {
  daba_status s;
  const size_t M = ctx->M, N = ctx->N;
  if (!ctx->st_bar) {
    for (int q = 0; q < 3; ++q) {
      if ((s = dalloc(ctx, &ctx->adj_c[q], M * AC_N * 8)) != DABA_OK) return s;
      if ((s = dalloc(ctx, &ctx->adj_l[q], N * AL_N * 8)) != DABA_OK) return s;
    }
    for (int q = 0; q < 2; ++q) {
      if ((s = dalloc(ctx, &ctx->zb_c[q], M * AC_N * 8)) != DABA_OK) return s;
      if ((s = dalloc(ctx, &ctx->zb_l[q], N * AL_N * 8)) != DABA_OK) return s;
    }
    if ((s = dalloc(ctx, &ctx->ab_bar, N * 4 * 8)) != DABA_OK) return s;
    if ((s = dalloc(ctx, &ctx->g_u, (size_t)ctx->nnz * 16)) != DABA_OK) return s;
    if ((s = dalloc(ctx, &ctx->st_bar, M * 40 * 8)) != DABA_OK) return s;
  }
  const size_t b = slot_layout(ctx).bytes;
  while (ctx->slots.size() < n_slots) {
    void* p = nullptr;
    if ((s = dalloc(ctx, &p, b)) != DABA_OK) return s;
    ctx->slots.push_back(p);
  }
  const size_t bi = it_layout(ctx).bytes;
  while (ctx->itslots.size() < (size_t)ADJ_CKPT) {
    void* p = nullptr;
    if ((s = dalloc(ctx, &p, bi)) != DABA_OK) return s;
    ctx->itslots.push_back(p);
  }
  return DABA_OK;
}

// keeps the statistics and decisions of the iteration just run (its landmark sums were written
// by the landmark pass through lm_sums_out)
cudaError_t save_iteration(daba_ctx* ctx, void* slot, cudaStream_t st) {
  const ItLayout L = it_layout(ctx);
  char* b = (char*)slot;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(b + L.part, ctx->chunk_part, (size_t)ctx->n_chunks * CP_STRIDE * 8, cudaMemcpyDeviceToDevice,
                           st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(b + L.rs_cam, ctx->cam_rs, (size_t)ctx->M, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  return cudaMemcpyAsync(b + L.rs_lm, ctx->lm_rs, (size_t)ctx->N, cudaMemcpyDeviceToDevice, st);
}

cudaError_t save_state(daba_ctx* ctx, void* slot, cudaStream_t st) {
  const SlotLayout L = slot_layout(ctx);
  char* b = (char*)slot;
  const size_t cb = (size_t)ctx->M * CSTRIDE * 8;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(b + L.x, ctx->cam_x, cb, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(b + L.dx, ctx->cam_dx, cb, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(b + L.S, ctx->cam_S, (size_t)ctx->M * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(b + L.E, ctx->cam_E, (size_t)ctx->M * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(b + L.lm, lmrec_at(ctx, ctx->k), (size_t)ctx->N * LREC * 8, cudaMemcpyDeviceToDevice,
                           st)) != cudaSuccess)
    return e;
  return cudaMemcpyAsync(b + L.first, ctx->d_first, sizeof(int), cudaMemcpyDeviceToDevice, st);
}

// restores a copy taken at iteration k (the landmark records go to the buffer of k's parity)
cudaError_t restore_state(daba_ctx* ctx, const void* slot, int64_t k, double s_k, cudaStream_t st) {
  const SlotLayout L = slot_layout(ctx);
  const char* b = (const char*)slot;
  const size_t cb = (size_t)ctx->M * CSTRIDE * 8;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(ctx->cam_x, b + L.x, cb, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(ctx->cam_dx, b + L.dx, cb, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(ctx->cam_S, b + L.S, (size_t)ctx->M * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(ctx->cam_E, b + L.E, (size_t)ctx->M * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(lmrec_at(ctx, k), b + L.lm, (size_t)ctx->N * LREC * 8, cudaMemcpyDeviceToDevice, st)) !=
      cudaSuccess)
    return e;
  ctx->k = k;
  ctx->s_k = s_k;
  return cudaMemcpyAsync(ctx->d_first, b + L.first, sizeof(int), cudaMemcpyDeviceToDevice, st);
}

// The entry state of daba_run: everything an iteration changes and a later call reads. It is
// copied (device to device, on the run's stream) before the first launch and put back when the
// run fails, so that a failing daba_run leaves the iterate and the restart metrics unchanged.
// The landmark records of x^k live in the buffer of k's parity, which a run of one iteration
// does not write: that run keeps no copy of them.
struct BackupLayout {
  size_t x, dx, S, E, F, Fb, crs, lm, lo, lrs, lF, lFb, first, bytes;
};
BackupLayout backup_layout(const daba_ctx* c) {
  BackupLayout L;
  const size_t M = c->M, N = c->N;
  size_t o = 0;
  auto take = [&](size_t& f, size_t b) {
    f = o;
    o = align256(o + b);
  };
  take(L.x, M * CSTRIDE * 8);
  take(L.dx, M * CSTRIDE * 8);
  take(L.S, M * 8);
  take(L.E, M * 8);
  take(L.F, M * 8);
  take(L.Fb, M * 8);
  take(L.crs, M);
  take(L.lm, N * LREC * real_sz(c));
  take(L.lo, N * 16);
  take(L.lrs, N);
  take(L.lF, is_mixed(c) ? 0 : N * 8);
  take(L.lFb, is_mixed(c) ? 0 : N * 8);
  take(L.first, 16);
  L.bytes = o;
  return L;
}

// copies between the live buffers and the backup (to_backup: live -> backup); lm_too: the
// landmark records and their low parts of iteration k as well
cudaError_t backup_copy(daba_ctx* ctx, bool to_backup, int64_t k, bool lm_too, cudaStream_t st) {
  const BackupLayout L = backup_layout(ctx);
  char* b = (char*)ctx->bk;
  const size_t M = ctx->M, N = ctx->N;
  struct Item {
    void* live;
    size_t off, bytes;
  };
  std::vector<Item> items = {{ctx->cam_x, L.x, M * CSTRIDE * 8}, {ctx->cam_dx, L.dx, M * CSTRIDE * 8},
                             {ctx->cam_S, L.S, M * 8},          {ctx->cam_E, L.E, M * 8},
                             {ctx->cam_F, L.F, M * 8},          {ctx->cam_Fb, L.Fb, M * 8},
                             {ctx->cam_rs, L.crs, M},           {ctx->lm_rs, L.lrs, N},
                             {ctx->d_first, L.first, sizeof(int)}};
  if (!is_mixed(ctx)) {
    items.push_back({ctx->lm_Fd, L.lF, N * 8});
    items.push_back({ctx->lm_Fbd, L.lFb, N * 8});
  }
  if (lm_too) {
    items.push_back({lmrec_at(ctx, k), L.lm, N * LREC * real_sz(ctx)});
    items.push_back({lmlo_at(ctx, k), L.lo, N * 16});
  }
  for (const Item& it : items) {
    void* dst = to_backup ? (void*)(b + it.off) : it.live;
    const void* src = to_backup ? (const void*)it.live : (const void*)(b + it.off);
    cudaError_t e = cudaMemcpyAsync(dst, src, it.bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// n iterations from the current state with direct launches (as daba_run without its
// synchronisation and objective trace)
cudaError_t advance(daba_ctx* ctx, cudaStream_t st, int n) {
  std::vector<double> gam((size_t)n + 1);
  const double s_from = ctx->s_k;
  double sk = s_from;
  for (int j = 0; j <= n; ++j) {
    const double s_next = (std::sqrt(4.0 * sk * sk + 1.0) + 1.0) / 2.0;
    gam[j] = (sk - 1.0) / s_next;
    sk = s_next;
    if (j == n - 1) ctx->s_k = sk;
  }
  cudaError_t e;
  if ((e = cudaMemcpyAsync(ctx->d_gam, gam.data(), ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  // momentum reset: the reduction continues s on the device from s^(k); s^(k+n) is read back
  if (ctx->opt.momentum_reset &&
      (e = cudaMemcpyAsync(ctx->s_dev, &s_from, 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(ctx->d_it, 0, sizeof(int), st)) != cudaSuccess) return e;
  if ((e = launch_prepare(ctx, st, ctx->k)) != cudaSuccess) return e;
  if ((e = enqueue_iters(ctx, st, ctx->k, n, 0)) != cudaSuccess) return e;
  ctx->k += n;
  if (ctx->opt.momentum_reset) {
    if ((e = cudaMemcpyAsync(&ctx->s_k, ctx->s_dev, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The adjoint of iteration k, whose forward results (statistics, records, decisions, pass
// pack) are in the live buffers; slot holds x^k and x^k - x^(k-1) of the cameras.
// a1: adjoint of x^(k+1) (read); a0, am: adjoints of x^k and x^(k-1) (accumulated).
template <int LOSS>
cudaError_t adjoint_iter(daba_ctx* ctx, cudaStream_t st, int64_t k, double gamma, const void* slot, const void* itslot,
                         int a1, int a0, int am) {
  const SlotLayout Ly = slot_layout(ctx);
  const ItLayout Li = it_layout(ctx);
  const double* sx = (const double*)((const char*)slot + Ly.x);
  const double* sdx = (const double*)((const char*)slot + Ly.dx);
  const double* part = (const double*)((const char*)itslot + Li.part);
  const double* sums = (const double*)((const char*)itslot + Li.sums);
  const uint8_t* rs_cam = (const uint8_t*)((const char*)itslot + Li.rs_cam);
  const uint8_t* rs_lm = (const uint8_t*)((const char*)itslot + Li.rs_lm);
  const int M = ctx->M, N = ctx->N;
  const int acc = ctx->opt.accelerated;
  const double xi = ctx->opt.xi;
  cudaError_t e;
  for (int q = 0; q < 2; ++q) {
    if ((e = cudaMemsetAsync(ctx->zb_c[q], 0, (size_t)M * AC_N * 8, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ctx->zb_l[q], 0, (size_t)N * AL_N * 8, st)) != cudaSuccess) return e;
  }
  if (M > 0)
    k_adj_cams<<<(M + 63) / 64, 64, 0, st>>>(M, (const int*)ctx->cam_chunk_ptr, part, sx, sdx,
                                             gamma, rs_cam, acc, xi, ctx->opt.cam_alternations,
                                             ctx->opt.cam_solver == DABA_CAM_LM ? 1 : 0,
                                             (const double*)ctx->adj_c[a1], (double*)ctx->st_bar,
                                             (double*)ctx->zb_c[0], (double*)ctx->zb_c[1]);
  if (N > 0)
    k_adj_lms<<<(N + 255) / 256, 256, 0, st>>>(N, sums, rs_lm, acc, xi, (const double*)ctx->adj_l[a1],
                                               (double*)ctx->ab_bar, (double*)ctx->zb_l[0], (double*)ctx->zb_l[1]);
  // rec_a / rec_b (free here) take the landmark terms at xbar / x^k
  if (ctx->n_chunks > 0)
    k_adj_obs<LOSS><<<ctx->n_chunks, 32, 0, st>>>(
        ctx->n_chunks, (const int*)ctx->chunk_cam, (const int*)ctx->chunk_beg, (const int*)ctx->c_lm,
        (const double2*)ctx->c_u, (const int*)ctx->c_rpos, (const int*)ctx->d_ci_order,
        (const V4<double>*)pack_at(ctx, k), (const V4<double>*)lmrec_at(ctx, k), gamma, rs_cam,
        rs_lm, acc, loss_consts<double>(ctx), 1.0 / ctx->s_norm, (const double*)ctx->st_bar,
        (const double*)ctx->ab_bar, (double*)ctx->chunk_part, (V4<double>*)ctx->rec_a, (V4<double>*)ctx->rec_b,
        (double2*)ctx->g_u);
  if (M > 0)
    k_adj_cams_sum<<<(M + 127) / 128, 128, 0, st>>>(M, (const int*)ctx->cam_chunk_ptr, (const double*)ctx->chunk_part,
                                                    sx, sdx, gamma, (const double*)ctx->zb_c[0],
                                                    (const double*)ctx->zb_c[1], (double*)ctx->adj_c[a0],
                                                    (double*)ctx->adj_c[am]);
  if (ctx->n_tiles > 0)
    k_adj_lms_sum<<<ctx->n_tiles, LPASS_THREADS, 0, st>>>(
        (const int*)ctx->tile_lm, (const int*)ctx->lm_ptr, (const uint16_t*)ctx->t_inv, (const V4<double>*)ctx->rec_a,
        (const V4<double>*)ctx->rec_b, (const double*)ctx->zb_l[0], (const double*)ctx->zb_l[1], gamma,
        (double*)ctx->adj_l[a0], (double*)ctx->adj_l[am]);
  ctx->launches += 5;
  return cudaGetLastError();
}

cudaError_t adjoint_iter_by_loss(daba_ctx* ctx, cudaStream_t st, int64_t k, double gamma, const void* slot,
                                 const void* itslot, int a1, int a0, int am) {
  switch (ctx->opt.loss) {
    case DABA_LOSS_TRIVIAL: return adjoint_iter<LOSS_TRIVIAL>(ctx, st, k, gamma, slot, itslot, a1, a0, am);
    case DABA_LOSS_HUBER: return adjoint_iter<LOSS_HUBER>(ctx, st, k, gamma, slot, itslot, a1, a0, am);
    case DABA_LOSS_CAUCHY: return adjoint_iter<LOSS_CAUCHY>(ctx, st, k, gamma, slot, itslot, a1, a0, am);
    default: return adjoint_iter<LOSS_WELSCH>(ctx, st, k, gamma, slot, itslot, a1, a0, am);
  }
}

daba_status run_iterations(daba_ctx* ctx, int32_t iters, double* obj_trace, int32_t* restarts, cudaStream_t st);
daba_status pipe_apply(daba_ctx* ctx, const daba_pipeline& p);

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

void daba_default_options(daba_options* o) {
  if (!o) return;
  o->loss = DABA_LOSS_HUBER;
  o->loss_scale_px = 1.0;
  o->xi = 1e-10;
  o->eta = 0.5;
  o->accelerated = 1;
  o->cam_alternations = 2;
  o->pixel_scale = 0.0;
  o->prec = DABA_MIXED;
  o->chunk_obs = 0;
  o->tile_obs = 0;
  o->tile_lms = 0;
  o->restart_mode = DABA_RESTART_BLOCK;
  o->momentum_reset = 0;
  o->cam_solver = DABA_CAM_SCAM;
}

const char* daba_last_error(const daba_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t daba_last_launch_count(const daba_ctx* ctx) { return ctx ? ctx->launches : 0; }

daba_status daba_device_bytes(const daba_ctx* ctx, int64_t* bytes, int64_t* peak) {
  if (!ctx || (!bytes && !peak)) return DABA_ERR_ARG;
  size_t b = ctx->dev_bytes, pk = ctx->dev_peak;
  if (ctx->shadow) {   // the FP64 context owned for the reverse mode of a MIXED context
    b += ctx->shadow->dev_bytes;
    pk += ctx->shadow->dev_peak;
  }
  if (bytes) *bytes = (int64_t)b;
  if (peak) *peak = (int64_t)pk;
  return DABA_OK;
}

void daba_destroy(daba_ctx* ctx) {
  if (!ctx) return;
  if (ctx->s_hi) cudaStreamSynchronize(ctx->s_hi);
  if (ctx->s_lo) cudaStreamSynchronize(ctx->s_lo);
  if (ctx->s_cap) cudaStreamSynchronize(ctx->s_cap);
  drop_graphs(ctx);
  for (const auto& a : ctx->allocs) cudaFree(a.first);
  for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
  for (cudaEvent_t e : {ctx->ev_fork, ctx->ev_hi, ctx->ev_lo, ctx->ev_cap0, ctx->ev_cap1})
    if (e) cudaEventDestroy(e);
  pipe_streams_free(ctx);
  if (ctx->s_hi) cudaStreamDestroy(ctx->s_hi);
  if (ctx->shadow) daba_destroy(ctx->shadow);
  if (ctx->s_lo) cudaStreamDestroy(ctx->s_lo);
  if (ctx->s_cap) cudaStreamDestroy(ctx->s_cap);
  delete ctx;
}

daba_status daba_create(int32_t M, int32_t N, int64_t nnz, const daba_options* opt, daba_ctx** out) {
  if (!out) return DABA_ERR_ARG;
  *out = nullptr;
  daba_ctx* ctx = new daba_ctx();
  daba_status st = DABA_OK;
  auto bad = [&](const char* why) {
    daba_destroy(ctx);
    return DABA_ERR_ARG;
    (void)why;
  };
  if (M < 1 || N < 1 || nnz < 1 || nnz >= (int64_t(1) << 31)) return bad("sizes");
  if (opt)
    ctx->opt = *opt;
  else
    daba_default_options(&ctx->opt);
  daba_options& o = ctx->opt;
  if (o.chunk_obs == 0) o.chunk_obs = CHUNK_OBS;
  if (o.tile_obs == 0) o.tile_obs = TILE_OBS;
  if (o.tile_lms == 0) o.tile_lms = TILE_LMS;
  if (o.chunk_obs < 32 || o.chunk_obs > 65536 || o.tile_obs < 32 || o.tile_obs > BIG_TILE_OBS || o.tile_lms < 1 ||
      o.tile_lms > LPASS_THREADS)
    return bad("schedule");
  if (!(o.xi > 0) || !(o.eta > 0) || !(o.eta <= 1) || o.cam_alternations < 1 || o.cam_alternations > 64 ||
      (int)o.loss < 0 || (int)o.loss > 3 || !(o.pixel_scale >= 0) ||
      (o.loss != DABA_LOSS_TRIVIAL && !(o.loss_scale_px > 0)) || (o.prec != DABA_FP64 && o.prec != DABA_MIXED) ||
      (o.restart_mode != DABA_RESTART_BLOCK && o.restart_mode != DABA_RESTART_GLOBAL) ||
      (o.momentum_reset != 0 && o.momentum_reset != 1) ||
      (o.momentum_reset && o.restart_mode != DABA_RESTART_GLOBAL) ||
      (o.cam_solver != DABA_CAM_SCAM && o.cam_solver != DABA_CAM_LM))
    return bad("options");
  ctx->M = M;
  ctx->N = N;
  ctx->nnz = nnz;
  cudaGetDevice(&ctx->dev);
  const size_t R = real_sz(ctx);
  ctx->max_chunks = (int)(M + nnz / o.chunk_obs + 1);
  ctx->max_tiles = (int)(2 * (nnz / o.tile_obs + N / o.tile_lms) + nnz / o.tile_obs + 8);
#define AL(field, bytes)                                   \
  if ((st = dalloc(ctx, &ctx->field, (bytes))) != DABA_OK) { \
    daba_ctx* c_ = ctx;                                    \
    daba_destroy(c_);                                      \
    return st;                                             \
  }
  AL(c_lm, nnz * 4);
  AL(c_u, nnz * 2 * R);
  AL(chunk_cam, (size_t)ctx->max_chunks * 4);
  AL(chunk_beg, (size_t)(ctx->max_chunks + 1) * 4);
  AL(cam_chunk_ptr, (size_t)(M + 1) * 4);
  AL(lm_ptr, (size_t)(N + 1) * 4);
  AL(tile_lm, (size_t)(ctx->max_tiles + 1) * 4);
  AL(c_rpos, nnz * 4);
  AL(t_inv, nnz * 2 + 16);   // + room for the 16-byte widening of the landmark pass copies
  AL(rec_a, nnz * 4 * R);
  AL(rec_b, nnz * 4 * R);
  AL(rec_c, nnz * 2 * R + 16);
  AL(cam_x, (size_t)M * CSTRIDE * 8);
  AL(cam_dx, (size_t)M * CSTRIDE * 8);
  AL(cam_Rbar, (size_t)M * 9 * 8);
  AL(pack2[0], (size_t)M * P4N * 4 * R);
  AL(pack2[1], (size_t)M * P4N * 4 * R);
  AL(cam_S, (size_t)M * 8);
  AL(cam_E, (size_t)M * 8);
  AL(cam_F, (size_t)M * 8);
  AL(cam_Fb, (size_t)M * 8);
  AL(cam_rs, (size_t)M);
  AL(lmrec2[0], (size_t)N * LREC * R);
  AL(lmrec2[1], (size_t)N * LREC * R);
  AL(lm_lo2[0], (size_t)N * 4 * 4);
  AL(lm_lo2[1], (size_t)N * 4 * 4);
  AL(lm_rs, (size_t)N);
  AL(lm_Fd, (size_t)N * 8);
  AL(lm_Fbd, (size_t)N * 8);
  AL(chunk_part, (size_t)ctx->max_chunks * CP_STRIDE * R);
  AL(chunk_f, (size_t)ctx->max_chunks * R);
  AL(tile_rs, (size_t)ctx->max_tiles * 4);
  AL(cam_Fsum, (size_t)M * 8);
  AL(fin_blk, (size_t)FIN_BLOCKS * 3 * 8);
  AL(fin_ticket, 16);
  AL(d_gam, (GSEG + 2) * 8);
  AL(d_it, 16);
  AL(d_first, 16);
  AL(d_flag, 16);
  AL(d_trace, (GSEG + 1) * 8);
  AL(d_rs, (GSEG + 1) * 4);
  AL(d_obj, 16);
  AL(st_cam, (size_t)M * 9 * 8);
  AL(st_lm, (size_t)N * 3 * 8);
  AL(d_linv, (size_t)N * 4);
  AL(d_chk, CHK_N * 4);
  AL(d_bad, 16);
  AL(d_scene_chunk, (size_t)(M + 1) * 4);
  AL(d_ci_order, nnz * 4);
  if (o.restart_mode == DABA_RESTART_GLOBAL) {
    AL(g_cam, (size_t)M * 8);
    AL(g_tile, (size_t)ctx->max_tiles * 8);
    AL(cam_alt, (size_t)M * 32 * 8);
    AL(lm_alt, (size_t)N * 2 * 4 * R);
    AL(g_fire, 16);
    AL(s_dev, 16);
  }
  AL(d_lperm, (size_t)N * 4);
  AL(d_scene_f, (size_t)M * 8);
  AL(bk, backup_layout(ctx).bytes);
  AL(d_gbar, 16);
  AL(d_tlist, (size_t)(ctx->max_tiles + 1) * 4);
  AL(d_ctr, 16 * PIPE_MAX_RANGES);
#undef AL
  cudaMemset(ctx->lm_lo2[0], 0, (size_t)N * 16);
  cudaMemset(ctx->lm_lo2[1], 0, (size_t)N * 16);
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (cudaStreamCreateWithPriority(&ctx->s_hi, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
      cudaStreamCreateWithPriority(&ctx->s_lo, cudaStreamNonBlocking, prio_least) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_hi, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_lo, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->s_cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_cap0, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_cap1, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    daba_destroy(ctx);
    return DABA_ERR_CUDA;
  }
  // the landmark pass's largest dynamic shared memory (one-landmark tiles), set once
  cudaFuncSetAttribute(k_lpass<float, float2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)lpass_smem_bytes<float>(BIG_TILE_OBS));
  cudaFuncSetAttribute(k_lpass<double, double2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)lpass_smem_bytes<double>(BIG_TILE_OBS));
  cudaMemset(ctx->d_flag, 0, 16);
  k_iota<<<(N + 255) / 256, 256>>>(N, (int*)ctx->d_linv);   // identity numbering until observations are set
  k_iota<<<(N + 255) / 256, 256>>>(N, (int*)ctx->d_lperm);
  cudaMemset(ctx->fin_ticket, 0, 16);
  cudaMemset(ctx->d_ctr, 0, 16 * PIPE_MAX_RANGES);
  cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->dev);
  cudaMemset(ctx->cam_rs, 0, (size_t)M);
  cudaMemset(ctx->lm_rs, 0, (size_t)N);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    daba_destroy(ctx);
    return DABA_ERR_CUDA;
  }
  // default schedule for problems of at least PIPE_MIN_NNZ observations: two camera ranges, or six
  // when the camera solves need more than one wave of CTAs (5 per SM), since later ranges then hide
  // more of them. Measured on B300, 100 MIXED iterations (ms per iteration): 26M observations and
  // 10k cameras (one wave) 0.742 with one range, 0.698 with 2, 0.702 with 4, 0.73 with 16; 8M
  // observations of 512 scenes and 29,784 cameras (1.3 waves) 0.361 / 0.356 with 2 / 0.359 with 4 /
  // 0.342 with 6 / 0.342 with 8; 1M observations 83.1 to 82.1 us with 2.
  daba_pipeline dp{};
  const bool solve_waves = (M + 31) / 32 > 5 * std::max(ctx->n_sm, 1);
  dp.ranges = nnz >= PIPE_MIN_NNZ ? (solve_waves ? 6 : 2) : 1;
  dp.prio[0] = 1;
  dp.prio[1] = 0;
  dp.prio[2] = 1;
  if (pipe_apply(ctx, dp) != DABA_OK) {
    daba_destroy(ctx);
    return DABA_ERR_CUDA;
  }
  *out = ctx;
  return DABA_OK;
}

daba_status daba_set_observations(daba_ctx* ctx, const int32_t* cam_idx, const int32_t* lm_idx, const double* uv,
                                  void* stream) {
  if (!ctx) return DABA_ERR_ARG;
  if (!cam_idx || !lm_idx || !uv) return fail(ctx, DABA_ERR_ARG, "null observation pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = ctx->nnz;
  std::vector<int32_t> ci(n), li(n);
  std::vector<double> uvh(2 * n);
  daba_status s;
  if ((s = fetch(ctx, ci.data(), cam_idx, n * 4, st)) != DABA_OK) return s;
  if ((s = fetch(ctx, li.data(), lm_idx, n * 4, st)) != DABA_OK) return s;
  if ((s = fetch(ctx, uvh.data(), uv, n * 16, st)) != DABA_OK) return s;
  for (int64_t o = 0; o < n; ++o) {
    if (ci[o] < 0 || ci[o] >= ctx->M || li[o] < 0 || li[o] >= ctx->N)
      return fail(ctx, DABA_ERR_INDEX, "observation %lld has index (%d, %d) out of range", (long long)o, ci[o], li[o]);
    if (!std::isfinite(uvh[2 * o]) || !std::isfinite(uvh[2 * o + 1]))
      return fail(ctx, DABA_ERR_NONFINITE, "observation %lld has a non-finite pixel", (long long)o);
  }
  const int M = ctx->M, N = ctx->N;
  std::vector<int32_t> c_order, cam_ptr, l_order, lm_ptr;
  counting_sort(ci, M, c_order, cam_ptr);
  counting_sort(li, N, l_order, lm_ptr);
  for (int j = 0; j < N; ++j)
    if (lm_ptr[j + 1] - lm_ptr[j] > MAX_TRACK)
      return fail(ctx, DABA_ERR_ARG, "landmark %d has %d observations (max %d)", j, lm_ptr[j + 1] - lm_ptr[j], MAX_TRACK);
  // internal landmark numbering: by the first camera that observes the landmark (landmarks
  // seen by the same cameras become neighbours), landmarks with long tracks last
  std::vector<int32_t> min_cam(N, M);
  for (int64_t o = 0; o < n; ++o) min_cam[li[o]] = std::min(min_cam[li[o]], ci[o]);
  // tile class of a landmark: 0 = at most TILE_OBS observations (small tiles),
  // 1 = longer (a tile of its own)
  const int tile_obs = ctx->opt.tile_obs, tile_lms = ctx->opt.tile_lms, chunk_obs = ctx->opt.chunk_obs;
  auto lclass = [&](int j) { return lm_ptr[j + 1] - lm_ptr[j] <= tile_obs ? 0 : 1; };
  std::vector<int32_t> lperm(N), linv(N);
  for (int j = 0; j < N; ++j) lperm[j] = j;
  std::stable_sort(lperm.begin(), lperm.end(), [&](int32_t a, int32_t b) {
    const int ca = lclass(a), cb = lclass(b);
    if (ca != cb) return ca < cb;
    return min_cam[a] < min_cam[b];
  });
  for (int q = 0; q < N; ++q) linv[lperm[q]] = q;
  std::vector<int32_t> lii(n), li_order, lmi_ptr;
  for (int64_t o = 0; o < n; ++o) lii[o] = linv[li[o]];
  counting_sort(lii, N, li_order, lmi_ptr);
  // device camera order: by camera, then internal landmark id, then input index (a stable
  // counting sort by camera of the landmark-sorted order), so that the observations of one
  // camera inside a landmark tile are contiguous
  std::vector<int32_t> ci_order(n);
  {
    std::vector<int32_t> pos(cam_ptr.begin(), cam_ptr.end() - 1);
    for (int64_t q = 0; q < n; ++q) {
      const int32_t o = li_order[q];
      ci_order[pos[ci[o]]++] = o;
    }
  }
  std::vector<int32_t> cpos_of(n);
  for (int64_t q = 0; q < n; ++q) cpos_of[ci_order[q]] = (int32_t)q;
  // camera chunks
  std::vector<int32_t> chunk_cam, chunk_beg, cam_chunk_ptr(M + 1, 0);
  for (int i = 0; i < M; ++i) {
    cam_chunk_ptr[i] = (int32_t)chunk_cam.size();
    for (int b = cam_ptr[i]; b < cam_ptr[i + 1]; b += chunk_obs) {
      chunk_cam.push_back(i);
      chunk_beg.push_back(b);
    }
  }
  cam_chunk_ptr[M] = (int32_t)chunk_cam.size();
  chunk_beg.push_back((int32_t)n);
  // landmark tiles over internal ids: consecutive landmarks with at most TILE_OBS
  // observations and TILE_LMS landmarks, then one tile per long-track landmark
  std::vector<int32_t> tile_lm;
  tile_lm.push_back(0);
  int class_end[2] = {0, 0};
  {
    int j = 0;
    for (int c = 0; c < 2; ++c) {
      while (j < N && lclass(lperm[j]) == c) {
        int j2 = j, cnt = 0;
        while (j2 < N && lclass(lperm[j2]) == c) {
          const int dg = lmi_ptr[j2 + 1] - lmi_ptr[j2];
          if (j2 > j && (c == 1 || j2 - j >= tile_lms || cnt + dg > tile_obs)) break;
          cnt += dg;
          ++j2;
        }
        j = j2;
        tile_lm.push_back(j);
      }
      class_end[c] = (int)tile_lm.size() - 1;
    }
  }
  const int n_tiles = (int)tile_lm.size() - 1;
  if ((int)chunk_cam.size() > ctx->max_chunks || n_tiles > ctx->max_tiles)
    return fail(ctx, DABA_ERR_ARG, "internal schedule bound exceeded");
  // inside each tile the records are kept in camera-sorted order: c_rpos gives each
  // camera-sorted observation its record position, t_inv a landmark-sorted slot's record position
  // relative to the tile start
  std::vector<int32_t> c_rpos(n), c_lm(n);
  std::vector<uint16_t> t_inv(n);
  std::vector<int32_t> t_order(n);
  for (int t = 0; t < n_tiles; ++t) {
    const int ob = lmi_ptr[tile_lm[t]], oe = lmi_ptr[tile_lm[t + 1]];
    for (int o = ob; o < oe; ++o) t_order[o] = o;
    std::sort(t_order.begin() + ob, t_order.begin() + oe,
              [&](int32_t a, int32_t b) { return cpos_of[li_order[a]] < cpos_of[li_order[b]]; });
    for (int o = ob; o < oe; ++o) {
      c_rpos[cpos_of[li_order[t_order[o]]]] = o;
      t_inv[t_order[o]] = (uint16_t)(o - ob);
    }
  }
  for (int64_t q = 0; q < n; ++q) c_lm[q] = lii[ci_order[q]];
  // keep the current iterate (if any) across the renumbering; displacements and the
  // restart metrics are reset (x^(k-1) = x^k, S = 0)
  std::vector<double> keep_l;
  if (ctx->state_set) {
    daba_status s2 = DABA_OK;
    keep_l.resize((size_t)N * 3);
    if ((s2 = daba_get_state(ctx, nullptr, keep_l.data(), stream)) != DABA_OK) return s2;
  }
  // upload
  CK(cudaMemcpyAsync(ctx->c_lm, c_lm.data(), n * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->chunk_cam, chunk_cam.data(), chunk_cam.size() * 4 + 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->chunk_beg, chunk_beg.data(), chunk_beg.size() * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->cam_chunk_ptr, cam_chunk_ptr.data(), (M + 1) * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->lm_ptr, lmi_ptr.data(), (N + 1) * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->tile_lm, tile_lm.data(), tile_lm.size() * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->c_rpos, c_rpos.data(), n * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->t_inv, t_inv.data(), n * 2, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_linv, linv.data(), (size_t)N * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_lperm, lperm.data(), (size_t)N * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_ci_order, ci_order.data(), n * 4, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  ctx->n_chunks = (int)chunk_cam.size();
  ctx->n_tiles = n_tiles;
  for (int c = 0; c < 2; ++c) ctx->tile_class_end[c] = class_end[c];
  ctx->h_cam_idx.swap(ci);
  ctx->h_lm_idx.swap(li);
  ctx->h_uv.swap(uvh);
  ctx->h_c_order.swap(c_order);
  ctx->h_cam_ptr.swap(cam_ptr);
  ctx->h_l_order.swap(l_order);
  ctx->h_lm_ptr.swap(lm_ptr);
  ctx->h_t_order.swap(t_order);
  ctx->h_li_order.swap(li_order);
  ctx->h_ci_order.swap(ci_order);
  ctx->h_lperm.swap(lperm);
  ctx->h_linv.swap(linv);
  ctx->h_tile_lm.swap(tile_lm);
  ctx->h_lmi_ptr.swap(lmi_ptr);
  ctx->h_cam_chunk_ptr.swap(cam_chunk_ptr);
  if ((s = pipe_cut(ctx, st)) != DABA_OK) return s;
  ctx->u_scale_uploaded = -1.0;
  ctx->h_uv_stale = false;
  drop_graphs(ctx);   // the graphs hold the old schedule sizes
  ctx->h_scene_cam.clear();
  ctx->n_scenes = 1;
  ctx->obs_set = true;
  ++ctx->obs_version;
  ctx->n_blocks = 0;   // a partition refers to the previous observations' numbering
  ctx->checked = false;
  if (ctx->state_set) {
    std::vector<double> cams((size_t)M * 9);
    daba_status s2;
    if ((s2 = daba_get_state(ctx, cams.data(), nullptr, stream)) != DABA_OK) return s2;
    const double keep_scale = ctx->s_norm;
    if ((s2 = daba_set_state(ctx, cams.data(), keep_l.data(), stream)) != DABA_OK) return s2;
    ctx->s_norm = keep_scale;
  }
  ctx->k = 0;
  ctx->s_k = 1.0;
  int one = 1;
  CK(cudaMemcpyAsync(ctx->d_first, &one, sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return DABA_OK;
}

daba_status daba_set_state(daba_ctx* ctx, const double* cams, const double* lms, void* stream) {
  if (!ctx) return DABA_ERR_ARG;
  if (!cams || !lms) return fail(ctx, DABA_ERR_ARG, "null state pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const int M = ctx->M, N = ctx->N;
  // device views of the inputs: the caller's device buffers, else one copy into staging
  const bool cdev = is_device_ptr(cams), ldev = is_device_ptr(lms);
  const double* dc = cdev ? cams : (const double*)ctx->st_cam;
  const double* dl = ldev ? lms : (const double*)ctx->st_lm;
  if (!cdev) CK(cudaMemcpyAsync(ctx->st_cam, cams, (size_t)M * 9 * 8, cudaMemcpyHostToDevice, st));
  if (!ldev) CK(cudaMemcpyAsync(ctx->st_lm, lms, (size_t)N * 3 * 8, cudaMemcpyHostToDevice, st));
  // validation before anything of the current state is overwritten
  k_chk_init<<<1, 32, 0, st>>>((int*)ctx->d_chk, (unsigned long long*)ctx->d_bad);
  k_check_state<<<148 * 4, 256, 0, st>>>(M, N, dc, dl, (int*)ctx->d_chk);
  CK(cudaGetLastError());
  int chk[CHK_N];
  CK(cudaMemcpyAsync(chk, ctx->d_chk, sizeof(chk), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (chk[CHK_CAM_NONFINITE] != INT_MAX)
    return fail(ctx, DABA_ERR_NONFINITE, "camera %d has a non-finite parameter", chk[CHK_CAM_NONFINITE]);
  if (chk[CHK_LM_NONFINITE] != INT_MAX)
    return fail(ctx, DABA_ERR_NONFINITE, "landmark %d has a non-finite coordinate", chk[CHK_LM_NONFINITE]);
  if (chk[CHK_FOCAL] != INT_MAX)
    return fail(ctx, DABA_ERR_ARG, "camera %d has a non-positive focal length", chk[CHK_FOCAL]);
  // internal unit s: the option, else the one fixed by the first state, else the median focal
  double sn = ctx->opt.pixel_scale;
  if (!(sn > 0)) {
    if (ctx->s_norm > 0) {
      sn = ctx->s_norm;
    } else {
      std::vector<double> f(M);
      if (cdev) {
        CK(cudaMemcpy2DAsync(f.data(), 8, cams + 6, 9 * 8, 8, M, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
      } else {
        for (int i = 0; i < M; ++i) f[i] = cams[(size_t)i * 9 + 6];
      }
      std::sort(f.begin(), f.end());
      sn = (M % 2) ? f[M / 2] : 0.5 * (f[M / 2 - 1] + f[M / 2]);
    }
  }
  ctx->s_norm = sn;
  k_set_cams<<<(M + 127) / 128, 128, 0, st>>>(M, dc, sn, (double*)ctx->cam_x, (double*)ctx->cam_dx,
                                               (double*)ctx->cam_S, (double*)ctx->cam_E);
  if (is_mixed(ctx))
    k_set_lms<float, true><<<(N + 255) / 256, 256, 0, st>>>(N, dl, (const int*)ctx->d_linv,
                                                            (V4<float>*)ctx->lmrec2[0], (V4<float>*)ctx->lm_lo2[0]);
  else
    k_set_lms<double, false><<<(N + 255) / 256, 256, 0, st>>>(N, dl, (const int*)ctx->d_linv,
                                                              (V4<double>*)ctx->lmrec2[0], nullptr);
  CK(cudaGetLastError());
  int one = 1;
  CK(cudaMemcpyAsync(ctx->d_first, &one, sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  ctx->state_set = true;
  ctx->checked = false;
  ctx->k = 0;
  ctx->s_k = 1.0;
  return DABA_OK;
}

daba_status daba_run(daba_ctx* ctx, int32_t iters, double* obj_trace, int32_t* restarts, void* stream) {
  if (!ctx) return DABA_ERR_ARG;
  if (iters < 0) return fail(ctx, DABA_ERR_ARG, "iters < 0");
  if (!ctx->obs_set || !ctx->state_set) return fail(ctx, DABA_ERR_STATE, "observations and state must be set first");
  cudaStream_t st = (cudaStream_t)stream;
  daba_status s;
  if ((s = check_degenerate(ctx, st)) != DABA_OK) return s;
  if ((s = ensure_u(ctx, st)) != DABA_OK) return s;
  // keep the entry state; a failed run puts it back (a run of one iteration leaves the landmark
  // buffer of x^k untouched, so only longer runs copy the landmarks)
  const int64_t k0 = ctx->k;
  const double s0 = ctx->s_k;
  const bool lm_too = iters > 1;
  CK(backup_copy(ctx, true, k0, lm_too, st));
  const size_t nb = (size_t)ctx->n_blocks;
  if (nb) {   // coarse blocks: their E, Fbar, F and restart flags too
    CK(cudaMemcpyAsync(ctx->blk_bk, ctx->blk_E, nb * 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync((char*)ctx->blk_bk + nb * 8, ctx->blk_Fbar, nb * 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync((char*)ctx->blk_bk + nb * 16, ctx->blk_F, nb * 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync((char*)ctx->blk_bk + nb * 24, ctx->blk_rs, nb, cudaMemcpyDeviceToDevice, st));
  }
  s = run_iterations(ctx, iters, obj_trace, restarts, st);
  if (s != DABA_OK) {
    const std::string why = ctx->err;
    ctx->k = k0;
    ctx->s_k = s0;
    cudaError_t e = backup_copy(ctx, false, k0, lm_too, st);
    if (nb) {
      if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->blk_E, ctx->blk_bk, nb * 8, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->blk_Fbar, (char*)ctx->blk_bk + nb * 8, nb * 8, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->blk_F, (char*)ctx->blk_bk + nb * 16, nb * 8, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->blk_rs, (char*)ctx->blk_bk + nb * 24, nb, cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
      return fail(ctx, s, "%s (restoring the entry state also failed: %s)", why.c_str(), cudaGetErrorString(e));
    ctx->err = why;
  }
  return s;
}

}  // extern "C"

namespace {
daba_status run_iterations(daba_ctx* ctx, int32_t iters, double* obj_trace, int32_t* restarts, cudaStream_t st) {
  daba_status s;
  ctx->launches = 0;
  for (double& t : ctx->tms) t = 0.0;
  std::vector<double> trace((size_t)iters + 1);
  std::vector<int32_t> rs((size_t)std::max(iters, 1));
  int done = 0;
  std::vector<double> gam(GSEG + 1);
  CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), st));
  CK(cudaMemsetAsync(ctx->d_ctr, 0, 16 * PIPE_MAX_RANGES, st));   // bounded-grid counters (range schedule)
  while (done < iters) {
    const int seg = std::min(GSEG, iters - done);
    // gamma^(k) .. gamma^(k+seg) (Eq. nesterov_scalar); the last one is the look-ahead used
    // by the camera solve to extrapolate iteration k+seg
    const double s_start = ctx->s_k;
    double sk = s_start;
    for (int j = 0; j <= seg; ++j) {
      const double s_next = (std::sqrt(4.0 * sk * sk + 1.0) + 1.0) / 2.0;
      gam[j] = (sk - 1.0) / s_next;
      sk = s_next;
      if (j == seg - 1) ctx->s_k = sk;
    }
    CK(cudaMemcpyAsync(ctx->d_gam, gam.data(), (seg + 1) * 8, cudaMemcpyHostToDevice, st));
    // momentum reset: the reduction continues s and the gamma table on the device from s^(k)
    if (ctx->opt.momentum_reset) CK(cudaMemcpyAsync(ctx->s_dev, &s_start, 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(ctx->d_it, 0, sizeof(int), st));
    size_t evi = 0;
    if (ctx->n_blocks > 0) {   // coarse blocks: the prepare kernel, then direct launches per iteration
      CK(launch_prepare(ctx, st, ctx->k));
      for (int j = 0; j < seg; ++j) CK(launch_blk_iter(ctx, st, ctx->k + j));
    } else if (ctx->persistent) {   // the prepare kernel, then every iteration of the segment in one cooperative launch
      CK(launch_prepare(ctx, st, ctx->k));
      CK(launch_persistent(ctx, st, ctx->k, seg));
    } else if (ctx->timing && seg > RUN_GRAPH_MAX) {   // direct launches with per-kernel events
      CK(cudaEventRecord(ev(ctx, evi++), st));
      CK(launch_prepare(ctx, st, ctx->k));
      CK(cudaEventRecord(ev(ctx, evi++), st));
      CK(enqueue_iters(ctx, st, ctx->k, seg, evi));
    } else if (seg <= RUN_GRAPH_MAX) {   // the whole run as one graph launch on s_cap, joined to st
      // (with timing, the graph's own event records time each kernel)
      if ((s = ensure_run_graph(ctx, seg)) != DABA_OK) return s;
      const int par = (int)(ctx->k & 1);
      CK(cudaEventRecord(ctx->ev_cap0, st));
      CK(cudaStreamWaitEvent(ctx->s_cap, ctx->ev_cap0, 0));
      CK(cudaGraphLaunch(ctx->run_graph[par], ctx->s_cap));
      ctx->launches += ctx->run_graph_nl[par];
      CK(cudaEventRecord(ctx->ev_cap1, ctx->s_cap));
      CK(cudaStreamWaitEvent(st, ctx->ev_cap1, 0));
    } else {   // longer runs: the prepare kernel, then 8-iteration graphs on s_cap, joined to st
      CK(launch_prepare(ctx, st, ctx->k));
      if ((s = ensure_graphs(ctx)) != DABA_OK) return s;
      CK(cudaEventRecord(ctx->ev_cap0, st));
      CK(cudaStreamWaitEvent(ctx->s_cap, ctx->ev_cap0, 0));
      for (int j = 0; j < seg;) {
        const int gi = seg - j >= GRAPH_ITERS ? 0 : 1;
        CK(cudaGraphLaunch(ctx->graph[gi][(ctx->k + j) & 1], ctx->s_cap));
        ctx->launches += ctx->graph_nl[gi];
        j += gi == 0 ? GRAPH_ITERS : 1;
      }
      CK(cudaEventRecord(ctx->ev_cap1, ctx->s_cap));
      CK(cudaStreamWaitEvent(st, ctx->ev_cap1, 0));
    }
    CK(cudaMemcpyAsync(trace.data() + done, ctx->d_trace, seg * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(rs.data() + done, ctx->d_rs, seg * 4, cudaMemcpyDeviceToHost, st));
    if (ctx->opt.momentum_reset) CK(cudaMemcpyAsync(&ctx->s_k, ctx->s_dev, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ctx->timing && !ctx->persistent && ctx->n_blocks == 0) {
      float ms = 0.f;
      auto elapsed = [&](size_t a, size_t b) {
        if (cudaEventElapsedTime(&ms, ctx->events[a], ctx->events[b]) == cudaSuccess) return true;
        cudaGetLastError();   // not sticky: the context stays usable
        return false;
      };
      if (!elapsed(0, 1)) return fail(ctx, DABA_ERR_CUDA, "reading the kernel timing events");
      ctx->tms[0] += ms;
      // per iteration: [0] cpass start, [1] cpass end, [2] camsolve end, [3] lpass start,
      // [4] lpass end (side stream), [5] finalize start, [6] finalize end
      for (int j = 0; j < seg; ++j) {
        const size_t b = 2 + (size_t)j * 7;
        const int pairs[4][2] = {{0, 1}, {3, 4}, {1, 2}, {5, 6}};
        for (int q = 0; q < 4; ++q) {
          if (!elapsed(b + pairs[q][0], b + pairs[q][1])) return fail(ctx, DABA_ERR_CUDA, "reading the kernel timing events");
          ctx->tms[1 + q] += ms;
        }
      }
    }
    done += seg;
    ctx->k += seg;
  }
  if (obj_trace) {
    if ((s = enqueue_objective(ctx, st, iters == 0)) != DABA_OK) return s;
    CK(cudaMemcpyAsync(&trace[iters], ctx->d_obj, 8, cudaMemcpyDeviceToHost, st));
  } else {
    trace[iters] = 0.0;
  }
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (flag & 2) return fail(ctx, DABA_ERR_TIMEOUT, "a landmark-pass copy did not complete in time (bounded wait ran out)");
  if (flag & 4) return fail(ctx, DABA_ERR_TIMEOUT, "a grid barrier of the persistent launch ran out");
  if (flag || !std::isfinite(trace[iters])) return fail(ctx, DABA_ERR_NONFINITE, "the objective became non-finite");
  if (obj_trace && (s = deliver(ctx, obj_trace, trace.data(), ((size_t)iters + 1) * 8, st)) != DABA_OK) return s;
  if (restarts && iters > 0 && (s = deliver(ctx, restarts, rs.data(), (size_t)iters * 4, st)) != DABA_OK) return s;
  return DABA_OK;
}
}  // namespace

extern "C" {

daba_status daba_objective(daba_ctx* ctx, double* out, void* stream) {
  if (!ctx || !out) return ctx ? fail(ctx, DABA_ERR_ARG, "null output") : DABA_ERR_ARG;
  if (!ctx->obs_set || !ctx->state_set) return fail(ctx, DABA_ERR_STATE, "observations and state must be set first");
  cudaStream_t st = (cudaStream_t)stream;
  daba_status s;
  if ((s = check_degenerate(ctx, st)) != DABA_OK) return s;
  if ((s = ensure_u(ctx, st)) != DABA_OK) return s;
  // gamma buffer entry 0 is read by the prepare kernel; any finite value will do
  double g0 = 0.0;
  CK(cudaMemcpyAsync(ctx->d_gam, &g0, 8, cudaMemcpyHostToDevice, st));
  if ((s = enqueue_objective(ctx, st, true)) != DABA_OK) return s;
  if (is_device_ptr(out)) {
    CK(cudaMemcpyAsync(out, ctx->d_obj, 8, cudaMemcpyDeviceToDevice, st));
  } else {
    CK(cudaMemcpyAsync(out, ctx->d_obj, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return DABA_OK;
}

daba_status daba_set_scenes(daba_ctx* ctx, int32_t n_scenes, const int32_t* cam_begin) {
  if (!ctx) return DABA_ERR_ARG;
  if (!ctx->obs_set) return fail(ctx, DABA_ERR_STATE, "observations must be set first");
  if (n_scenes < 1 || n_scenes > ctx->M || !cam_begin) return fail(ctx, DABA_ERR_ARG, "n_scenes out of range");
  std::vector<int32_t> cb(cam_begin, cam_begin + n_scenes + 1);
  if (cb[0] != 0 || cb[n_scenes] != ctx->M) return fail(ctx, DABA_ERR_ARG, "cam_begin must run from 0 to M");
  for (int s = 0; s < n_scenes; ++s)
    if (cb[s + 1] < cb[s]) return fail(ctx, DABA_ERR_ARG, "cam_begin must be non-decreasing");
  // every landmark must be observed by the cameras of one scene only
  std::vector<int32_t> scene_of_cam(ctx->M), lm_scene(ctx->N, -1);
  for (int s = 0; s < n_scenes; ++s)
    for (int i = cb[s]; i < cb[s + 1]; ++i) scene_of_cam[i] = s;
  for (int64_t o = 0; o < ctx->nnz; ++o) {
    const int j = ctx->h_lm_idx[o], sc = scene_of_cam[ctx->h_cam_idx[o]];
    if (lm_scene[j] < 0) lm_scene[j] = sc;
    if (lm_scene[j] != sc)
      return fail(ctx, DABA_ERR_ARG, "landmark %d is observed by cameras of scenes %d and %d", j, lm_scene[j], sc);
  }
  // chunk ranges: the chunks of a camera are consecutive, in camera order
  std::vector<int32_t> cc(ctx->M + 1);
  CK(cudaMemcpy(cc.data(), ctx->cam_chunk_ptr, (size_t)(ctx->M + 1) * 4, cudaMemcpyDeviceToHost));
  std::vector<int32_t> sc(n_scenes + 1);
  for (int s = 0; s <= n_scenes; ++s) sc[s] = cc[cb[s]];
  CK(cudaMemcpy(ctx->d_scene_chunk, sc.data(), (size_t)(n_scenes + 1) * 4, cudaMemcpyHostToDevice));
  ctx->h_scene_cam.swap(cb);
  ctx->n_scenes = n_scenes;
  return DABA_OK;
}

daba_status daba_scene_objectives(daba_ctx* ctx, double* out, void* stream) {
  if (!ctx || !out) return ctx ? fail(ctx, DABA_ERR_ARG, "null output") : DABA_ERR_ARG;
  if (!ctx->obs_set || !ctx->state_set) return fail(ctx, DABA_ERR_STATE, "observations and state must be set first");
  if (ctx->h_scene_cam.empty()) return fail(ctx, DABA_ERR_STATE, "no scene partition set");
  cudaStream_t st = (cudaStream_t)stream;
  daba_status s;
  if ((s = check_degenerate(ctx, st)) != DABA_OK) return s;
  if ((s = ensure_u(ctx, st)) != DABA_OK) return s;
  if ((s = enqueue_objective(ctx, st, true)) != DABA_OK) return s;
  const double s2 = ctx->s_norm * ctx->s_norm;
  if (is_mixed(ctx))
    k_segment_sum<float><<<ctx->n_scenes, 256, 0, st>>>((const int*)ctx->d_scene_chunk, (const float*)ctx->chunk_f,
                                                       s2, (double*)ctx->d_scene_f);
  else
    k_segment_sum<double><<<ctx->n_scenes, 256, 0, st>>>((const int*)ctx->d_scene_chunk,
                                                        (const double*)ctx->chunk_f, s2, (double*)ctx->d_scene_f);
  CK(cudaGetLastError());
  const size_t bytes = (size_t)ctx->n_scenes * 8;
  CK(cudaMemcpyAsync(out, ctx->d_scene_f, bytes, is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     st));
  CK(cudaStreamSynchronize(st));
  return DABA_OK;
}

daba_status daba_objective_grad(daba_ctx* ctx, double* F, double* g_cams, double* g_lms, double* g_uv,
                                void* stream) {
  if (!ctx) return DABA_ERR_ARG;
  if (!ctx->obs_set || !ctx->state_set) return fail(ctx, DABA_ERR_STATE, "observations and state must be set first");
  cudaStream_t st = (cudaStream_t)stream;
  daba_status s;
  if ((s = check_degenerate(ctx, st)) != DABA_OK) return s;
  if ((s = ensure_u(ctx, st)) != DABA_OK) return s;
  // the pass pack of x^k (gamma = 0), as for the objective
  CK(cudaMemsetAsync(ctx->d_it, 0, sizeof(int), st));
  CK(cudaMemsetAsync(ctx->d_gam, 0, sizeof(double), st));
  CK(launch_prepare(ctx, st, ctx->k));
  if (is_mixed(ctx))
    CK((launch_grad_by_loss<float, float2, true>(ctx, st)));
  else
    CK((launch_grad_by_loss<double, double2, false>(ctx, st)));
  const int M = ctx->M, N = ctx->N;
  const double sn = ctx->s_norm;
  const bool cdev = g_cams && is_device_ptr(g_cams), ldev = g_lms && is_device_ptr(g_lms);
  double* gc = cdev ? g_cams : (double*)ctx->st_cam;
  double* gl = ldev ? g_lms : (double*)ctx->st_lm;
  if (is_mixed(ctx))
    k_grad_cams<float><<<(M + 127) / 128, 128, 0, st>>>(M, (const int*)ctx->cam_chunk_ptr, (const float*)ctx->chunk_part,
                                                       (const double*)ctx->cam_x, sn, gc, (double*)ctx->cam_Fsum);
  else
    k_grad_cams<double><<<(M + 127) / 128, 128, 0, st>>>(M, (const int*)ctx->cam_chunk_ptr,
                                                        (const double*)ctx->chunk_part, (const double*)ctx->cam_x, sn,
                                                        gc, (double*)ctx->cam_Fsum);
  k_sum<double><<<1, 1024, 0, st>>>(M, (const double*)ctx->cam_Fsum, sn * sn, (double*)ctx->d_obj);
  if (ctx->n_tiles > 0) {
    if (is_mixed(ctx))
      k_grad_lms<float><<<ctx->n_tiles, LPASS_THREADS, 0, st>>>(
          (const int*)ctx->tile_lm, (const int*)ctx->lm_ptr, (const uint16_t*)ctx->t_inv, (const V4<float>*)ctx->rec_a,
          (const int*)ctx->d_lperm, sn * sn, gl);
    else
      k_grad_lms<double><<<ctx->n_tiles, LPASS_THREADS, 0, st>>>(
          (const int*)ctx->tile_lm, (const int*)ctx->lm_ptr, (const uint16_t*)ctx->t_inv,
          (const V4<double>*)ctx->rec_a, (const int*)ctx->d_lperm, sn * sn, gl);
  }
  CK(cudaGetLastError());
  // every landmark is in one tile (those without observations get a zero gradient)
  if (F) CK(cudaMemcpyAsync(F, ctx->d_obj, 8, is_device_ptr(F) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (g_cams && !cdev) CK(cudaMemcpyAsync(g_cams, gc, (size_t)M * 9 * 8, cudaMemcpyDeviceToHost, st));
  if (g_lms && !ldev) CK(cudaMemcpyAsync(g_lms, gl, (size_t)N * 3 * 8, cudaMemcpyDeviceToHost, st));
  if (g_uv)
    CK(cudaMemcpyAsync(g_uv, ctx->rec_b, (size_t)ctx->nnz * 16,
                       is_device_ptr(g_uv) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return DABA_OK;
}

}  // extern "C"

namespace {

// The state of a MIXED context at its iteration ctx->k into a state slot of the FP64 layout of
// `sh` (cameras as they are, landmarks widened: k_lm_widen).
cudaError_t save_mixed_state(daba_ctx* ctx, daba_ctx* sh, void* slot, cudaStream_t st) {
  const SlotLayout L = slot_layout(sh);
  char* b = (char*)slot;
  const size_t cb = (size_t)ctx->M * CSTRIDE * 8;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(b + L.x, ctx->cam_x, cb, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(b + L.dx, ctx->cam_dx, cb, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(b + L.S, ctx->cam_S, (size_t)ctx->M * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(b + L.E, ctx->cam_E, (size_t)ctx->M * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  if (ctx->N > 0)
    k_lm_widen<<<(ctx->N + 255) / 256, 256, 0, st>>>(ctx->N, (const V4<float>*)lmrec_at(ctx, ctx->k),
                                                     (const V4<float>*)lmlo_at(ctx, ctx->k), (V4<double>*)(b + L.lm));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaMemcpyAsync(b + L.first, ctx->d_first, sizeof(int), cudaMemcpyDeviceToDevice, st);
}

// Reverse mode of a MIXED context (daba_unrolled_grad): the vector-Jacobian product of the
// iteration map along the MIXED run's own iterates and decisions, with FP64 adjoint arithmetic.
// The MIXED forward keeps every iterate (widened to the FP64 layout) and its restart decisions;
// then, per iteration from the last, an FP64 context with the same observations and unit (the
// shadow) starts from the MIXED iterate, runs the iteration once to form, in FP64, the
// statistics and landmark sums the adjoint reads, takes the MIXED run's decisions, and runs
// the FP64 adjoint kernels.
daba_status unrolled_grad_mixed(daba_ctx* ctx, int K, const double* seed_cams, const double* seed_lms, double* g_cams,
                                double* g_lms, double* g_uv, cudaStream_t st) {
  const int M = ctx->M, N = ctx->N;
  const size_t nnz = (size_t)ctx->nnz;
  daba_status s;
  if (ctx->h_uv_stale)
    return fail(ctx, DABA_ERR_STATE, "the reverse mode of a MIXED context needs its pixels set from host memory");
  if (ctx->shadow && ctx->shadow->s_norm != ctx->s_norm) {   // a new unit: a new shadow
    daba_destroy(ctx->shadow);
    ctx->shadow = nullptr;
  }
  if (!ctx->shadow || ctx->shadow_version != ctx->obs_version) {
    if (!ctx->shadow) {
      daba_options o = ctx->opt;
      o.prec = DABA_FP64;
      o.pixel_scale = ctx->s_norm;
      daba_ctx* sh = nullptr;
      if ((s = daba_create(M, N, ctx->nnz, &o, &sh)) != DABA_OK)
        return fail(ctx, s, "creating the FP64 context of the reverse mode failed");
      ctx->shadow = sh;
    }
    daba_ctx* sh = ctx->shadow;
    if ((s = daba_set_observations(sh, ctx->h_cam_idx.data(), ctx->h_lm_idx.data(), ctx->h_uv.data(), st)) != DABA_OK)
      return fail(ctx, s, "the reverse mode's FP64 context: %s", sh->err.c_str());
    std::vector<double> cams((size_t)M * 9), lms((size_t)N * 3);
    if ((s = daba_get_state(ctx, cams.data(), lms.data(), st)) != DABA_OK) return s;
    if ((s = daba_set_state(sh, cams.data(), lms.data(), st)) != DABA_OK)
      return fail(ctx, s, "the reverse mode's FP64 context: %s", sh->err.c_str());
    ctx->shadow_version = ctx->obs_version;
  }
  daba_ctx* sh = ctx->shadow;
  if ((s = ensure_u(sh, st)) != DABA_OK) return fail(ctx, s, "the reverse mode's FP64 context: %s", sh->err.c_str());
  if ((s = ensure_adjoint(sh, (size_t)K + 1)) != DABA_OK) return fail(ctx, s, "the reverse mode's FP64 context: out of memory");
  if ((s = dgrow(ctx, &ctx->mx_dec, (size_t)K * (M + N))) != DABA_OK) return s;
  char* dec = (char*)ctx->mx_dec;
  std::vector<double> s_hist((size_t)K + 1);
  CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), st));
  CK(cudaMemsetAsync(sh->d_flag, 0, sizeof(int), st));
  // MIXED forward: every iterate and every iteration's decisions
  for (int k = 0; k < K; ++k) {
    CK(save_mixed_state(ctx, sh, sh->slots[k], st));
    s_hist[k] = ctx->s_k;
    CK(advance(ctx, st, 1));
    CK(cudaMemcpyAsync(dec + (size_t)k * (M + N), ctx->cam_rs, (size_t)M, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(dec + (size_t)k * (M + N) + M, ctx->lm_rs, (size_t)N, cudaMemcpyDeviceToDevice, st));
  }
  s_hist[K] = ctx->s_k;
  CK(save_mixed_state(ctx, sh, sh->slots[K], st));
  // seed: adjoint of x^K (its camera parameterisation read at x^K)
  CK(restore_state(sh, sh->slots[K], K, s_hist[K], st));
  const bool cdev = is_device_ptr(seed_cams), ldev = is_device_ptr(seed_lms);
  const double* dsc = cdev ? seed_cams : (const double*)sh->st_cam;
  const double* dsl = ldev ? seed_lms : (const double*)sh->st_lm;
  if (!cdev) CK(cudaMemcpyAsync(sh->st_cam, seed_cams, (size_t)M * 9 * 8, cudaMemcpyHostToDevice, st));
  if (!ldev) CK(cudaMemcpyAsync(sh->st_lm, seed_lms, (size_t)N * 3 * 8, cudaMemcpyHostToDevice, st));
  int i1 = 0, i0 = 1, im = 2;
  for (int q = 0; q < 3; ++q) {
    CK(cudaMemsetAsync(sh->adj_c[q], 0, (size_t)M * AC_N * 8, st));
    CK(cudaMemsetAsync(sh->adj_l[q], 0, (size_t)N * AL_N * 8, st));
  }
  CK(cudaMemsetAsync(sh->g_u, 0, nnz * 16, st));
  if (M > 0)
    k_adj_seed_cams<<<(M + 127) / 128, 128, 0, st>>>(M, (const double*)sh->cam_x, dsc, sh->s_norm,
                                                     (double*)sh->adj_c[i1]);
  if (N > 0)
    k_adj_seed_lms<<<(N + 255) / 256, 256, 0, st>>>(N, dsl, (const int*)sh->d_linv, (double*)sh->adj_l[i1]);
  CK(cudaGetLastError());
  const ItLayout Li = it_layout(sh);
  void* its = sh->itslots[0];
  for (int k = K - 1; k >= 0; --k) {
    void* slot = sh->slots[k];
    // the iteration once in FP64 from the MIXED iterate: statistics and landmark sums at its points
    CK(restore_state(sh, slot, k, s_hist[k], st));
    sh->lm_sums_out = (char*)its + Li.sums;
    const cudaError_t e = advance(sh, st, 1);
    sh->lm_sums_out = nullptr;
    CK(e);
    CK(save_iteration(sh, its, st));
    CK(cudaMemcpyAsync((char*)its + Li.rs_cam, dec + (size_t)k * (M + N), (size_t)M, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync((char*)its + Li.rs_lm, dec + (size_t)k * (M + N) + M, (size_t)N, cudaMemcpyDeviceToDevice, st));
    // its adjoint at the MIXED iterate with the MIXED decisions
    const double sk = s_hist[k];
    const double gamma = (sk - 1.0) / ((std::sqrt(4.0 * sk * sk + 1.0) + 1.0) / 2.0);
    CK(restore_state(sh, slot, k, sk, st));
    CK(cudaMemcpyAsync(sh->d_gam, &gamma, 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(sh->d_it, 0, sizeof(int), st));
    CK(launch_prepare(sh, st, k));
    CK(adjoint_iter_by_loss(sh, st, k, gamma, slot, its, i1, i0, im));
    if (k > 0) {
      const int t = i1;
      i1 = i0;
      i0 = im;
      im = t;
      CK(cudaMemsetAsync(sh->adj_c[im], 0, (size_t)M * AC_N * 8, st));
      CK(cudaMemsetAsync(sh->adj_l[im], 0, (size_t)N * AL_N * 8, st));
    }
  }
  // adjoint of x^0 = x^(-1) to the boundary
  const SlotLayout Ly = slot_layout(sh);
  const bool gcdev = g_cams && is_device_ptr(g_cams), gldev = g_lms && is_device_ptr(g_lms);
  double* gc = gcdev ? g_cams : (double*)sh->st_cam;
  double* gl = gldev ? g_lms : (double*)sh->st_lm;
  if (M > 0)
    k_adj_out_cams<<<(M + 127) / 128, 128, 0, st>>>(M, (const double*)((const char*)sh->slots[0] + Ly.x),
                                                    (const double*)sh->adj_c[i0], (const double*)sh->adj_c[im],
                                                    sh->s_norm, gc);
  if (N > 0)
    k_adj_out_lms<<<(N + 255) / 256, 256, 0, st>>>(N, (const double*)sh->adj_l[i0], (const double*)sh->adj_l[im],
                                                   (const int*)sh->d_lperm, gl);
  CK(cudaGetLastError());
  if (g_cams && !gcdev) CK(cudaMemcpyAsync(g_cams, gc, (size_t)M * 9 * 8, cudaMemcpyDeviceToHost, st));
  if (g_lms && !gldev) CK(cudaMemcpyAsync(g_lms, gl, (size_t)N * 3 * 8, cudaMemcpyDeviceToHost, st));
  if (g_uv)
    CK(cudaMemcpyAsync(g_uv, sh->g_u, nnz * 16, is_device_ptr(g_uv) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       st));
  int flag = 0, flag_sh = 0;
  CK(cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&flag_sh, sh->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if ((flag | flag_sh) & 2)
    return fail(ctx, DABA_ERR_TIMEOUT, "a landmark-pass copy did not complete in time (bounded wait ran out)");
  if (flag | flag_sh) return fail(ctx, DABA_ERR_NONFINITE, "the objective became non-finite");
  return DABA_OK;   // the MIXED context is left at x^K by its forward run
}

}  // namespace

extern "C" {

daba_status daba_unrolled_grad(daba_ctx* ctx, int32_t K, const double* seed_cams, const double* seed_lms,
                               double* g_cams, double* g_lms, double* g_uv, void* stream) {
  if (!ctx) return DABA_ERR_ARG;
  if (K < 1) return fail(ctx, DABA_ERR_ARG, "K must be >= 1");
  if (!seed_cams || !seed_lms) return fail(ctx, DABA_ERR_ARG, "null seed pointer");
  if (ctx->n_blocks) return fail(ctx, DABA_ERR_ARG, "the unrolled gradient covers one block per camera and landmark");
  if (!ctx->obs_set || !ctx->state_set) return fail(ctx, DABA_ERR_STATE, "observations and state must be set first");
  if (ctx->k != 0) return fail(ctx, DABA_ERR_STATE, "iterations have run since the state was set");
  cudaStream_t st = (cudaStream_t)stream;
  daba_status s;
  if ((s = check_degenerate(ctx, st)) != DABA_OK) return s;
  if ((s = ensure_u(ctx, st)) != DABA_OK) return s;
  if (is_mixed(ctx)) {   // the MIXED trajectory with FP64 adjoint arithmetic (direct launches)
    const bool was = ctx->timing;
    ctx->timing = false;
    s = unrolled_grad_mixed(ctx, K, seed_cams, seed_lms, g_cams, g_lms, g_uv, st);
    ctx->timing = was;
    return s;
  }
  const int C = ADJ_CKPT;
  const int n_seg = (K + C - 1) / C;
  // slots: [0, n_seg) the states at k = 0, C, 2C, ...; [n_seg, n_seg + C) the states of one
  // segment; n_seg + C the state after K iterations
  if ((s = ensure_adjoint(ctx, (size_t)n_seg + C + 1)) != DABA_OK) return s;
  struct TimingOff {   // direct launches without per-kernel events; restored on every return
    daba_ctx* c;
    bool was;
    ~TimingOff() { c->timing = was; }
  } timing_off{ctx, ctx->timing};
  ctx->timing = false;
  const int M = ctx->M, N = ctx->N;
  const size_t nnz = (size_t)ctx->nnz;
  std::vector<double> s_hist((size_t)K + 1);   // s^(k) before iteration k
  CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), st));
  // forward sweep, keeping every C-th state
  for (int sg = 0; sg < n_seg; ++sg) {
    const int n = std::min(C, K - sg * C);
    CK(save_state(ctx, ctx->slots[sg], st));
    for (int j = 0; j < n; ++j) {
      s_hist[(size_t)sg * C + j] = ctx->s_k;
      CK(advance(ctx, st, 1));
    }
  }
  s_hist[K] = ctx->s_k;
  void* fin = ctx->slots[(size_t)n_seg + C];
  CK(save_state(ctx, fin, st));
  // seed: adjoint of x^K
  const bool cdev = is_device_ptr(seed_cams), ldev = is_device_ptr(seed_lms);
  const double* dsc = cdev ? seed_cams : (const double*)ctx->st_cam;
  const double* dsl = ldev ? seed_lms : (const double*)ctx->st_lm;
  if (!cdev) CK(cudaMemcpyAsync(ctx->st_cam, seed_cams, (size_t)M * 9 * 8, cudaMemcpyHostToDevice, st));
  if (!ldev) CK(cudaMemcpyAsync(ctx->st_lm, seed_lms, (size_t)N * 3 * 8, cudaMemcpyHostToDevice, st));
  int i1 = 0, i0 = 1, im = 2;
  for (int q = 0; q < 3; ++q) {
    CK(cudaMemsetAsync(ctx->adj_c[q], 0, (size_t)M * AC_N * 8, st));
    CK(cudaMemsetAsync(ctx->adj_l[q], 0, (size_t)N * AL_N * 8, st));
  }
  CK(cudaMemsetAsync(ctx->g_u, 0, nnz * 16, st));
  if (M > 0)
    k_adj_seed_cams<<<(M + 127) / 128, 128, 0, st>>>(M, (const double*)ctx->cam_x, dsc, ctx->s_norm,
                                                     (double*)ctx->adj_c[i1]);
  if (N > 0)
    k_adj_seed_lms<<<(N + 255) / 256, 256, 0, st>>>(N, dsl, (const int*)ctx->d_linv, (double*)ctx->adj_l[i1]);
  CK(cudaGetLastError());
  // backward over the segments: recompute the segment's states, then per iteration replay it
  // (statistics, records, decisions) and run its adjoint
  const ItLayout Li = it_layout(ctx);
  for (int sg = n_seg - 1; sg >= 0; --sg) {
    const int kb = sg * C, ke = std::min(K, kb + C);
    // the segment's forward sweep keeps each state and what its adjoint reads
    CK(restore_state(ctx, ctx->slots[sg], kb, s_hist[kb], st));
    for (int k = kb; k < ke; ++k) {
      CK(save_state(ctx, ctx->slots[(size_t)n_seg + (k - kb)], st));
      ctx->lm_sums_out = (char*)ctx->itslots[k - kb] + Li.sums;
      const cudaError_t e = advance(ctx, st, 1);
      ctx->lm_sums_out = nullptr;
      CK(e);
      CK(save_iteration(ctx, ctx->itslots[k - kb], st));
    }
    for (int k = ke - 1; k >= kb; --k) {
      const void* slot = ctx->slots[(size_t)n_seg + (k - kb)];
      const double sk = s_hist[k];
      const double gamma = (sk - 1.0) / ((std::sqrt(4.0 * sk * sk + 1.0) + 1.0) / 2.0);
      // x^k in the live buffers (the landmark records of k's parity) and its pass pack
      CK(restore_state(ctx, slot, k, s_hist[k], st));
      CK(cudaMemcpyAsync(ctx->d_gam, &gamma, 8, cudaMemcpyHostToDevice, st));
      CK(cudaMemsetAsync(ctx->d_it, 0, sizeof(int), st));
      CK(launch_prepare(ctx, st, k));
      CK(adjoint_iter_by_loss(ctx, st, k, gamma, slot, ctx->itslots[k - kb], i1, i0, im));
      if (k > 0) {
        const int t = i1;
        i1 = i0;
        i0 = im;
        im = t;
        CK(cudaMemsetAsync(ctx->adj_c[im], 0, (size_t)M * AC_N * 8, st));
        CK(cudaMemsetAsync(ctx->adj_l[im], 0, (size_t)N * AL_N * 8, st));
      }
    }
  }
  // adjoint of x^0 = x^(-1) to the boundary
  const SlotLayout Ly = slot_layout(ctx);
  const bool gcdev = g_cams && is_device_ptr(g_cams), gldev = g_lms && is_device_ptr(g_lms);
  double* gc = gcdev ? g_cams : (double*)ctx->st_cam;
  double* gl = gldev ? g_lms : (double*)ctx->st_lm;
  if (M > 0)
    k_adj_out_cams<<<(M + 127) / 128, 128, 0, st>>>(M, (const double*)((const char*)ctx->slots[0] + Ly.x),
                                                    (const double*)ctx->adj_c[i0], (const double*)ctx->adj_c[im],
                                                    ctx->s_norm, gc);
  if (N > 0)
    k_adj_out_lms<<<(N + 255) / 256, 256, 0, st>>>(N, (const double*)ctx->adj_l[i0], (const double*)ctx->adj_l[im],
                                                   (const int*)ctx->d_lperm, gl);
  CK(cudaGetLastError());
  if (g_cams && !gcdev) CK(cudaMemcpyAsync(g_cams, gc, (size_t)M * 9 * 8, cudaMemcpyDeviceToHost, st));
  if (g_lms && !gldev) CK(cudaMemcpyAsync(g_lms, gl, (size_t)N * 3 * 8, cudaMemcpyDeviceToHost, st));
  if (g_uv)
    CK(cudaMemcpyAsync(g_uv, ctx->g_u, nnz * 16, is_device_ptr(g_uv) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       st));
  // leave the state after K iterations
  CK(restore_state(ctx, fin, K, s_hist[K], st));
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (flag & 2) return fail(ctx, DABA_ERR_TIMEOUT, "a landmark-pass copy did not complete in time (bounded wait ran out)");
  if (flag) return fail(ctx, DABA_ERR_NONFINITE, "the objective became non-finite");
  return DABA_OK;
}

daba_status daba_set_pixels(daba_ctx* ctx, const double* uv, void* stream) {
  if (!ctx) return DABA_ERR_ARG;
  if (!uv) return fail(ctx, DABA_ERR_ARG, "null pixel pointer");
  if (!ctx->obs_set || !ctx->state_set) return fail(ctx, DABA_ERR_STATE, "observations and state must be set first");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = ctx->nnz;
  const bool dev = is_device_ptr(uv);
  if (!dev) std::memcpy(ctx->h_uv.data(), uv, (size_t)n * 16);   // the host copy stays current
  const double* du = uv;
  if (!dev) {   // staged through rec_b (nnz x 16 bytes)
    CK(cudaMemcpyAsync(ctx->rec_b, uv, (size_t)n * 16, cudaMemcpyHostToDevice, st));
    du = (const double*)ctx->rec_b;
  }
  k_chk_init<<<1, 32, 0, st>>>((int*)ctx->d_chk, (unsigned long long*)ctx->d_bad);
  const int blocks = (int)((n + 255) / 256);
  if (is_mixed(ctx))
    k_set_pixels<float2><<<blocks, 256, 0, st>>>(n, (const int*)ctx->d_ci_order, du, ctx->s_norm, (float2*)ctx->c_u,
                                                 (int*)ctx->d_chk);
  else
    k_set_pixels<double2><<<blocks, 256, 0, st>>>(n, (const int*)ctx->d_ci_order, du, ctx->s_norm,
                                                  (double2*)ctx->c_u, (int*)ctx->d_chk);
  CK(cudaGetLastError());
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, ctx->d_chk, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ctx->u_scale_uploaded = ctx->s_norm;
  if (dev) ctx->h_uv_stale = true;
  ++ctx->obs_version;
  if (bad != INT_MAX) return fail(ctx, DABA_ERR_NONFINITE, "observation %d has a non-finite pixel", bad);
  return DABA_OK;
}

daba_status daba_get_state(daba_ctx* ctx, double* cams, double* lms, void* stream) {
  if (!ctx) return DABA_ERR_ARG;
  if (!ctx->state_set) return fail(ctx, DABA_ERR_STATE, "state not set");
  cudaStream_t st = (cudaStream_t)stream;
  const int M = ctx->M, N = ctx->N;
  // converted on the device into the caller's device buffer, else into staging + one copy
  if (cams) {
    const bool dev = is_device_ptr(cams);
    double* out = dev ? cams : (double*)ctx->st_cam;
    k_get_cams<<<(M + 127) / 128, 128, 0, st>>>(M, (const double*)ctx->cam_x, ctx->s_norm, out);
    CK(cudaGetLastError());
    if (!dev) CK(cudaMemcpyAsync(cams, out, (size_t)M * 9 * 8, cudaMemcpyDeviceToHost, st));
  }
  if (lms) {
    const bool dev = is_device_ptr(lms);
    double* out = dev ? lms : (double*)ctx->st_lm;
    if (is_mixed(ctx))
      k_get_lms<float, true><<<(N + 255) / 256, 256, 0, st>>>(N, (const V4<float>*)lmrec_at(ctx, ctx->k),
                                                              (const V4<float>*)lmlo_at(ctx, ctx->k),
                                                              (const int*)ctx->d_linv, out);
    else
      k_get_lms<double, false><<<(N + 255) / 256, 256, 0, st>>>(N, (const V4<double>*)lmrec_at(ctx, ctx->k), nullptr,
                                                                (const int*)ctx->d_linv, out);
    CK(cudaGetLastError());
    if (!dev) CK(cudaMemcpyAsync(lms, out, (size_t)N * 3 * 8, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  return DABA_OK;
}

daba_status daba_get_block_metrics(daba_ctx* ctx, double* F_cam, double* Fbar_cam, double* F_lm, double* Fbar_lm,
                                   uint8_t* rs_cam, uint8_t* rs_lm, void* stream) {
  if (!ctx) return DABA_ERR_ARG;
  if ((F_lm || Fbar_lm) && is_mixed(ctx))
    return fail(ctx, DABA_ERR_STATE, "landmark F and Fbar are reported only by the FP64 path");
  cudaStream_t st = (cudaStream_t)stream;
  const double s2 = ctx->s_norm * ctx->s_norm;
  const int M = ctx->M, N = ctx->N;
  daba_status s;
  // landmark arrays live in the internal order; `lm` maps them back to external ids
  auto getd = [&](double* dst, const void* src, int n, bool lm) -> daba_status {
    std::vector<double> h(n), o(n);
    CK(cudaMemcpyAsync(h.data(), src, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int j = 0; j < n; ++j) o[j] = s2 * h[lm ? lm_internal(ctx, j) : (size_t)j];
    return deliver(ctx, dst, o.data(), (size_t)n * 8, st);
  };
  auto getb = [&](uint8_t* dst, const void* src, int n, bool lm) -> daba_status {
    std::vector<uint8_t> h(n), o(n);
    CK(cudaMemcpyAsync(h.data(), src, (size_t)n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int j = 0; j < n; ++j) o[j] = h[lm ? lm_internal(ctx, j) : (size_t)j];
    return deliver(ctx, dst, o.data(), (size_t)n, st);
  };
  if (F_cam && (s = getd(F_cam, ctx->cam_F, M, false)) != DABA_OK) return s;
  if (Fbar_cam && (s = getd(Fbar_cam, ctx->cam_Fb, M, false)) != DABA_OK) return s;
  if (F_lm && (s = getd(F_lm, ctx->lm_Fd, N, true)) != DABA_OK) return s;
  if (Fbar_lm && (s = getd(Fbar_lm, ctx->lm_Fbd, N, true)) != DABA_OK) return s;
  if (rs_cam && (s = getb(rs_cam, ctx->cam_rs, M, false)) != DABA_OK) return s;
  if (rs_lm && (s = getb(rs_lm, ctx->lm_rs, N, true)) != DABA_OK) return s;
  return DABA_OK;
}

daba_status daba_get_sort(daba_ctx* ctx, int32_t* cam_order, int32_t* cam_ptr, int32_t* lm_order, int32_t* lm_ptr,
                          void* stream) {
  if (!ctx) return DABA_ERR_ARG;
  if (!ctx->obs_set) return fail(ctx, DABA_ERR_STATE, "observations not set");
  cudaStream_t st = (cudaStream_t)stream;
  daba_status s;
  // the stable sorts built by daba_set_observations (the device schedules are derived from them)
  if (cam_order && (s = deliver(ctx, cam_order, ctx->h_c_order.data(), (size_t)ctx->nnz * 4, st)) != DABA_OK) return s;
  if (cam_ptr && (s = deliver(ctx, cam_ptr, ctx->h_cam_ptr.data(), (size_t)(ctx->M + 1) * 4, st)) != DABA_OK) return s;
  if (lm_order && (s = deliver(ctx, lm_order, ctx->h_l_order.data(), (size_t)ctx->nnz * 4, st)) != DABA_OK) return s;
  if (lm_ptr && (s = deliver(ctx, lm_ptr, ctx->h_lm_ptr.data(), (size_t)(ctx->N + 1) * 4, st)) != DABA_OK) return s;
  return DABA_OK;
}

namespace {
struct CkptHeader {
  uint64_t magic;
  int64_t M, N, nnz, prec, k;
  double s_k, s_norm;
  int64_t first;
  int64_t n_blocks;    // coarse blocks: their number and the partition's fingerprint (0, 0 without)
  uint64_t blk_hash;
};
// the block section (coarse blocks): E^alpha, Fbar^alpha, F^alpha and the restart flags per block
size_t ckpt_blk_bytes(const daba_ctx* c) {
  return c->n_blocks ? (size_t)c->n_blocks * 24 + (((size_t)c->n_blocks + 7) & ~(size_t)7) : 0;
}
size_t ckpt_bytes(const daba_ctx* c) {
  return sizeof(CkptHeader) + (size_t)c->M * CSTRIDE * 8 * 2 + (size_t)c->M * 8 * 2 + (size_t)c->N * LREC * real_sz(c) +
         (size_t)c->N * 16 + ckpt_blk_bytes(c);
}
}  // namespace

daba_status daba_export_checkpoint(daba_ctx* ctx, void* buf, size_t* bytes) {
  if (!ctx || !bytes) return DABA_ERR_ARG;
  if (!ctx->state_set) return fail(ctx, DABA_ERR_STATE, "state not set");
  const size_t need = ckpt_bytes(ctx);
  if (!buf) {
    *bytes = need;
    return DABA_OK;
  }
  if (*bytes < need) return fail(ctx, DABA_ERR_ARG, "checkpoint buffer too small (%zu < %zu)", *bytes, need);
  CK(cudaDeviceSynchronize());
  CkptHeader h{CKPT_MAGIC, ctx->M, ctx->N, ctx->nnz, (int64_t)ctx->opt.prec, ctx->k, ctx->s_k, ctx->s_norm, 0,
               ctx->n_blocks, ctx->n_blocks ? ctx->blk_hash : 0};
  int first = 0;
  CK(cudaMemcpy(&first, ctx->d_first, sizeof(int), cudaMemcpyDeviceToHost));
  h.first = first;
  char* p = (char*)buf;
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  const size_t cb = (size_t)ctx->M * CSTRIDE * 8;
  CK(cudaMemcpy(p, ctx->cam_x, cb, cudaMemcpyDeviceToHost));
  p += cb;
  CK(cudaMemcpy(p, ctx->cam_dx, cb, cudaMemcpyDeviceToHost));
  p += cb;
  CK(cudaMemcpy(p, ctx->cam_S, (size_t)ctx->M * 8, cudaMemcpyDeviceToHost));
  p += (size_t)ctx->M * 8;
  CK(cudaMemcpy(p, ctx->cam_E, (size_t)ctx->M * 8, cudaMemcpyDeviceToHost));
  p += (size_t)ctx->M * 8;
  const size_t lb = (size_t)ctx->N * LREC * real_sz(ctx);
  CK(cudaMemcpy(p, lmrec_at(ctx, ctx->k), lb, cudaMemcpyDeviceToHost));
  p += lb;
  CK(cudaMemcpy(p, lmlo_at(ctx, ctx->k), (size_t)ctx->N * 16, cudaMemcpyDeviceToHost));
  p += (size_t)ctx->N * 16;
  if (ctx->n_blocks) {
    const size_t sb = (size_t)ctx->n_blocks * 8;
    CK(cudaMemcpy(p, ctx->blk_E, sb, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(p + sb, ctx->blk_Fbar, sb, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(p + 2 * sb, ctx->blk_F, sb, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(p + 3 * sb, ctx->blk_rs, (size_t)ctx->n_blocks, cudaMemcpyDeviceToHost));
  }
  *bytes = need;
  return DABA_OK;
}

daba_status daba_import_checkpoint(daba_ctx* ctx, const void* buf, size_t bytes) {
  if (!ctx || !buf) return DABA_ERR_ARG;
  if (!ctx->obs_set) return fail(ctx, DABA_ERR_STATE, "observations must be set before importing a checkpoint");
  if (bytes < ckpt_bytes(ctx)) return fail(ctx, DABA_ERR_ARG, "checkpoint too small");
  CkptHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != CKPT_MAGIC || h.M != ctx->M || h.N != ctx->N || h.nnz != ctx->nnz || h.prec != (int64_t)ctx->opt.prec)
    return fail(ctx, DABA_ERR_ARG, "checkpoint does not match this context");
  if (h.n_blocks != ctx->n_blocks || h.blk_hash != (ctx->n_blocks ? ctx->blk_hash : 0))
    return fail(ctx, DABA_ERR_ARG, "checkpoint was taken with another partition into blocks");
  const char* p = (const char*)buf + sizeof(h);
  const size_t cb = (size_t)ctx->M * CSTRIDE * 8;
  CK(cudaMemcpy(ctx->cam_x, p, cb, cudaMemcpyHostToDevice));
  p += cb;
  CK(cudaMemcpy(ctx->cam_dx, p, cb, cudaMemcpyHostToDevice));
  p += cb;
  CK(cudaMemcpy(ctx->cam_S, p, (size_t)ctx->M * 8, cudaMemcpyHostToDevice));
  p += (size_t)ctx->M * 8;
  CK(cudaMemcpy(ctx->cam_E, p, (size_t)ctx->M * 8, cudaMemcpyHostToDevice));
  p += (size_t)ctx->M * 8;
  const size_t lb = (size_t)ctx->N * LREC * real_sz(ctx);
  CK(cudaMemcpy(lmrec_at(ctx, h.k), p, lb, cudaMemcpyHostToDevice));
  p += lb;
  CK(cudaMemcpy(lmlo_at(ctx, h.k), p, (size_t)ctx->N * 16, cudaMemcpyHostToDevice));
  p += (size_t)ctx->N * 16;
  if (ctx->n_blocks) {
    const size_t sb = (size_t)ctx->n_blocks * 8;
    CK(cudaMemcpy(ctx->blk_E, p, sb, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->blk_Fbar, p + sb, sb, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->blk_F, p + 2 * sb, sb, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->blk_rs, p + 3 * sb, (size_t)ctx->n_blocks, cudaMemcpyHostToDevice));
  }
  int first = (int)h.first;
  CK(cudaMemcpy(ctx->d_first, &first, sizeof(int), cudaMemcpyHostToDevice));
  ctx->k = h.k;
  ctx->s_k = h.s_k;
  ctx->s_norm = h.s_norm;
  ctx->state_set = true;
  // host copies used by the Assumption 2 check: rebuild from the imported iterate
  ctx->checked = true;
  return DABA_OK;
}

daba_status daba_set_partition(daba_ctx* ctx, int32_t n_blocks, const int32_t* cam_block, const int32_t* lm_block) {
  if (!ctx) return DABA_ERR_ARG;
  if (!ctx->obs_set) return fail(ctx, DABA_ERR_STATE, "observations must be set first");
  if (n_blocks == 0) {   // back to one block per camera and per landmark
    ctx->n_blocks = 0;
    return DABA_OK;
  }
  if (is_mixed(ctx)) return fail(ctx, DABA_ERR_ARG, "coarse blocks run on FP64 contexts");
  const int M = ctx->M, N = ctx->N;
  if (n_blocks < 0 || (int64_t)n_blocks > (int64_t)M + N || !cam_block || !lm_block)
    return fail(ctx, DABA_ERR_ARG, "n_blocks must lie in 1 .. M + N, with both block arrays given");
  const int S = n_blocks;
  std::vector<int32_t> cb(M), lb(N);
  daba_status s;
  if ((s = fetch(ctx, cb.data(), cam_block, (size_t)M * 4, nullptr)) != DABA_OK) return s;
  if ((s = fetch(ctx, lb.data(), lm_block, (size_t)N * 4, nullptr)) != DABA_OK) return s;
  // cameras per block (ascending), their position in that list and their local index
  std::vector<int32_t> cam_ptr(S + 1, 0), cams(M), cpos(M), cloc(M);
  for (int i = 0; i < M; ++i) {
    if (cb[i] < 0 || cb[i] >= S) return fail(ctx, DABA_ERR_ARG, "cam_block[%d] out of range", i);
    cam_ptr[cb[i] + 1]++;
  }
  int most = 0;
  for (int b = 0; b < S; ++b) {
    if (cam_ptr[b + 1] > BLK_MAX_CAMS)
      return fail(ctx, DABA_ERR_ARG, "block %d holds %d cameras (at most %d)", b, cam_ptr[b + 1], BLK_MAX_CAMS);
    most = std::max(most, cam_ptr[b + 1]);
    cam_ptr[b + 1] += cam_ptr[b];
  }
  {
    std::vector<int32_t> pos(cam_ptr.begin(), cam_ptr.end() - 1);
    for (int i = 0; i < M; ++i) {
      cloc[i] = pos[cb[i]] - cam_ptr[cb[i]];
      cpos[i] = pos[cb[i]];
      cams[pos[cb[i]]++] = i;
    }
  }
  // landmarks per block (internal ids, ascending) and the position of each in that list
  std::vector<int32_t> lm_ptr(S + 1, 0), lms(N), lpos(N);
  for (int j = 0; j < N; ++j) {
    if (lb[j] < 0 || lb[j] >= S) return fail(ctx, DABA_ERR_ARG, "lm_block[%d] out of range", j);
  }
  for (int ji = 0; ji < N; ++ji) lm_ptr[lb[ctx->h_lperm[ji]] + 1]++;
  for (int b = 0; b < S; ++b) lm_ptr[b + 1] += lm_ptr[b];
  {
    std::vector<int32_t> pos(lm_ptr.begin(), lm_ptr.end() - 1);
    for (int ji = 0; ji < N; ++ji) {
      const int b = lb[ctx->h_lperm[ji]];
      lpos[ji] = pos[b];
      lms[pos[b]++] = ji;
    }
  }
  // the intra pairs (E'), camera-sorted: per landmark entry by camera, per camera entry by observation
  const int64_t n = ctx->nnz;
  std::vector<uint8_t> intra(n, 0);
  std::vector<int32_t> io_ptr(N + 1, 0), ci_ptr(M + 1, 0);
  int64_t n_in = 0;
  for (int64_t o = 0; o < n; ++o) {
    const int32_t in = ctx->h_ci_order[o];   // input index of the camera-sorted observation o
    const int i = ctx->h_cam_idx[in], j = ctx->h_lm_idx[in];
    if (cb[i] != lb[j]) continue;
    intra[o] = 1;
    io_ptr[lpos[lm_internal(ctx, j)] + 1]++;
    ci_ptr[cpos[i] + 1]++;
    n_in++;
  }
  for (int e = 0; e < N; ++e) io_ptr[e + 1] += io_ptr[e];
  for (int e = 0; e < M; ++e) ci_ptr[e + 1] += ci_ptr[e];
  std::vector<int32_t> io_cam(n_in), io_obs(n_in), ci_obs(n_in), ci_lm(n_in), ci_e(n_in), ci_io(n_in);
  {
    std::vector<int32_t> ip(io_ptr.begin(), io_ptr.end() - 1), cp(ci_ptr.begin(), ci_ptr.end() - 1);
    for (int64_t o = 0; o < n; ++o) {
      if (!intra[o]) continue;
      const int32_t in = ctx->h_ci_order[o];
      const int i = ctx->h_cam_idx[in], j = ctx->h_lm_idx[in];
      const int ji = (int)lm_internal(ctx, j), e = lpos[ji];
      // observations run by camera, so a landmark's pairs arrive by ascending camera
      if (ip[e] > io_ptr[e] && io_cam[ip[e] - 1] == cloc[i])
        return fail(ctx, DABA_ERR_ARG, "camera %d observes landmark %d twice inside a block", i, j);
      ci_e[cp[cpos[i]]] = e;
      ci_io[cp[cpos[i]]] = ip[e];
      io_cam[ip[e]] = cloc[i];
      io_obs[ip[e]++] = (int32_t)o;
      ci_lm[cp[cpos[i]]] = ji;
      ci_obs[cp[cpos[i]]++] = (int32_t)o;
    }
  }
  // the block scratch: in shared memory when every block has at most BLK_SMEM_CAMS cameras (per
  // camera scratch, two vectors and the Schur matrix of the largest block), else in global memory
  // (per camera entry, and each block's Schur matrix of stride 9 x its cameras)
  // automatic: one CTA per block with shared scratch when the blocks are small and one CTA per
  // block already gives every SM at least half a CTA; otherwise clusters over the global scratch
  const int pref = ctx->blk_pref;
  const bool in_smem = most <= BLK_SMEM_CAMS && (pref == 1 || (pref == 0 && (int64_t)S * 4 > 2LL * ctx->n_sm));
  const int ld = 9 * most;
  const size_t smem = in_smem ? (size_t)most * sizeof(BlkCam) + (size_t)(3 * ld + ld * ld) * 8 : 0;
  std::vector<long long> soff(S + 1, 0);
  for (int b = 0; b < S; ++b) {
    const long long nb = 9LL * (cam_ptr[b + 1] - cam_ptr[b]);
    soff[b + 1] = soff[b] + (in_smem ? 0 : nb * nb);
  }
  CK(cudaFuncSetAttribute(k_blk_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // global scratch: a cluster of CTAs per block, the largest of 16, 8, 4, 2 that the device can
  // place and that keeps the grid within two CTAs per SM (else one CTA per block)
  int csz = 1;
  if (!in_smem && pref != 1) {
    CK(cudaFuncSetAttribute(k_blk_solve, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    for (int c : {16, 8, 4, 2}) {
      if (pref > 1 ? c > pref : (int64_t)S * c > 2LL * ctx->n_sm) continue;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(S * c));
      cfg.blockDim = dim3(BLK_THREADS);
      cfg.dynamicSmemBytes = 0;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)c;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n_cl = 0;
      if (cudaOccupancyMaxActiveClusters(&n_cl, k_blk_solve, &cfg) == cudaSuccess && n_cl > 0) {
        csz = c;
        break;
      }
      cudaGetLastError();   // not sticky
    }
  }
  const size_t ni = (size_t)n_in;
  if (!in_smem) {
    if ((s = dgrow(ctx, &ctx->blk_gcam, (size_t)M * sizeof(BlkCam))) != DABA_OK) return s;
    if ((s = dgrow(ctx, &ctx->blk_gvec, (size_t)M * 27 * 8)) != DABA_OK) return s;
    if ((s = dgrow(ctx, &ctx->blk_gS, (size_t)std::max(soff[S], 1LL) * 8)) != DABA_OK) return s;
  }
  if ((s = dgrow(ctx, &ctx->blk_soff, (size_t)(S + 1) * 8)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_ci_e, std::max(ni, (size_t)1) * 4)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_ci_io, std::max(ni, (size_t)1) * 4)) != DABA_OK) return s;
  CK(cudaMemcpy(ctx->blk_soff, soff.data(), (size_t)(S + 1) * 8, cudaMemcpyHostToDevice));
  if ((s = dgrow(ctx, &ctx->c_intra, (size_t)n)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_cam_ptr, (size_t)(S + 1) * 4)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_cams, (size_t)M * 4)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_lm_ptr, (size_t)(S + 1) * 4)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_lms, (size_t)N * 4)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_io_ptr, (size_t)(N + 1) * 4)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_io_cam, ni * 4)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_io_obs, ni * 4)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_ci_ptr, (size_t)(M + 1) * 4)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_ci_obs, ni * 4)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_ci_lm, ni * 4)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_sums, (size_t)N * LS_N * 8)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_lsc, (size_t)N * BL_N * 8)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_isc, ni * BI_N * 8)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_E, (size_t)S * 8)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_Fbar, (size_t)S * 8)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_F, (size_t)S * 8)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_rs, (size_t)S)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_g, (size_t)S * 8)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_Ealt, (size_t)S * 8)) != DABA_OK) return s;
  if ((s = dgrow(ctx, &ctx->blk_bk, (size_t)S * 32)) != DABA_OK) return s;
  CK(cudaMemcpy(ctx->c_intra, intra.data(), (size_t)n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->blk_cam_ptr, cam_ptr.data(), (size_t)(S + 1) * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->blk_cams, cams.data(), (size_t)M * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->blk_lm_ptr, lm_ptr.data(), (size_t)(S + 1) * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->blk_lms, lms.data(), (size_t)N * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->blk_io_ptr, io_ptr.data(), (size_t)(N + 1) * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->blk_ci_ptr, ci_ptr.data(), (size_t)(M + 1) * 4, cudaMemcpyHostToDevice));
  if (ni) {
    CK(cudaMemcpy(ctx->blk_io_cam, io_cam.data(), ni * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->blk_io_obs, io_obs.data(), ni * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->blk_ci_obs, ci_obs.data(), ni * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->blk_ci_lm, ci_lm.data(), ni * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->blk_ci_e, ci_e.data(), ni * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->blk_ci_io, ci_io.data(), ni * 4, cudaMemcpyHostToDevice));
  }
  CK(cudaMemset(ctx->blk_rs, 0, (size_t)S));
  ctx->n_blocks = S;
  ctx->blk_ld = in_smem ? ld : 0;
  ctx->blk_smem = smem;
  ctx->blk_cs = csz;
  ctx->blk_ncam = 0;
  for (int b = 0; b < S; ++b) ctx->blk_ncam += cam_ptr[b + 1] > cam_ptr[b] ? 1 : 0;
  {   // the partition's fingerprint (FNV-1a over n_blocks and both block arrays)
    uint64_t hsh = 1469598103934665603ull;
    auto mix = [&](const void* d, size_t n) {
      const unsigned char* q = (const unsigned char*)d;
      for (size_t i = 0; i < n; ++i) hsh = (hsh ^ q[i]) * 1099511628211ull;
    };
    mix(&S, sizeof(S));
    mix(cb.data(), (size_t)M * 4);
    mix(lb.data(), (size_t)N * 4);
    ctx->blk_hash = hsh;
  }
  drop_graphs(ctx);
  return DABA_OK;
}

daba_status daba_set_block_ctas(daba_ctx* ctx, int32_t ctas) {
  if (!ctx) return DABA_ERR_ARG;
  if (ctas < 0 || ctas > 16) return fail(ctx, DABA_ERR_ARG, "ctas must lie in 0 .. 16");
  ctx->blk_pref = ctas;
  return DABA_OK;
}

daba_status daba_get_partition_metrics(daba_ctx* ctx, double* F_blk, double* Fbar_blk, uint8_t* rs_blk, void* stream) {
  if (!ctx) return DABA_ERR_ARG;
  if (ctx->n_blocks == 0) return fail(ctx, DABA_ERR_STATE, "no partition set");
  cudaStream_t st = (cudaStream_t)stream;
  const int S = ctx->n_blocks;
  const double s2 = ctx->s_norm * ctx->s_norm;
  std::vector<double> h(S);
  daba_status s;
  for (int q = 0; q < 2; ++q) {
    double* dst = q == 0 ? F_blk : Fbar_blk;
    if (!dst) continue;
    CK(cudaMemcpyAsync(h.data(), q == 0 ? ctx->blk_F : ctx->blk_Fbar, (size_t)S * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (double& v : h) v *= s2;
    if ((s = deliver(ctx, dst, h.data(), (size_t)S * 8, st)) != DABA_OK) return s;
  }
  if (rs_blk) {
    std::vector<uint8_t> r(S);
    CK(cudaMemcpyAsync(r.data(), ctx->blk_rs, (size_t)S, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if ((s = deliver(ctx, rs_blk, r.data(), (size_t)S, st)) != DABA_OK) return s;
  }
  return DABA_OK;
}

daba_status daba_set_pipeline(daba_ctx* ctx, const daba_pipeline* p) {
  if (!ctx) return DABA_ERR_ARG;
  if (!p) return fail(ctx, DABA_ERR_ARG, "null schedule");
  if (p->ranges < 1 || p->ranges > PIPE_MAX_RANGES) return fail(ctx, DABA_ERR_ARG, "ranges must lie in [1, 64]");
  if (p->cpass_warps < 0 || p->cpass_warps > 64 || p->lpass_ctas < 0 || p->lpass_ctas > 64)
    return fail(ctx, DABA_ERR_ARG, "grid bounds must lie in [0, 64]");
  for (int r = 0; r < 3; ++r)
    if (p->prio[r] < 0 || p->prio[r] > 2) return fail(ctx, DABA_ERR_ARG, "priority ranks must lie in [0, 2]");
  return pipe_apply(ctx, *p);
}

}  // extern "C"

namespace {
// Sets the range schedule (arguments checked by the caller): the stream pools at the roles'
// priorities (only for more than one range) and the ranges for the current observations.
daba_status pipe_apply(daba_ctx* ctx, const daba_pipeline& p) {
  pipe_streams_free(ctx);
  drop_graphs(ctx);
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  for (int role = 0; role < 3 && p.ranges > 1; ++role) {   // one range needs no pools
    const int prio = std::min(least, greatest + p.prio[role]);   // greater numbers are lower priorities
    for (cudaStream_t& q : ctx->s_pool[role])
      if (cudaStreamCreateWithPriority(&q, cudaStreamNonBlocking, prio) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        pipe_streams_free(ctx);
        ctx->pipe = daba_pipeline{};
        ctx->pipe_R = 1;
        return fail(ctx, DABA_ERR_CUDA, "creating the schedule's streams: %s", cudaGetErrorString(e));
      }
  }
  ctx->pipe = p;
  return pipe_cut(ctx, nullptr);
}
}  // namespace

extern "C" {

daba_status daba_set_persistent(daba_ctx* ctx, int enable) {
  if (!ctx) return DABA_ERR_ARG;
  if (enable && (!is_mixed(ctx) || ctx->opt.restart_mode != DABA_RESTART_BLOCK || ctx->opt.cam_solver != DABA_CAM_SCAM))
    return fail(ctx, DABA_ERR_ARG, "the persistent path runs MIXED contexts with per-block restart and S-CAM");
  ctx->persistent = enable != 0;
  return DABA_OK;
}

daba_status daba_set_wait_limit(daba_ctx* ctx, int64_t first_wait_ns) {
  if (!ctx) return DABA_ERR_ARG;
  if (first_wait_ns < 0) return fail(ctx, DABA_ERR_ARG, "first_wait_ns < 0");
  if (first_wait_ns != ctx->wait_ns) {
    ctx->wait_ns = first_wait_ns;
    drop_graphs(ctx);   // the captured launches hold the old limit
  }
  return DABA_OK;
}

daba_status daba_set_timing(daba_ctx* ctx, int enable) {
  if (!ctx) return DABA_ERR_ARG;
  ctx->timing = enable != 0;
  return DABA_OK;
}

daba_status daba_get_timing(daba_ctx* ctx, double* ms5) {
  if (!ctx || !ms5) return DABA_ERR_ARG;
  for (int q = 0; q < 5; ++q) ms5[q] = ctx->tms[q];
  return DABA_OK;
}

}  // extern "C"
