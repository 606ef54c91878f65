// daba_noalloc.cu -- objective evaluation that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that hands the whole device to its own
// memory pool (frameworks that pre-reserve HBM and forbid raw allocations), real-time
// loops that must not risk an allocation failing or stalling mid-run, or plugins that
// may only touch the buffers they are given. daba_objective_noalloc serves them: it is
// the objective pass of the library with its scratch (internal camera parameters and
// per-block partial sums) in one file-scope __device__ array instead of a context's
// allocations. The caller passes device inputs and a device output only.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/daba.h"
#include "daba_device.cuh"

namespace {

constexpr int NA_MAX_CAMS = 16384;     // cameras the scratch can hold
constexpr int NA_CAM_STRIDE = 18;      // R[9] t[3] pad[3] d[3] (d at the pack offset PK_D)
constexpr int NA_BLOCKS = 148 * 8;     // observation-pass blocks (multiple of the SM count)
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_DEVICES = 64;

// One scratch per GPU that loads the library, kept until the process exits:
// [0, NA_MAX_CAMS * NA_CAM_STRIDE)   internal camera parameters
// [.., + NA_BLOCKS)                  per-block partial sums of F_ij
// [.., + 1)                          invalid-input flag (stored as a double)
constexpr size_t NA_PARTS = (size_t)NA_MAX_CAMS * NA_CAM_STRIDE;
constexpr size_t NA_FLAG = NA_PARTS + NA_BLOCKS;
static __device__ __align__(256) double g_noalloc_scratch[NA_FLAG + 1];

std::mutex g_mu;
double* g_scratch_addr[NA_MAX_DEVICES] = {nullptr};

// Device address of the scratch on the current device (looked up once per device).
daba_status scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    cudaGetLastError();
    return DABA_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return DABA_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return DABA_OK;
}

// true for managed memory and for device memory of GPU `dev` (memory of another GPU is
// rejected: the kernels would reach it without peer access)
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

// boundary camera (axis-angle, centre, f, k1, k2) -> internal (R, t, d) in units of s pixels
__global__ void k_na_cams(int M, const double* __restrict__ cams, double s, double* __restrict__ scratch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) scratch[NA_FLAG] = 0.0;   // clear the invalid-input flag of this call
  if (i >= M) return;
  const double* c = cams + (size_t)i * 9;
  double* o = scratch + (size_t)i * NA_CAM_STRIDE;
  daba::rodrigues(c, o + daba::PK_R);
  const double f = c[6];
  o[daba::PK_TH + 0] = c[3];
  o[daba::PK_TH + 1] = c[4];
  o[daba::PK_TH + 2] = c[5];
  o[daba::PK_D + 0] = f / s;
  o[daba::PK_D + 1] = c[7] * s / f;
  o[daba::PK_D + 2] = c[8] * s * s * s / (f * f * f);
}

// F_ij over a fixed grid of NA_BLOCKS blocks; each block writes its own partial sum
template <int LOSS>
__global__ void __launch_bounds__(NA_THREADS)
    k_na_obs(int M, int N, long long nnz, const int32_t* __restrict__ cam_idx, const int32_t* __restrict__ lm_idx,
             const double* __restrict__ uv, const double* __restrict__ lms, double inv_s, daba::LossC<double> L,
             double* __restrict__ scratch) {
  double f = 0.0;
  bool bad = false;
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < nnz; o += (long long)gridDim.x * blockDim.x) {
    const int i = cam_idx[o], j = lm_idx[o];
    if (i < 0 || i >= M || j < 0 || j >= N) {
      bad = true;
      continue;
    }
    const double* pk = scratch + (size_t)i * NA_CAM_STRIDE;
    const double q0 = lms[(size_t)j * 3 + 0] - pk[daba::PK_TH + 0];
    const double q1 = lms[(size_t)j * 3 + 1] - pk[daba::PK_TH + 1];
    const double q2 = lms[(size_t)j * 3 + 2] - pk[daba::PK_TH + 2];
    f += daba::eval_F<LOSS, double>(pk, q0, q1, q2, uv[2 * o] * inv_s, uv[2 * o + 1] * inv_s, L);
  }
  __shared__ double red[NA_THREADS / 32];
  __shared__ int redb;
  if (threadIdx.x == 0) redb = 0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
  __syncthreads();
  if (bad) redb = 1;
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) t += red[w];
    scratch[NA_PARTS + blockIdx.x] = t;
    if (redb) scratch[NA_FLAG] = 1.0;
  }
}

__global__ void k_na_sum(const double* __restrict__ scratch, double s2, double* __restrict__ out) {
  __shared__ double red[32];
  double f = 0.0;
  for (int b = threadIdx.x; b < NA_BLOCKS; b += blockDim.x) f += scratch[NA_PARTS + b];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = scratch[NA_FLAG] != 0.0 ? nan("") : t * s2;
  }
}

template <int LOSS>
cudaError_t launch_na(int M, int N, long long nnz, const double* cams, const double* lms, const int32_t* ci,
                      const int32_t* li, const double* uv, double c, double s, double* scratch, double* out,
                      cudaStream_t st) {
  daba::LossC<double> L;
  L.c = c;
  L.c2 = c * c;
  L.inv_c2 = 1.0 / (c * c);
  k_na_cams<<<(M + 127) / 128, 128, 0, st>>>(M, cams, s, scratch);
  k_na_obs<LOSS><<<NA_BLOCKS, NA_THREADS, 0, st>>>(M, N, nnz, ci, li, uv, lms, 1.0 / s, L, scratch);
  k_na_sum<<<1, 1024, 0, st>>>(scratch, s * s, out);
  return cudaGetLastError();
}

}  // namespace

extern "C" daba_status daba_objective_noalloc(int32_t M, int32_t N, int64_t nnz, const double* cams,
                                              const double* lms, const int32_t* cam_idx, const int32_t* lm_idx,
                                              const double* uv, int32_t loss, double loss_scale_px,
                                              double pixel_scale, double* out, void* stream) {
  if (M < 1 || N < 1 || nnz < 1 || M > NA_MAX_CAMS || nnz >= (int64_t(1) << 40)) return DABA_ERR_ARG;
  if (loss < 0 || loss > 3 || !(pixel_scale > 0) || (loss != DABA_LOSS_TRIVIAL && !(loss_scale_px > 0)))
    return DABA_ERR_ARG;
  if (!cams || !lms || !cam_idx || !lm_idx || !uv || !out) return DABA_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return DABA_ERR_CUDA;
  }
  if (!on_device(cams, dev) || !on_device(lms, dev) || !on_device(cam_idx, dev) || !on_device(lm_idx, dev) ||
      !on_device(uv, dev) || !on_device(out, dev))
    return DABA_ERR_ARG;
  double* scratch = nullptr;
  daba_status s = scratch_for_current_device(&scratch);
  if (s != DABA_OK) return s;
  const double c = loss == DABA_LOSS_TRIVIAL ? 1.0 : loss_scale_px / pixel_scale;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (loss) {
    case DABA_LOSS_TRIVIAL:
      e = launch_na<daba::LOSS_TRIVIAL>(M, N, nnz, cams, lms, cam_idx, lm_idx, uv, c, pixel_scale, scratch, out, st);
      break;
    case DABA_LOSS_HUBER:
      e = launch_na<daba::LOSS_HUBER>(M, N, nnz, cams, lms, cam_idx, lm_idx, uv, c, pixel_scale, scratch, out, st);
      break;
    case DABA_LOSS_CAUCHY:
      e = launch_na<daba::LOSS_CAUCHY>(M, N, nnz, cams, lms, cam_idx, lm_idx, uv, c, pixel_scale, scratch, out, st);
      break;
    default:
      e = launch_na<daba::LOSS_WELSCH>(M, N, nnz, cams, lms, cam_idx, lm_idx, uv, c, pixel_scale, scratch, out, st);
      break;
  }
  return e == cudaSuccess ? DABA_OK : DABA_ERR_CUDA;
}
