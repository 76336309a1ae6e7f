// sipo_noalloc.cu -- dose-field metrics for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: a print controller that must
// not allocate once its real-time loop is running, or host code embedded in a
// framework whose caching allocator owns the whole device-memory budget (a
// foreign cudaMalloc there can fail or fragment the pool).  For them this
// file provides sipo_dose_metrics_noalloc: the same reductions as the metrics
// pass at the end of sipo_solve, with its per-block partial sums kept in a
// file-scope static device array instead of context-owned scratch.
//
// The array is part of the library image: every GPU that loads the library
// holds it (8 x 8192 + 8 doubles, 512 KiB) until the process exits.  Its address is
// looked up once per device with cudaGetSymbolAddress by the first call made
// with that device current; make that first call before any stream capture.
// The address is kept for the life of the process, keyed by device ordinal:
// it stays valid while the device's primary context lives, so the entry
// point must not be called again after a cudaDeviceReset of that device.
// All calls share the array and overwrite it completely, so nothing needs
// clearing, but calls that overlap on the GPU (concurrent streams, several
// host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "sipo.h"
#include "sipo_device.cuh"

namespace sipo {
void set_last_error(const std::string& msg);  // message returned by sipo_last_error()

namespace {

constexpr int kNaSlots = 8;                        // reductions per block
constexpr int kNaItems = 64;                       // voxels per thread (upper bound)
constexpr int kNaMaxBlocks = 8192;                 // partial rows the array holds
constexpr long long kNaMaxVoxels = (long long)kNaMaxBlocks * kThreads * kNaItems;  // 2^27

// partials [slot][block] followed by the kNaSlots final values
static __device__ __align__(256) double g_noalloc_scratch[kNaSlots * kNaMaxBlocks + kNaSlots];
static_assert(sizeof(double) * (kNaSlots * kNaMaxBlocks + kNaSlots) <= 600 * 1024,
              "the static scratch must stay modest");

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
double* g_na_addr[kMaxDevices] = {};


// Per block: 0 min_gel d/f~T, 1 max_gel d/f~T, 2 max_band d, 3 min_gel d,
// 4 sum_gel d f_T, 5 sum_gel d^2, 6 min_gel d/f~_L, 7 max_gel d/f~_L
// (the same quantities as the metrics pass of sipo_solve).
template <typename C>
__global__ void __launch_bounds__(kThreads)
k_metrics_noalloc(const C* __restrict__ d, const uint8_t* __restrict__ lab, const float* __restrict__ fT,
                  double f_crit, double lower_scale, long long n, double* __restrict__ part) {
  double v[kNaSlots] = {1e300, -1e300, -1e300, 1e300, 0.0, 0.0, 1e300, -1e300};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint8_t l = lab[i];
    if (l == kBand) {
      v[2] = fmax(v[2], double(d[i]));
    } else if (l == kGel) {
      const double dv = double(d[i]);
      const double r = dv / (double(fT[i]) / f_crit);
      v[0] = fmin(v[0], r);
      v[1] = fmax(v[1], r);
      v[3] = fmin(v[3], dv);
      v[4] += dv * double(fT[i]);
      v[5] += dv * dv;
      const double lo = dv / (double(fT[i]) * lower_scale);
      v[6] = fmin(v[6], lo);
      v[7] = fmax(v[7], lo);
    }
  }
  __shared__ double sh[kThreads];
  for (int q = 0; q < kNaSlots; ++q) {
    sh[threadIdx.x] = v[q];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) {
        const double a = sh[threadIdx.x], b = sh[threadIdx.x + st];
        sh[threadIdx.x] = (q == 0 || q == 3 || q == 6) ? fmin(a, b) : (q == 4 || q == 5) ? a + b : fmax(a, b);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)q * kNaMaxBlocks + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

// One block folds the partial rows of `nblocks` blocks into the final values.
__global__ void __launch_bounds__(kThreads) k_metrics_noalloc_finish(double* part, int nblocks) {
  __shared__ double sh[kThreads];
  for (int q = 0; q < kNaSlots; ++q) {
    const bool is_min = (q == 0 || q == 3 || q == 6), is_sum = (q == 4 || q == 5);
    double acc = is_min ? 1e300 : (is_sum ? 0.0 : -1e300);
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      const double x = part[(size_t)q * kNaMaxBlocks + b];
      acc = is_min ? fmin(acc, x) : (is_sum ? acc + x : fmax(acc, x));
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) {
        const double a = sh[threadIdx.x], b = sh[threadIdx.x + st];
        sh[threadIdx.x] = is_min ? fmin(a, b) : (is_sum ? a + b : fmax(a, b));
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)kNaSlots * kNaMaxBlocks + q] = sh[0];
    __syncthreads();
  }
}

int na_fail(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

// Device address of the static scratch for the current device (looked up on
// the first call per device).
int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return na_fail(SIPO_ERR_CUDA, "sipo_dose_metrics_noalloc: no current CUDA device");
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return na_fail(SIPO_ERR_CUDA, std::string("sipo_dose_metrics_noalloc: cudaGetSymbolAddress failed: ") +
                                        cudaGetErrorString(e));
    g_na_addr[dev] = static_cast<double*>(p);
  }
  *out = g_na_addr[dev];
  return SIPO_OK;
}

}  // namespace
}  // namespace sipo

extern "C" {

int sipo_dose_metrics_noalloc(const void* dose, int dtype, const uint8_t* labels, const float* f_T,
                              long long n_voxels, double f_crit, double lower_scale, double* metrics,
                              void* stream) {
  using namespace sipo;
  set_last_error("");
  if (!dose || !labels || !f_T || !metrics)
    return na_fail(SIPO_ERR_INVALID_ARG, "sipo_dose_metrics_noalloc: null argument");
  if (dtype != SIPO_F32 && dtype != SIPO_F64)
    return na_fail(SIPO_ERR_INVALID_ARG, "sipo_dose_metrics_noalloc: dtype must be SIPO_F32 or SIPO_F64");
  if (n_voxels <= 0)
    return na_fail(SIPO_ERR_INVALID_ARG, "sipo_dose_metrics_noalloc: n_voxels must be positive");
  if (n_voxels > kNaMaxVoxels)
    return na_fail(SIPO_ERR_INVALID_ARG,
                   "sipo_dose_metrics_noalloc: n_voxels exceeds the static scratch limit of 134217728 "
                   "voxels (8192 blocks x 256 threads x 64 voxels)");
  if (!(f_crit > 0) || !(lower_scale > 0))
    return na_fail(SIPO_ERR_INVALID_ARG, "sipo_dose_metrics_noalloc: f_crit and lower_scale must be > 0");
  double* part = nullptr;
  const int rc = scratch_address(&part);
  if (rc != SIPO_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long per_block = (long long)kThreads * kNaItems;
  const int nblocks = int((n_voxels + per_block - 1) / per_block);
  if (dtype == SIPO_F32)
    k_metrics_noalloc<float><<<nblocks, kThreads, 0, s>>>(static_cast<const float*>(dose), labels, f_T,
                                                          f_crit, lower_scale, n_voxels, part);
  else
    k_metrics_noalloc<double><<<nblocks, kThreads, 0, s>>>(static_cast<const double*>(dose), labels, f_T,
                                                           f_crit, lower_scale, n_voxels, part);
  k_metrics_noalloc_finish<<<1, kThreads, 0, s>>>(part, nblocks);
  double h[kNaSlots];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, part + (size_t)kNaSlots * kNaMaxBlocks, sizeof(h),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return na_fail(SIPO_ERR_CUDA, std::string("sipo_dose_metrics_noalloc: ") + cudaGetErrorString(e));
  const double mn_r = h[0], mx_r = h[1], mx_b = h[2], mn_d = h[3];
  const bool has_band = mx_b > -1e299;
  metrics[0] = mn_r > 0 ? mx_r / mn_r : INFINITY;                 // max / min gel ratio d / f~_T
  metrics[1] = (mn_r > 0 && has_band) ? mx_b / mn_r : INFINITY;   // band maximum over the minimum ratio
  metrics[2] = (has_band && mx_b > 0) ? mn_d / mx_b : INFINITY;   // gel minimum over band maximum
  metrics[3] = h[5] > 0 ? h[4] / h[5] : 0.0;                      // least-squares scale onto f_T
  metrics[4] = h[6];                                              // min_gel d / (lower_scale f_T)
  return SIPO_OK;
}

}  // extern "C"
