// Instantiations of the projector P_mu (gather form) for every storage type
// and epilogue used by the library.
#include "sipo_launch.h"
#include "sipo_ops.cuh"

#include <algorithm>

namespace sipo {

// Bits recorded by this translation unit's kernels in a checked build (0 in
// plain builds); cleared by the read.
unsigned int check_flags_project() {
#ifdef SIPO_CHECKED
  unsigned int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_sipo_check, sizeof(v)) != cudaSuccess) return 0;
  cudaMemcpyToSymbol(g_sipo_check, &zero, sizeof(zero));
  return v;
#else
  return 0;
#endif
}


// bits[line][word] from flags need[y][x]; by_rows selects line = y (bits over
// x) or line = x (bits over y).
__global__ void k_need_bits(const uint8_t* __restrict__ need, uint32_t* __restrict__ bits, int nx, int ny,
                            int words, int by_rows) {
  const int lines = by_rows ? ny : nx, len = by_rows ? nx : ny;
  const long long n = (long long)lines * words;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int line = int(i / words), w = int(i % words);
    uint32_t v = 0;
    for (int bt = 0; bt < 32; ++bt) {
      const int pos = w * 32 + bt - kNbPad;
      if (pos >= 0 && pos < len) {
        const int x = by_rows ? pos : line, y = by_rows ? line : pos;
        if (need[(size_t)y * nx + x]) v |= 1u << bt;
      }
    }
    bits[i] = v;
  }
}


template <typename SI, typename S, typename C, int MODE, typename O>
void launch_project(const Geo<C>& g, const SI* vol, const Bufs<S, C>& b, O* out,
                    const uint8_t* act_col, int zl, cudaStream_t stream, const NeedBits& nb,
                    const int2* rspan) {
  constexpr int G = z_group<C>();
  // the slice-mode certificate keeps one 8-byte maximum per z in shared memory
  const size_t dyn = MODE == kFpCertZ ? size_t(g.nz) * sizeof(unsigned long long) : 0;
  if (zl == 2 * G)
    k_project<SI, S, C, 2 * G, MODE, O><<<kRedBlocks, kThreads, dyn, stream>>>(g, vol, b, out, act_col, nb, rspan);
  else if (zl == G)
    k_project<SI, S, C, G, MODE, O><<<kRedBlocks, kThreads, dyn, stream>>>(g, vol, b, out, act_col, nb, rspan);
  else
    k_project<SI, S, C, 1, MODE, O><<<kRedBlocks, kThreads, dyn, stream>>>(g, vol, b, out, act_col, nb, rspan);
}

void launch_need_bits(const uint8_t* need, uint32_t* rows, uint32_t* cols, int nx, int ny, int wr, int wc,
                      cudaStream_t stream) {
  const int gr = int(std::min<long long>(((long long)ny * wr + kThreads - 1) / kThreads, (long long)device_sms() * 16));
  const int gc = int(std::min<long long>(((long long)nx * wc + kThreads - 1) / kThreads, (long long)device_sms() * 16));
  k_need_bits<<<gr, kThreads, 0, stream>>>(need, rows, nx, ny, wr, 1);
  k_need_bits<<<gc, kThreads, 0, stream>>>(need, cols, nx, ny, wc, 0);
}

template <typename C>
void launch_ray_spans(const Geo<C>& g, const uint8_t* need, int2* out, cudaStream_t stream) {
  const long long n = (long long)g.na * g.nd;
  const int grid = int(std::min<long long>((n + kThreads - 1) / kThreads, (long long)device_sms() * 16));
  k_ray_spans<C><<<grid, kThreads, 0, stream>>>(g, need, out);
}
template void launch_ray_spans<float>(const Geo<float>&, const uint8_t*, int2*, cudaStream_t);
template void launch_ray_spans<double>(const Geo<double>&, const uint8_t*, int2*, cudaStream_t);

#define SIPO_FP(SI, S, C, M, O) \
  template void launch_project<SI, S, C, M, O>(const Geo<C>&, const SI*, const Bufs<S, C>&, O*, \
                                                const uint8_t*, int, cudaStream_t, const NeedBits&, \
                                                const int2*);
#define SIPO_FP_SOLVER(S, C)          \
  SIPO_FP(S, S, C, kFpPrimal, C)      \
  SIPO_FP(S, S, C, kFpPrimalCheck, C) \
  SIPO_FP(S, S, C, kFpResid, C)

SIPO_FP_SOLVER(float, float)
SIPO_FP_SOLVER(__nv_bfloat16, float)
SIPO_FP_SOLVER(double, double)
// bound-based certificate: the candidate volume is in the compute type
SIPO_FP(float, float, float, kFpCert, float)
SIPO_FP(float, __nv_bfloat16, float, kFpCert, float)
SIPO_FP(double, double, double, kFpCert, double)
SIPO_FP(float, float, float, kFpCertZ, float)
SIPO_FP(float, __nv_bfloat16, float, kFpCertZ, float)
SIPO_FP(double, double, double, kFpCertZ, double)
SIPO_FP(float, float, float, kFpStore, float)
SIPO_FP(double, double, double, kFpStore, double)
SIPO_FP(__nv_bfloat16, __nv_bfloat16, float, kFpStore, float)

}  // namespace sipo
