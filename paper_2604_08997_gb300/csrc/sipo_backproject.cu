// Instantiations of the backprojector P_mu^T for every storage type and
// epilogue used by the library.
#include <cudaTypedefs.h>

#include <mutex>

#include "sipo_bp_tma.cuh"
#include "sipo_launch.h"
#include "sipo_ops.cuh"

#include <type_traits>

namespace sipo {

// Bits recorded by this translation unit's kernels in a checked build (0 in
// plain builds); cleared by the read.
unsigned int check_flags_backproject() {
#ifdef SIPO_CHECKED
  unsigned int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_sipo_check, sizeof(v)) != cudaSuccess) return 0;
  cudaMemcpyToSymbol(g_sipo_check, &zero, sizeof(zero));
  return v;
#else
  return 0;
#endif
}


unsigned int bp3_fault_take() {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_bp3_fault, sizeof(v)) != cudaSuccess) return 0;
  if (v) {
    const unsigned int zero = 0;
    cudaMemcpyToSymbol(g_bp3_fault, &zero, sizeof(zero));
  }
  return v;
}

int wait_selftest(long long budget, int arrive, int threads, unsigned int* timed_out) {
  unsigned int* d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned int)) != cudaSuccess) return -1;
  cudaError_t e = cudaMemset(d, 0, sizeof(unsigned int));
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, threads>>>(budget, arrive, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(timed_out, d, sizeof(unsigned int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? 0 : -1;
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 3-D tensor map of a sinogram [na][nd][nz] with boxes of 256 z x kBp3Rows
// bins x 1 angle; bins off the detector read as zeros.  False when the map
// cannot be made (no driver entry point, unaligned buffer).
template <typename SI>
bool sino_map(const SI* sino, int nz, int nd, int na, CUtensorMap* map) {
  const auto fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(sino) & 15u) != 0) return false;
  const cuuint64_t dims[3] = {cuuint64_t(nz), cuuint64_t(nd), cuuint64_t(na)};
  const cuuint64_t strides[2] = {cuuint64_t(nz) * sizeof(SI), cuuint64_t(nz) * nd * sizeof(SI)};
  const cuuint32_t box[3] = {cuuint32_t(kBp3ZC), cuuint32_t(kBp3Rows), 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUtensorMapDataType dt = sizeof(SI) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  return fn(map, dt, 3, const_cast<SI*>(sino), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename SI, typename S, int MINB, int MODE, typename O>
bool launch_bp3(const Geo<float>& g, const SI* sino, const Bufs<S, float>& b, O* out, const uint8_t* need,
                cudaStream_t stream) {
  CUtensorMap map;
  if (!sino_map<SI>(sino, g.nz, g.nd, g.na, &map)) return false;
  constexpr size_t bytes = Bp3Smem<SI>::kBytes;
  // more than the 48 KB default of dynamic shared memory (per device, cheap)
  if (cudaFuncSetAttribute(k_backproject3<SI, S, MINB, MODE, O>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(bytes)) != cudaSuccess)
    return false;
  k_backproject3<SI, S, MINB, MODE, O><<<kRedBlocks, kThreads, bytes, stream>>>(g, sino, map, b, out, need);
  return true;
}

}  // namespace

// Tile table: 0 = 8 columns per warp, 2 blocks/SM; 1 = 4 columns, 2 blocks/SM;
// 2 = 4 columns, 3 blocks/SM (tighter register budget); 3 and 4 = the
// row-pattern kernel (4 columns, packed FP32 multiply-adds) at 2 and 3
// blocks/SM; 5 and 6 = the row-pattern kernel fed by tensor-memory copies of
// the rows into shared memory (k_backproject3) at 3 and 2 blocks/SM, for
// 256 z values per warp (nz a multiple of 256).  The row-pattern kernels are
// single precision: FP64 solves map entries 3-6 to entry 2; other z extents
// map 5 and 6 to 4.
template <typename SI, typename S, typename C, int ZL, int MODE, typename O>
static void launch_bp_zl(const Geo<C>& g, const SI* sino, const Bufs<S, C>& b, O* out, const uint8_t* need,
                         cudaStream_t stream, int tile) {
  if constexpr (std::is_same<C, float>::value) {
    if constexpr (ZL == 8) {
      if (tile == 5 || tile == 6) {
        const bool ok = tile == 5 ? launch_bp3<SI, S, 3, MODE, O>(g, sino, b, out, need, stream)
                                  : launch_bp3<SI, S, 2, MODE, O>(g, sino, b, out, need, stream);
        if (ok) return;
        tile = 4;  // no tensor map: the row-pattern kernel with global loads
      }
    }
    if (tile >= 5) tile = 4;
    if (tile == 3) {
      k_backproject2<SI, S, ZL, 2, MODE, O><<<kRedBlocks, kThreads, 0, stream>>>(g, sino, b, out, need);
      return;
    }
    if (tile == 4) {
      k_backproject2<SI, S, ZL, 3, MODE, O><<<kRedBlocks, kThreads, 0, stream>>>(g, sino, b, out, need);
      return;
    }
  }
  if (tile == 1)
    k_backproject<SI, S, C, ZL, 4, 2, MODE, O><<<kRedBlocks, kThreads, 0, stream>>>(g, sino, b, out, need);
  else if (tile >= 2)
    k_backproject<SI, S, C, ZL, 4, 3, MODE, O><<<kRedBlocks, kThreads, 0, stream>>>(g, sino, b, out, need);
  else
    k_backproject<SI, S, C, ZL, 8, 2, MODE, O><<<kRedBlocks, kThreads, 0, stream>>>(g, sino, b, out, need);
}

template <typename SI, typename S, typename C, int MODE, typename O>
void launch_backproject(const Geo<C>& g, const SI* sino, const Bufs<S, C>& b, O* out,
                        const uint8_t* need, int zl, cudaStream_t stream, int tile) {
  constexpr int G = z_group<C>();
  if (zl == 2 * G)
    launch_bp_zl<SI, S, C, 2 * G, MODE, O>(g, sino, b, out, need, stream, tile);
  else if (zl == G)
    launch_bp_zl<SI, S, C, G, MODE, O>(g, sino, b, out, need, stream, tile);
  else
    launch_bp_zl<SI, S, C, 1, MODE, O>(g, sino, b, out, need, stream, tile);
}

#define SIPO_BP(SI, S, C, M, O) \
  template void launch_backproject<SI, S, C, M, O>(const Geo<C>&, const SI*, const Bufs<S, C>&, \
                                                    O*, const uint8_t*, int, cudaStream_t, int);
#define SIPO_BP_SOLVER(S, C)       \
  SIPO_BP(S, S, C, kBpDual, C)     \
  SIPO_BP(S, S, C, kBpStore, C)

SIPO_BP_SOLVER(float, float)
SIPO_BP_SOLVER(__nv_bfloat16, float)
SIPO_BP_SOLVER(double, double)

}  // namespace sipo
