// Instantiations of the projector P_mu (gather form) for every storage type
// and epilogue used by the library.
#include "sipo_launch.h"
#include "sipo_ops.cuh"

namespace sipo {

template <typename SI, typename S, typename C, int MODE, typename O>
void launch_project(const Geo<C>& g, const SI* vol, const Bufs<S, C>& b, O* out,
                    const uint8_t* act_col, bool vec, cudaStream_t stream) {
  constexpr int ZLV = sizeof(SI) == 8 ? 4 : 8;
  if (vec)
    k_project<SI, S, C, ZLV, MODE, O><<<kRedBlocks, kThreads, 0, stream>>>(g, vol, b, out, act_col);
  else
    k_project<SI, S, C, 1, MODE, O><<<kRedBlocks, kThreads, 0, stream>>>(g, vol, b, out, act_col);
}

#define SIPO_FP(SI, S, C, M, O) \
  template void launch_project<SI, S, C, M, O>(const Geo<C>&, const SI*, const Bufs<S, C>&, O*, \
                                                const uint8_t*, bool, cudaStream_t);
#define SIPO_FP_SOLVER(S, C)          \
  SIPO_FP(S, S, C, kFpPrimal, C)      \
  SIPO_FP(S, S, C, kFpPrimalCheck, C) \
  SIPO_FP(S, S, C, kFpResid, C)

SIPO_FP_SOLVER(float, float)
SIPO_FP_SOLVER(__nv_bfloat16, float)
SIPO_FP_SOLVER(double, double)
SIPO_FP(float, float, float, kFpStore, float)
SIPO_FP(double, double, double, kFpStore, double)
SIPO_FP(__nv_bfloat16, __nv_bfloat16, float, kFpStore, float)

}  // namespace sipo
