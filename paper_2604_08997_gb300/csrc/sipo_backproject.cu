// Instantiations of the backprojector P_mu^T for every storage type and
// epilogue used by the library.
#include "sipo_launch.h"
#include "sipo_ops.cuh"

namespace sipo {

template <typename SI, typename S, typename C, int MODE, typename O>
void launch_backproject(const Geo<C>& g, const SI* sino, const Bufs<S, C>& b, O* out,
                        const uint8_t* need, bool vec, cudaStream_t stream, int nv) {
  constexpr int ZLV = sizeof(SI) == 8 ? 4 : 8;
  if (vec) {
    if (nv == 4)
      k_backproject<SI, S, C, ZLV, 4, MODE, O><<<kRedBlocks, kThreads, 0, stream>>>(g, sino, b, out, need);
    else
      k_backproject<SI, S, C, ZLV, 8, MODE, O><<<kRedBlocks, kThreads, 0, stream>>>(g, sino, b, out, need);
  } else {
    if (nv == 4)
      k_backproject<SI, S, C, 1, 4, MODE, O><<<kRedBlocks, kThreads, 0, stream>>>(g, sino, b, out, need);
    else
      k_backproject<SI, S, C, 1, 8, MODE, O><<<kRedBlocks, kThreads, 0, stream>>>(g, sino, b, out, need);
  }
}

#define SIPO_BP(SI, S, C, M, O) \
  template void launch_backproject<SI, S, C, M, O>(const Geo<C>&, const SI*, const Bufs<S, C>&, \
                                                    O*, const uint8_t*, bool, cudaStream_t, int);
#define SIPO_BP_SOLVER(S, C)       \
  SIPO_BP(S, S, C, kBpDual, C)     \
  SIPO_BP(S, S, C, kBpDualCheck, C) \
  SIPO_BP(S, S, C, kBpStore, C)

SIPO_BP_SOLVER(float, float)
SIPO_BP_SOLVER(__nv_bfloat16, float)
SIPO_BP_SOLVER(double, double)

}  // namespace sipo
