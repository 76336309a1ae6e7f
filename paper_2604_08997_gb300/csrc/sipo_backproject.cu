// Instantiations of the backprojector P_mu^T for every storage type and
// epilogue used by the library.
#include "sipo_launch.h"
#include "sipo_ops.cuh"

#include <type_traits>

namespace sipo {

// Tile table: 0 = 8 columns per warp, 2 blocks/SM; 1 = 4 columns, 2 blocks/SM;
// 2 = 4 columns, 3 blocks/SM (tighter register budget); 3 and 4 = the
// row-pattern kernel (4 columns, packed FP32 multiply-adds) at 2 and 3
// blocks/SM.  The row-pattern kernel is single precision: FP64 solves map
// entries 3 and 4 to entry 2.
template <typename SI, typename S, typename C, int ZL, int MODE, typename O>
static void launch_bp_zl(const Geo<C>& g, const SI* sino, const Bufs<S, C>& b, O* out, const uint8_t* need,
                         cudaStream_t stream, int tile) {
  if constexpr (std::is_same<C, float>::value) {
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
