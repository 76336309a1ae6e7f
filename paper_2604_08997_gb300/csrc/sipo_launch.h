// sipo_launch.h -- host launchers of the operator kernels (one translation
// unit per operator so that the builds compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include "sipo_solver.cuh"

namespace sipo {

// vec selects the 16-byte vector z-path (needs nz % ZL == 0, ZL = 8 for
// 4/2-byte elements and 4 for doubles) over the scalar path (ZL = 1).
template <typename SI, typename S, typename C, int MODE, typename O>
void launch_project(const Geo<C>& g, const SI* vol, const Bufs<S, C>& b, O* out,
                    const uint8_t* act_col, bool vec, cudaStream_t stream);

// nv: voxel columns per warp (4 or 8; the tile table of sipo_tile_count).
template <typename SI, typename S, typename C, int MODE, typename O>
void launch_backproject(const Geo<C>& g, const SI* sino, const Bufs<S, C>& b, O* out,
                        const uint8_t* need, bool vec, cudaStream_t stream, int nv = 8);

template <typename C> constexpr int vec_zl() { return sizeof(C) == 8 ? 4 : 8; }

}  // namespace sipo
