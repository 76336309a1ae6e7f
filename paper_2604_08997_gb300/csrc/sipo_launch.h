// sipo_launch.h -- host launchers of the operator kernels (one translation
// unit per operator so that the builds compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include "sipo_solver.cuh"
#include "sipo_ops.cuh"

namespace sipo {

// zl: z values per lane (z_lanes<C>(nz) picks it): 2G or G, G = 16 bytes of
// compute elements, for the vector paths, 1 for the scalar path.
// nb: packed per-column flags of voxels whose input may be non-zero (rows ==
// nullptr: every in-vial voxel); rspan: per-ray walked-axis span holding such
// columns (nullptr: whole ray).
template <typename SI, typename S, typename C, int MODE, typename O>
void launch_project(const Geo<C>& g, const SI* vol, const Bufs<S, C>& b, O* out,
                    const uint8_t* act_col, int zl, cudaStream_t stream,
                    const NeedBits& nb = NeedBits{}, const int2* rspan = nullptr);

// Packs need[y][x] into the row-major and column-major bit arrays of NeedBits.
void launch_need_bits(const uint8_t* need, uint32_t* rows, uint32_t* cols, int nx, int ny, int wr, int wc,
                      cudaStream_t stream);

// Per-ray span of the projector walk that meets flagged columns (k_ray_spans).
template <typename C>
void launch_ray_spans(const Geo<C>& g, const uint8_t* need, int2* out, cudaStream_t stream);

// tile: entry of the backprojector tile table (0: 8 columns per warp, 2
// blocks/SM; 1: 4 columns, 2 blocks/SM; 2: 4 columns, 3 blocks/SM; 3, 4: the
// single-precision row-pattern kernel at 2 and 3 blocks/SM, entry 2 in FP64;
// 5, 6: the row-pattern kernel with rows staged by tensor-memory copies, at 3
// and 2 blocks/SM, for nz a multiple of 256, else entry 4).
constexpr int kBpTiles = 7;

// Reads and clears the fault flag of the staged backprojector (nonzero: a
// bounded wait on a tensor-memory copy gave up; the launch's sums are not
// valid).  Synchronous: call outside stream capture.
unsigned int bp3_fault_take();

// Runs the bounded mbarrier wait of the staged backprojector on its own: one
// block of `threads` threads waits `budget` cycles on a barrier that receives
// its one arrival only if `arrive`; *timed_out = threads whose wait gave up.
// 0 on success, -1 on a CUDA error.  Synchronous.
int wait_selftest(long long budget, int arrive, int threads, unsigned int* timed_out);

// Checked builds (-DSIPO_CHECKED): the check bits recorded by the kernels of
// each translation unit, read and cleared; 0 in plain builds.
unsigned int check_flags_project();
unsigned int check_flags_backproject();
template <typename SI, typename S, typename C, int MODE, typename O>
void launch_backproject(const Geo<C>& g, const SI* sino, const Bufs<S, C>& b, O* out,
                        const uint8_t* need, int zl, cudaStream_t stream, int tile = 0);

// Group size G of the z layout (elements of C in 16 bytes).
template <typename C> constexpr int z_group() { return 16 / int(sizeof(C)); }

// z values per lane for a z extent nz: two groups when a warp's 64 G values
// tile nz exactly, one group when nz is a multiple of G (the last warp of a
// column may then be partly idle, lane by lane), else the scalar path.
template <typename C> inline int z_lanes(int nz) {
  constexpr int G = z_group<C>();
  return nz % (64 * G) == 0 ? 2 * G : (nz % G == 0 ? G : 1);
}

}  // namespace sipo
