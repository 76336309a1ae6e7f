// sipo_bp_tma.cuh -- backprojector with the sinogram rows staged in shared
// memory by the Tensor Memory Accelerator (sm_103a).
//
// Same tiles, table, row patterns, packed multiply-adds and epilogues as
// k_backproject2 (8 warps = 8 voxel rows of 4 columns, 256 z values per warp),
// and the same sums bit for bit.  What changes is where the rows come from.
// For each angle the block needs the detector rows that its 32 voxel columns
// reach: with u = x cos + y sin over a 4 x 8 tile, floor(u) spans at most
// ceil(3 |cos| + 7 |sin|) + 1 <= 9 bins, so a box of kBp3Rows = 10 rows
// starting at the block's smallest floor(u) holds every tap (a tile whose span
// is larger, which rounding cannot produce, is reported as a fault).  One
// elected thread copies that box ([256 z] x [10 bins] of one angle) from the
// sinogram into shared memory with one cp.async.bulk.tensor per angle; bins
// off the detector are filled with zeros by the copy itself.  Copies run
// kBp3Stages stages of kBp3Angles angles ahead of the warps, each stage
// completing on its own mbarrier, so the warps read their rows from shared
// memory (tens of cycles) instead of waiting on L2 for every angle.
//
// Waits are bounded: a wait that outlives kBp3WaitCycles clock cycles sets a fault
// flag (read by bp3_fault_take on the host), stops the block and leaves its
// sums unwritten; an angle whose rows do not fit the box sets another bit.
#pragma once

#include <cuda.h>

#include "sipo_ops.cuh"

namespace sipo {

constexpr int kBp3Rows = 10;     // bins per staged box
constexpr int kBp3Angles = 2;    // angles per pipeline stage
constexpr int kBp3Stages = 2;    // stages in flight
constexpr int kBp3ZC = 256;      // z values per warp (ZL = 8 floats per lane)
constexpr long long kBp3WaitCycles = 4000000000LL;  // ~2 s at 2 GHz: a wait that long has failed

// Fault flag of the staged backprojector (bit 0: an mbarrier wait timed out).
// Defined here: one translation unit (sipo_backproject.cu) includes this file.
__device__ unsigned int g_bp3_fault = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false once `budget` SM
// clock cycles have passed without it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget = kBp3WaitCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > budget) return false;
  return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Self-test of the bounded wait: one mbarrier expecting one arrival, which
// thread 0 makes only when `arrive` is set; every thread waits on the first
// phase with a budget of `budget` cycles.  out[0] = number of threads whose wait
// gave up (blockDim.x when nothing arrives, 0 otherwise).
__global__ void k_wait_selftest(long long budget, int arrive, unsigned int* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && arrive) mbar_arrive(&bar);
  if (!mbar_wait(&bar, 0u, budget)) atomicAdd(out, 1u);
}

// One box of the 3-D tensor map (z, bin, angle) into shared memory,
// completing on `bar` (its byte count is announced by mbar_expect_tx).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int z, int bin, int angle,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(z), "r"(bin), "r"(angle),
      "r"(smem_u32(bar))
      : "memory");
}

// ZL values of one staged row (lane layout of load_z, from shared memory).
template <typename SI, int ZL>
__device__ __forceinline__ void lds_row(const SI* p, float (&v)[ZL]) {
  using L = ZLayout<float, ZL>;
#pragma unroll
  for (int q = 0; q < L::NG; ++q) {
    const SI* pq = p + q * L::kStride;
    if constexpr (sizeof(SI) == 4) {
      const float4 r = *reinterpret_cast<const float4*>(pq);
      v[q * 4] = r.x; v[q * 4 + 1] = r.y; v[q * 4 + 2] = r.z; v[q * 4 + 3] = r.w;
    } else {
      const uint2 r = *reinterpret_cast<const uint2*>(pq);
      v[q * 4] = __uint_as_float(r.x << 16);
      v[q * 4 + 1] = __uint_as_float(r.x & 0xffff0000u);
      v[q * 4 + 2] = __uint_as_float(r.y << 16);
      v[q * 4 + 3] = __uint_as_float(r.y & 0xffff0000u);
    }
  }
}

// One angle of the warp's four voxels from the staged rows: rows[r] is bin
// (table b + r) of the angle, r < kBp3Rows - (b - block start).
template <typename SI, int ZL, int PAT>
__device__ __forceinline__ void bp3_body(const SI* rows, const Bp2Ent& e, float (&acc)[kBp2NV][ZL]) {
  constexpr int NR = bp2_rows(PAT);
  float r[NR][ZL];
#pragma unroll
  for (int j = 0; j < NR; ++j) lds_row<SI, ZL>(rows + j * kBp3ZC, r[j]);
#pragma unroll
  for (int v = 0; v < kBp2NV; ++v) bp2_fma<ZL>(acc[v], e.w[v], r[bp2_off(PAT, v)], r[bp2_off(PAT, v) + 1]);
}

template <typename SI, int ZL>
__device__ __forceinline__ void bp3_generic(const SI* rows, int b0, const Bp2Ent& e, float (&acc)[kBp2NV][ZL]) {
  const int i0[kBp2NV] = {e.i0.x, e.i0.y, e.i0.z, e.i0.w};
#pragma unroll
  for (int v = 0; v < kBp2NV; ++v) {
    float r0[ZL], r1[ZL];
    lds_row<SI, ZL>(rows + (i0[v] - b0) * kBp3ZC, r0);
    lds_row<SI, ZL>(rows + (i0[v] - b0 + 1) * kBp3ZC, r1);
    bp2_fma<ZL>(acc[v], e.w[v], r0, r1);
  }
}

// Highest bin (exclusive) a warp's entry reads: b + rows of the pattern, or
// max floor(u) + 2 for the generic body.
__device__ __forceinline__ int bp3_top(const Bp2Ent& e) {
  if (e.pat != kBp2Generic) return e.b + bp2_rows(e.pat);
  return max(max(e.i0.x, e.i0.y), max(e.i0.z, e.i0.w)) + 2;
}

// rows: the staged box of the angle (bin b0 first), lane offset included.
template <typename SI, int ZL>
__device__ __forceinline__ void bp3_angle(const SI* rows, int b0, const Bp2Ent& e, float (&acc)[kBp2NV][ZL]) {
  SIPO_DCHECK(e.b >= b0 && bp3_top(e) - b0 <= kBp3Rows, 1);
  const SI* own = rows + (e.b - b0) * kBp3ZC;
  switch (e.pat) {
#define SIPO_BP3_CASE(P) \
  case P:                \
    bp3_body<SI, ZL, P>(own, e, acc); break;
    SIPO_BP2_PATTERNS(SIPO_BP3_CASE)
#undef SIPO_BP3_CASE
    default:
      bp3_generic<SI, ZL>(rows, b0, e, acc);
  }
}

// Shared-memory plan of the kernel (dynamic, one allocation, offsets from a
// 1024-byte aligned base): the stage boxes, per warp its angle table, the
// block's per-angle first bin and fit flags, live-warp flags, the abort flag
// and the stage barriers.  After a tile's last stage the boxes are free and
// hold the warps' accumulators for the fused epilogue.
template <typename SI>
struct Bp3Smem {
  static constexpr int kRowBytes = kBp3ZC * int(sizeof(SI));
  static constexpr int kBoxBytes = kBp3Rows * kRowBytes;
  static constexpr int kStageBytes = kBp3Angles * kBoxBytes;
  static constexpr size_t kTableBytes = sizeof(Bp2Ent) * kBp2Chunk;
  static constexpr size_t kAccBytes = size_t(kBp2NV) * 8 * 32 * sizeof(float);
  static constexpr size_t kStagesOff = 0;
  static constexpr size_t kBoxesBytes = size_t(kBp3Stages) * kStageBytes;
  static constexpr size_t kWarpOff = kBoxesBytes > kWarps * kAccBytes ? kBoxesBytes : kWarps * kAccBytes;
  static constexpr size_t kBlkOff = kWarpOff + kWarps * kTableBytes;      // int bstart[32], fits[32], live[8]
  static constexpr size_t kBarOff = (kBlkOff + (2 * kBp2Chunk + kWarps + 4) * sizeof(int) + 7) / 8 * 8;
  static constexpr size_t kBytes = kBarOff + kBp3Stages * sizeof(uint64_t) + 1024;  // + alignment slack
};

// ZL = 8 (256 z values per warp, nz a multiple of 256); C = float.
template <typename SI, typename S, int MINB, int MODE, typename O>
__global__ void __launch_bounds__(kThreads, MINB)
k_backproject3(const Geo<float> g, const SI* __restrict__ sino, const __grid_constant__ CUtensorMap tmap,
               const Bufs<S, float> b, O* __restrict__ out, const uint8_t* __restrict__ need) {
  using C = float;
  using SM = Bp3Smem<SI>;
  constexpr int ZL = 8, NV = kBp2NV, KC = kBp2Chunk;
  if (MODE != kBpStore && b.st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* stages = smem + SM::kStagesOff;
  int* bstart = reinterpret_cast<int*>(smem + SM::kBlkOff);
  int* fits = bstart + KC;
  int* live = fits + KC;
  int* abort_flag = live + kWarps;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SM::kBarOff);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Bp2Ent* tb = reinterpret_cast<Bp2Ent*>(smem + SM::kWarpOff + warp * SM::kTableBytes);
  constexpr int NR = MODE == kBpDual ? 2 : 0;
  double red[NR > 0 ? NR : 1] = {};
  StepScalars<C> sc{};
  if (MODE != kBpStore) sc = read_scalars<C>(b.st);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kBp3Stages; ++s) mbar_init(bars + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  __syncthreads();
  int stage_seq = 0;  // pipeline stages used by this block so far (same in every thread)

  const int ntx = (g.nx + NV - 1) / NV, nty = (g.ny + kWarps - 1) / kWarps;
  const int nzc = g.nz / kBp3ZC;
  const long long ntiles = (long long)ntx * nty * nzc;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int tz = int(t % nzc);
    const long long t1 = t / nzc;
    const int tx = int(t1 % ntx);
    const int ty = int(t1 / ntx);
    const int iy = ty * kWarps + warp;
    const int zt = tz * kBp3ZC;
    const int z0 = zt + lane * ZLayout<C, ZL>::G;
    unsigned mask = 0;
    if (iy < g.ny) {
      const int2 sp = g.xspan[iy];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int ix = tx * NV + v;
        if (ix < g.nx && ix >= sp.x && ix <= sp.y && (need == nullptr || need[(size_t)iy * g.nx + ix]))
          mask |= 1u << v;
      }
    }
    if (!__syncthreads_or(mask != 0u)) {
      // nothing to sum in the whole block tile; the plain operator over every
      // column (need == nullptr) still writes its zeros
      if constexpr (MODE == kBpStore) {
        if (need == nullptr && iy < g.ny) {
          C zero[ZL];
#pragma unroll
          for (int i = 0; i < ZL; ++i) zero[i] = C(0);
#pragma unroll
          for (int v = 0; v < NV; ++v)
            if (tx * NV + v < g.nx) store_z<O, C, ZL>(out + ((size_t)iy * g.nx + tx * NV + v) * g.nz + z0, zero);
        }
      }
      continue;
    }
    if (lane == 0) live[warp] = mask != 0u;
    C acc[NV][ZL];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int i = 0; i < ZL; ++i) acc[v][i] = C(0);
    const C yf = C(iy) - g.cy;
    const C xf0 = C(tx * NV) - g.cx;
    for (int k0 = 0; k0 < g.na; k0 += KC) {
      const int kn = min(KC, g.na - k0);
      if (mask != 0u && lane < kn) bp2_fill(g, k0 + lane, yf, xf0, iy, tx * NV, mask, tb[lane]);
      __syncthreads();
      // the block's first bin per angle, and whether every live warp's rows
      // fit in the staged box
      if (warp == 0 && lane < kn) {
        int lo = 0x7fffffff, hi = -0x7fffffff;
        for (int w = 0; w < kWarps; ++w) {
          if (!live[w]) continue;
          const Bp2Ent* tw = reinterpret_cast<const Bp2Ent*>(smem + SM::kWarpOff + w * SM::kTableBytes);
          const Bp2Ent& e = tw[lane];
          lo = min(lo, e.pat == kBp2Generic ? min(min(e.i0.x, e.i0.y), min(e.i0.z, e.i0.w)) : e.b);
          hi = max(hi, bp3_top(e));
        }
        bstart[lane] = lo;
        fits[lane] = (hi - lo <= kBp3Rows) ? 1 : 0;
      }
      __syncthreads();
      const int nst = (kn + kBp3Angles - 1) / kBp3Angles;
      auto issue = [&](int q) {  // thread 0: stage q of this chunk
        const int slot = int((stage_seq + q) % kBp3Stages);
        const int a_lo = q * kBp3Angles, a_n = min(kBp3Angles, kn - a_lo);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bars + slot, uint32_t(a_n * SM::kBoxBytes));
        for (int a = 0; a < a_n; ++a)
          tma_load_3d(stages + slot * SM::kStageBytes + a * SM::kBoxBytes, &tmap, zt, bstart[a_lo + a],
                      k0 + a_lo + a, bars + slot);
      };
      if (threadIdx.x == 0)
        for (int q = 0; q < min(nst, kBp3Stages); ++q) issue(q);
      for (int q = 0; q < nst; ++q) {
        const int seq = stage_seq + q;
        const int slot = int(seq % kBp3Stages);
        const uint32_t parity = uint32_t((seq / kBp3Stages) & 1);
        if (!mbar_wait(bars + slot, parity)) {
          atomicOr(&g_bp3_fault, 1u);
          *abort_flag = 1;
        }
        if (mask != 0u && !*abort_flag) {
          const int a_lo = q * kBp3Angles, a_n = min(kBp3Angles, kn - a_lo);
          for (int a = 0; a < a_n; ++a) {
            const int kk = a_lo + a;
            const Bp2Ent& e = tb[kk];
            if (fits[kk]) {
              const SI* box = reinterpret_cast<const SI*>(stages + slot * SM::kStageBytes + a * SM::kBoxBytes) +
                              lane * ZLayout<C, ZL>::G;
              bp3_angle<SI, ZL>(box, bstart[kk], e, acc);
            } else if (lane == 0) {
              atomicOr(&g_bp3_fault, 2u);  // a span wider than the box: not reachable for 4 x 8 tiles
            }
          }
        }
        __syncthreads();  // every warp is done with the slot
        if (*abort_flag) {
          // the copies still in flight write this block's shared memory: wait
          // for them (bounded) before the block ends
          if (threadIdx.x == 0)
            for (int j = q; j < min(nst, q + kBp3Stages); ++j) {
              const int sj = stage_seq + j;
              mbar_wait(bars + sj % kBp3Stages, uint32_t((sj / kBp3Stages) & 1));
            }
          __syncthreads();
          break;
        }
        if (threadIdx.x == 0 && q + kBp3Stages < nst) issue(q + kBp3Stages);
      }
      stage_seq += nst;
      if (*abort_flag) break;
    }
    if (*abort_flag) break;
    // epilogue (as k_backproject2): the accumulators go through the stage
    // boxes, free after the tile's last stage
    using LS = ZLayout<C, ZL>;
    C* stage = reinterpret_cast<C*>(stages + warp * SM::kAccBytes);
    constexpr bool kStage = MODE != kBpStore;
    if constexpr (kStage) {
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int q = 0; q < LS::NG; ++q)
#pragma unroll
          for (int i = 0; i < LS::G; ++i) stage[((v * LS::NG + q) * 32 + lane) * LS::G + i] = acc[v][q * LS::G + i];
      __syncwarp();
    }
    if (iy < g.ny) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int ix = tx * NV + v;
        if (ix >= g.nx) continue;
        const size_t base = ((size_t)iy * g.nx + ix) * g.nz + z0;
        if constexpr (MODE == kBpStore) {
          if (need == nullptr || ((mask >> v) & 1u)) store_z<O, C, ZL>(out + base, acc[v]);
        } else if ((mask >> v) & 1u) {
          using L = ZLayout<C, ZL>;
#pragma unroll
          for (int q = 0; q < L::NG; ++q) {
            C part[L::G];
#pragma unroll
            for (int i = 0; i < L::G; ++i) part[i] = stage[((v * L::NG + q) * 32 + lane) * L::G + i];
            dual_update<S, C, L::G, false>(b, sc, base + q * L::kStride, part, red);
          }
        }
      }
    }
    __syncthreads();  // tables and live flags are rewritten by the next tile
  }
  if constexpr (MODE == kBpDual) block_reduce_store<2>(red, b.part, kSlSBand);
}

}  // namespace sipo
