// sipo_psf.cuh -- single-precision separable PSF passes staged in shared
// memory (nz a multiple of 4).
//
// K = Kz Ky Kx with zero padding (each pass: out = sum over m of
// taps[m] * in[pos - R + m], m increasing, as k_conv_xy / k_conv_z).
//
// k_conv_xy_fused applies Kx and Ky in one pass over the volume: a block
// stages a tile of (16 + 2 Ry) x (16 + 2 Rx) columns x 16 z values (four
// 16-byte groups) in shared memory, zero outside the grid, runs the x pass
// over every staged row into a second buffer and the y pass from there into
// the output.  Each thread makes a run of outputs along the blurred axis with
// a sliding register window, so a staged value is read from shared memory
// once per run instead of once per tap.  The volume is read and written once
// for both axes, where two separate passes read and write it twice.
//
// k_conv_z_chunk applies Kz: a warp stages 128 z values of one column with
// R rounded up to 4 on each side (zeros outside the column); each lane reads
// its 4 + 2R inputs as 16-byte groups into registers and makes four
// consecutive outputs (R is a template parameter, up to kZMaxR).
#pragma once

#include <algorithm>
#include <type_traits>

#include "sipo_device.cuh"

namespace sipo {

constexpr int kXyT = 16;   // tile side along x and y
constexpr int kXyZG = 4;   // 16-byte z groups per tile (16 z values)
constexpr int kXyRunX = 8; // x outputs per thread in the x pass
constexpr int kXyRunY = 4; // y outputs per thread in the y pass
constexpr int kXyLoads = 8; // staging loads in flight per thread

// Rows of the staged tiles are padded by one column so that the lanes of a
// warp, which take consecutive z groups of rows of both parities, hit all 32
// banks (conflict-free 16-byte accesses).
__host__ __device__ constexpr int conv_xy_pitch_a(int rx) { return kXyT + 2 * rx + 1; }
constexpr int kXyPitchB = kXyT + 1;

// Dynamic shared memory of k_conv_xy_fused for radii (rx, ry), in bytes.
__host__ __device__ constexpr size_t conv_xy_smem(int rx, int ry) {
  return (size_t(kXyT + 2 * ry) * conv_xy_pitch_a(rx) + size_t(kXyT + 2 * ry) * kXyPitchB) * kXyZG *
             sizeof(float4) +
         size_t(2 * rx + 1 + 2 * ry + 1) * sizeof(float);
}

// acc += t * v, as two packed FP32 multiply-adds (each lane rounded like fmaf)
__device__ __forceinline__ void f4_fma(float4& acc, float t, const float4& v) {
  const float2 tt = make_float2(t, t);
  const float2 lo = __ffma2_rn(tt, make_float2(v.x, v.y), make_float2(acc.x, acc.y));
  const float2 hi = __ffma2_rn(tt, make_float2(v.z, v.w), make_float2(acc.z, acc.w));
  acc = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// A run of RUN outputs of one pass with a radius fixed at compile time:
// acc[i] = sum over m of taps[m] * src[(i + m) * stride], terms added in
// increasing m, each staged input read once and applied to every output it
// reaches (no register window to shift).
template <int RUN, int R>
__device__ __forceinline__ void conv_run(const float4* src, int stride, const float* taps, float4 (&acc)[RUN]) {
  float t[2 * R + 1];
#pragma unroll
  for (int m = 0; m <= 2 * R; ++m) t[m] = taps[m];
#pragma unroll
  for (int i = 0; i < RUN; ++i) acc[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
  for (int p = 0; p < RUN + 2 * R; ++p) {
    const float4 v = src[p * stride];
#pragma unroll
    for (int i = 0; i < RUN; ++i) {
      const int m = p - i;
      if (m >= 0 && m <= 2 * R) f4_fma(acc[i], t[m], v);
    }
  }
}

// RC >= 0: both radii are RC, fixed at compile time (tap loops unrolled, tile
// index arithmetic on constants); RC < 0: the radii rx_arg, ry_arg.
template <typename TI, typename TO, int RC>
__global__ void __launch_bounds__(kThreads)
k_conv_xy_fused(const TI* __restrict__ in, TO* __restrict__ out, const float* __restrict__ taps_x, int rx_arg,
                const float* __restrict__ taps_y, int ry_arg, int nx, int ny, int nz) {
  extern __shared__ __align__(16) float4 xy_smem[];
  const int rx = RC >= 0 ? RC : rx_arg, ry = RC >= 0 ? RC : ry_arg;
  const int wx = kXyT + 2 * rx, wy = kXyT + 2 * ry, pa = conv_xy_pitch_a(rx);
  float4* A = xy_smem;                                      // [wy][pa][kXyZG] input tile (wx used)
  float4* B = A + size_t(wy) * pa * kXyZG;                  // [wy][kXyPitchB][kXyZG] after the x pass
  float* tx = reinterpret_cast<float*>(B + size_t(wy) * kXyPitchB * kXyZG);
  float* ty = tx + 2 * rx + 1;
  for (int i = threadIdx.x; i < 2 * rx + 1; i += blockDim.x) tx[i] = taps_x[i];
  for (int i = threadIdx.x; i < 2 * ry + 1; i += blockDim.x) ty[i] = taps_y[i];
  const int nzg = nz / 4;
  const int ntz = (nzg + kXyZG - 1) / kXyZG, ntx = (nx + kXyT - 1) / kXyT, nty = (ny + kXyT - 1) / kXyT;
  const long long ntiles = (long long)nty * ntx * ntz;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int tz = int(t % ntz);
    const long long t1 = t / ntz;
    const int txi = int(t1 % ntx), tyi = int(t1 / ntx);
    const int gx0 = txi * kXyT - rx, gy0 = tyi * kXyT - ry, zg0 = tz * kXyZG;
    __syncthreads();  // the previous tile is done with A and B (and the taps are staged)
    if constexpr (RC >= 0) {
      // staging by rows: warp w takes rows w, w + kWarps, ...; lane l keeps z
      // group l % 4 and columns l / 4 + 8 j, so addresses advance by fixed
      // strides; two rows (2 JN loads per lane) in flight before any store
      constexpr int W = kXyT + 2 * (RC >= 0 ? RC : 0);
      constexpr int JN = (W * kXyZG + 31) / 32;
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      const int zg = lane % kXyZG, xl = lane / kXyZG;
      const bool zok = zg0 + zg < nzg;
      const size_t row_stride = (size_t)nx * nz;
      for (int yy0 = warp; yy0 < W; yy0 += 2 * kWarps) {
        float v[2][JN][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int yy = yy0 + h * kWarps;
          const int gy = gy0 + yy;
          const bool yok = yy < W && gy >= 0 && gy < ny && zok;
          const TI* prow = in + (size_t)(yok ? gy : 0) * row_stride + 4 * (zg0 + zg);
#pragma unroll
          for (int j = 0; j < JN; ++j) {
            const int xx = xl + 8 * j, gx = gx0 + xx;
            v[h][j][0] = v[h][j][1] = v[h][j][2] = v[h][j][3] = 0.0f;
            if (yok && xx < W && gx >= 0 && gx < nx) load_group<TI, float, 4>(prow + (size_t)gx * nz, v[h][j]);
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int yy = yy0 + h * kWarps;
          if (yy >= W) break;
#pragma unroll
          for (int j = 0; j < JN; ++j) {
            const int xx = xl + 8 * j;
            if (xx < W) A[(yy * pa + xx) * kXyZG + zg] = make_float4(v[h][j][0], v[h][j][1], v[h][j][2], v[h][j][3]);
          }
        }
      }
    } else {
    // staging: kXyLoads loads per thread in flight before any is stored
    const int na = wy * wx * kXyZG;
    for (int e0 = 0; e0 < na; e0 += kXyLoads * kThreads) {
      float v[kXyLoads][4];
#pragma unroll
      for (int i = 0; i < kXyLoads; ++i) {
        const int e = e0 + i * kThreads + threadIdx.x;
        const int zg = e % kXyZG, r = e / kXyZG;
        const int gx = gx0 + r % wx, gy = gy0 + r / wx, gzg = zg0 + zg;
        v[i][0] = v[i][1] = v[i][2] = v[i][3] = 0.0f;
        if (e < na && gx >= 0 && gx < nx && gy >= 0 && gy < ny && gzg < nzg)
          load_group<TI, float, 4>(in + ((size_t)gy * nx + gx) * nz + 4 * gzg, v[i]);
      }
#pragma unroll
      for (int i = 0; i < kXyLoads; ++i) {
        const int e = e0 + i * kThreads + threadIdx.x;
        if (e >= na) break;
        const int zg = e % kXyZG, r = e / kXyZG;
        A[(size_t(r / wx) * pa + r % wx) * kXyZG + zg] = make_float4(v[i][0], v[i][1], v[i][2], v[i][3]);
      }
    }
    }
    __syncthreads();
    // x pass over every staged row: item = (row, run, z group)
    constexpr int kRunsX = kXyT / kXyRunX;
    for (int it = threadIdx.x; it < wy * kRunsX * kXyZG; it += blockDim.x) {
      const int zg = it % kXyZG, r = it / kXyZG;
      const int run = r % kRunsX, yy = r / kRunsX;
      const float4* a = A + (size_t(yy) * pa + run * kXyRunX) * kXyZG + zg;
      float4 acc[kXyRunX];
      if constexpr (RC >= 0) {
        conv_run<kXyRunX, (RC >= 0 ? RC : 0)>(a, kXyZG, tx, acc);
      } else {
        float4 win[kXyRunX];
#pragma unroll
        for (int i = 0; i < kXyRunX; ++i) {
          acc[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          win[i] = a[i * kXyZG];
        }
        for (int m = 0; m <= 2 * rx; ++m) {
          const float tp = tx[m];
#pragma unroll
          for (int i = 0; i < kXyRunX; ++i) f4_fma(acc[i], tp, win[i]);
#pragma unroll
          for (int i = 0; i + 1 < kXyRunX; ++i) win[i] = win[i + 1];
          if (m < 2 * rx) win[kXyRunX - 1] = a[(m + kXyRunX) * kXyZG];
        }
      }
      float4* b = B + (size_t(yy) * kXyPitchB + run * kXyRunX) * kXyZG + zg;
#pragma unroll
      for (int i = 0; i < kXyRunX; ++i) b[i * kXyZG] = acc[i];
    }
    __syncthreads();
    // y pass: item = (run, x, z group)
    constexpr int kRunsY = kXyT / kXyRunY;
    for (int it = threadIdx.x; it < kRunsY * kXyT * kXyZG; it += blockDim.x) {
      const int zg = it % kXyZG, r = it / kXyZG;
      const int x = r % kXyT, run = r / kXyT;
      const float4* b = B + (size_t(run * kXyRunY) * kXyPitchB + x) * kXyZG + zg;
      constexpr int kRow = kXyPitchB * kXyZG;  // float4 between rows of B
      float4 acc[kXyRunY];
      if constexpr (RC >= 0) {
        conv_run<kXyRunY, (RC >= 0 ? RC : 0)>(b, kRow, ty, acc);
      } else {
        float4 win[kXyRunY];
#pragma unroll
        for (int i = 0; i < kXyRunY; ++i) {
          acc[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          win[i] = b[i * kRow];
        }
        for (int m = 0; m <= 2 * ry; ++m) {
          const float tp = ty[m];
#pragma unroll
          for (int i = 0; i < kXyRunY; ++i) f4_fma(acc[i], tp, win[i]);
#pragma unroll
          for (int i = 0; i + 1 < kXyRunY; ++i) win[i] = win[i + 1];
          if (m < 2 * ry) win[kXyRunY - 1] = b[(m + kXyRunY) * kRow];
        }
      }
      const int gx = txi * kXyT + x, gzg = zg0 + zg;
      if (gx >= nx || gzg >= nzg) continue;
#pragma unroll
      for (int i = 0; i < kXyRunY; ++i) {
        const int gy = tyi * kXyT + run * kXyRunY + i;
        if (gy >= ny) continue;
        const float v[4] = {acc[i].x, acc[i].y, acc[i].z, acc[i].w};
        store_group<TO, float, 4>(out + ((size_t)gy * nx + gx) * nz + 4 * gzg, v);
      }
    }
  }
}

// Launches k_conv_xy_fused (radii compiled in when rx == ry <= 12).
template <typename TI, typename TO>
void launch_conv_xy_fused(const TI* in, TO* out, const float* tx, int rx, const float* ty, int ry, int nx, int ny,
                          int nz, int grid, size_t smem, cudaStream_t s) {
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    kern<<<grid, kThreads, smem, s>>>(in, out, tx, rx, ty, ry, nx, ny, nz);
  };
  switch (rx == ry ? rx : -1) {
#define SIPO_XYCASE(RR) \
  case RR:              \
    go(k_conv_xy_fused<TI, TO, RR>); return;
    SIPO_XYCASE(1) SIPO_XYCASE(2) SIPO_XYCASE(3) SIPO_XYCASE(4) SIPO_XYCASE(5) SIPO_XYCASE(6) SIPO_XYCASE(7)
    SIPO_XYCASE(8) SIPO_XYCASE(9) SIPO_XYCASE(10) SIPO_XYCASE(11) SIPO_XYCASE(12)
#undef SIPO_XYCASE
    default:
      go(k_conv_xy_fused<TI, TO, -1>);
  }
}

constexpr int kZChunk = 128;   // z outputs per warp item
constexpr int kZMaxR = 16;     // largest z radius with a compiled kernel

// Staged values per warp for radius R: kZChunk + 2 RP, RP = R rounded up to 4.
__host__ __device__ constexpr int conv_z_span(int r) { return kZChunk + 2 * ((r + 3) & ~3); }

template <typename TI, typename TO, int R>
__global__ void __launch_bounds__(kThreads)
k_conv_z_chunk(const TI* __restrict__ in, TO* __restrict__ out, const float* __restrict__ taps, int nx, int ny,
               int nz) {
  constexpr int RP = (R + 3) & ~3;
  constexpr int SPAN = conv_z_span(R);
  constexpr int NQ = RP / 2 + 1;  // 16-byte groups a lane reads: staged [4 lane, 4 lane + 2 RP + 4)
  __shared__ __align__(16) float w_all[kWarps][SPAN];
  __shared__ float tp[2 * R + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* w = w_all[warp];
  for (int i = threadIdx.x; i < 2 * R + 1; i += blockDim.x) tp[i] = taps[i];
  __syncthreads();
  const int nch = (nz + kZChunk - 1) / kZChunk;
  const long long items = (long long)nx * ny * nch;
  for (long long it = (long long)blockIdx.x * kWarps + warp; it < items; it += (long long)gridDim.x * kWarps) {
    const long long col = it / nch;
    const int z0 = int(it % nch) * kZChunk;
    const TI* p = in + (size_t)col * nz;
    __syncwarp();  // the warp's previous item is done with w
    // the staged groups (at most 64 for R <= kZMaxR): both of a lane's loads
    // in flight before either is stored
    static_assert(SPAN / 4 <= 64, "two staged groups per lane");
    float st[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = lane + 32 * h, z = z0 - RP + 4 * g;
      st[h][0] = st[h][1] = st[h][2] = st[h][3] = 0.0f;
      // nz % 4 == 0: a group is wholly inside the column or wholly outside
      if (g < SPAN / 4 && z >= 0 && z < nz) load_group<TI, float, 4>(p + z, st[h]);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = lane + 32 * h;
      if (g < SPAN / 4) reinterpret_cast<float4*>(w)[g] = make_float4(st[h][0], st[h][1], st[h][2], st[h][3]);
    }
    __syncwarp();
    const int zo = z0 + 4 * lane;
    if (zo >= nz) continue;
    // staged index of input zo + j - R + m is 4 lane + RP - R + j + m
    float v[4 * NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float4 r4 = reinterpret_cast<const float4*>(w)[lane + q];
      v[4 * q] = r4.x; v[4 * q + 1] = r4.y; v[4 * q + 2] = r4.z; v[4 * q + 3] = r4.w;
    }
    float2 a01 = make_float2(0.0f, 0.0f), a23 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int m = 0; m <= 2 * R; ++m) {
      const float2 t = make_float2(tp[m], tp[m]);
      a01 = __ffma2_rn(t, make_float2(v[RP - R + m], v[RP - R + m + 1]), a01);
      a23 = __ffma2_rn(t, make_float2(v[RP - R + m + 2], v[RP - R + m + 3]), a23);
    }
    const float acc[4] = {a01.x, a01.y, a23.x, a23.y};
    store_group<TO, float, 4>(out + (size_t)col * nz + zo, acc);
  }
}

// Launches k_conv_z_chunk for radius r (0..kZMaxR); false for a larger r.
template <typename TI, typename TO>
bool launch_conv_z_chunk(const TI* in, TO* out, const float* taps, int r, int nx, int ny, int nz, int grid,
                         cudaStream_t s) {
  switch (r) {
#define SIPO_ZCASE(RR) \
  case RR:             \
    k_conv_z_chunk<TI, TO, RR><<<grid, kThreads, 0, s>>>(in, out, taps, nx, ny, nz); return true;
    SIPO_ZCASE(0) SIPO_ZCASE(1) SIPO_ZCASE(2) SIPO_ZCASE(3) SIPO_ZCASE(4) SIPO_ZCASE(5) SIPO_ZCASE(6)
    SIPO_ZCASE(7) SIPO_ZCASE(8) SIPO_ZCASE(9) SIPO_ZCASE(10) SIPO_ZCASE(11) SIPO_ZCASE(12) SIPO_ZCASE(13)
    SIPO_ZCASE(14) SIPO_ZCASE(15) SIPO_ZCASE(16)
#undef SIPO_ZCASE
    default:
      return false;
  }
}

}  // namespace sipo
