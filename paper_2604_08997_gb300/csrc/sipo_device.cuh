// sipo_device.cuh -- device-side building blocks of the SiPO solver (sm_103a).
//
// Layouts (z = rotation axis, fastest): volume [ny][nx][nz], sinogram
// [n_angles][n_det][nz].  Every operator kernel maps the 32 lanes of a warp
// onto one z column segment of 32 * ZL values (ZL per lane, in 16-byte groups
// interleaved across the lanes), so all geometry (detector coordinate,
// interpolation weight, attenuation factor) is warp-uniform and every
// sinogram / volume access is a fully coalesced vector load.
#pragma once

#include <cuda_bf16.h>
#include <math_constants.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sipo {

constexpr int kThreads = 256;     // threads per block for every kernel
constexpr int kWarps = kThreads / 32;
// Grid of every reducing kernel: 8 blocks per SM of a 152-SM GB300.  It is a
// constant on purpose: the FP64 reductions sum one partial per block in block
// order, so a fixed grid keeps every solve bit-reproducible from one device to
// another whatever its SM count; the grid-stride loops stay correct on any.
constexpr int kRedBlocks = 1216;

// Streaming multiprocessors of the current device (cudaDeviceProp
// multiProcessorCount), cached per device: the element-wise kernels size
// their grids as a multiple of it.
inline int device_sms() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cache[dev] = n;
  }
  return cache[dev];
}
constexpr double kEta = 0.99;     // step factor on the Pock-Chambolle steps

enum Label : uint8_t { kExt = 0, kBand = 1, kGel = 2 };

// ------------------------------------------------------------ checked build
// Built with -DSIPO_CHECKED, the kernels test their computed indices (and the
// finiteness of their FP64 block sums) and record a violated check as a bit of
// a per-translation-unit device flag, read and cleared by sipo_check_flags();
// they neither trap nor stop, and the access goes ahead as in the plain build
// only when the check holds.  Plain builds compile the checks away.
//   bit 0: projector tap column or z offset out of range
//   bit 1: backprojector detector row or staged-box row out of range
//   bit 2: element-wise update index out of its array
//   bit 3: non-finite FP64 block sum
#ifdef SIPO_CHECKED
static __device__ unsigned int g_sipo_check = 0;
#define SIPO_DCHECK(cond, bit)                                      \
  do {                                                              \
    if (!(cond)) atomicOr(&::sipo::g_sipo_check, 1u << (bit));      \
  } while (0)
#else
#define SIPO_DCHECK(cond, bit) \
  do {                         \
  } while (0)
#endif

// ---------------------------------------------------------------- conversions
__device__ __forceinline__ float to_c(float x) { return x; }
__device__ __forceinline__ double to_c(double x) { return x; }
__device__ __forceinline__ float to_c(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename S> struct FromC {
  template <typename T> __device__ __forceinline__ static S cvt(T x) { return S(x); }
};
template <> struct FromC<__nv_bfloat16> {
  template <typename T> __device__ __forceinline__ static __nv_bfloat16 cvt(T x) {
    return __float2bfloat16_rn(float(x));
  }
};
// compute value -> storage element (round to nearest for bf16)
template <typename S, typename T> __device__ __forceinline__ S from_c(T x) { return FromC<S>::cvt(x); }

template <typename S> struct Compute { using type = float; };
template <> struct Compute<double> { using type = double; };

// ------------------------------------------------- z-vector loads and stores
// A z-vector of ZL elements per lane is NG = ZL / G groups of G consecutive
// elements, G = the number of compute elements in 16 bytes (4 floats, 2
// doubles; 1 on the scalar path).  Group q of lane l sits at
// p + q * 32 * G, where p = tile start + l * G: one access of the warp to a
// group covers 32 * G consecutive elements, so each request uses every byte of
// its sectors (16 bytes a lane for 4-byte data, 8 for bf16, 4 for labels).
// The host picks ZL = G or 2G only when nz is a multiple of G (and of 64 G for
// 2G), which keeps every group access aligned and inside its z column.
template <typename C, int ZL>
struct ZLayout {
  static constexpr int kVec = 16 / int(sizeof(C));
  static constexpr int G = ZL < kVec ? ZL : kVec;
  static constexpr int NG = ZL / G;
  static constexpr int kStride = 32 * G;  // elements between a lane's groups
  static_assert(ZL % G == 0, "ZL must be a multiple of the group size");
};

// Offset of element i of a lane's z-vector from its first group.
template <typename C, int ZL>
__device__ __forceinline__ constexpr int z_offset(int i) {
  using L = ZLayout<C, ZL>;
  return (i / L::G) * L::kStride + i % L::G;
}

// One group: G elements of storage type S at p.
template <typename S, typename C, int G>
__device__ __forceinline__ void load_group(const S* __restrict__ p, C* v) {
  constexpr int kBytes = int(sizeof(S)) * G;
  if constexpr (kBytes == 16) {
    const uint4 r = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
    if constexpr (sizeof(S) == 4) {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(w[j]);
    } else if constexpr (sizeof(S) == 8) {
#pragma unroll
      for (int j = 0; j < 2; ++j) v[j] = __hiloint2double(int(w[2 * j + 1]), int(w[2 * j]));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        v[2 * j] = __uint_as_float(w[j] << 16);
        v[2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
      }
    }
  } else if constexpr (kBytes == 8 && sizeof(S) == 2) {
    const uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
    v[0] = __uint_as_float(r.x << 16);
    v[1] = __uint_as_float(r.x & 0xffff0000u);
    v[2] = __uint_as_float(r.y << 16);
    v[3] = __uint_as_float(r.y & 0xffff0000u);
  } else {
#pragma unroll
    for (int i = 0; i < G; ++i) v[i] = to_c(p[i]);
  }
}

template <typename S, typename C, int G>
__device__ __forceinline__ void store_group(S* __restrict__ p, const C* v) {
  constexpr int kBytes = int(sizeof(S)) * G;
  if constexpr (kBytes == 16 && sizeof(S) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (kBytes == 16 && sizeof(S) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else if constexpr (sizeof(S) == 2 && (G == 4 || G == 8)) {
    uint32_t w[G / 2];
#pragma unroll
    for (int j = 0; j < G / 2; ++j) {
      __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      w[j] = *reinterpret_cast<uint32_t*>(&h);
    }
    if constexpr (G == 4) *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
    else *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
  } else {
#pragma unroll
    for (int i = 0; i < G; ++i) p[i] = from_c<S>(v[i]);
  }
}

// The lane's z-vector whose first group starts at p (layout above).
template <typename S, typename C, int ZL>
__device__ __forceinline__ void load_z(const S* __restrict__ p, C (&v)[ZL]) {
  using L = ZLayout<C, ZL>;
#pragma unroll
  for (int q = 0; q < L::NG; ++q) load_group<S, C, L::G>(p + q * L::kStride, v + q * L::G);
}

template <typename S, typename C, int ZL>
__device__ __forceinline__ void store_z(S* __restrict__ p, const C (&v)[ZL]) {
  using L = ZLayout<C, ZL>;
#pragma unroll
  for (int q = 0; q < L::NG; ++q) store_group<S, C, L::G>(p + q * L::kStride, v + q * L::G);
}

// Labels (one byte each) of the lane's z-vector, same layout.
template <typename C, int ZL>
__device__ __forceinline__ void load_labels(const uint8_t* __restrict__ p, uint8_t (&lab)[ZL]) {
  using L = ZLayout<C, ZL>;
#pragma unroll
  for (int q = 0; q < L::NG; ++q) {
    const uint8_t* pq = p + q * L::kStride;
    if constexpr (L::G == 4) {
      const uint32_t r = __ldg(reinterpret_cast<const uint32_t*>(pq));
#pragma unroll
      for (int j = 0; j < 4; ++j) lab[q * 4 + j] = (r >> (8 * j)) & 0xff;
    } else if constexpr (L::G == 2) {
      const uint32_t r = __ldg(reinterpret_cast<const unsigned short*>(pq));
      lab[q * 2] = r & 0xff;
      lab[q * 2 + 1] = (r >> 8) & 0xff;
    } else {
#pragma unroll
      for (int j = 0; j < L::G; ++j) lab[q * L::G + j] = pq[j];
    }
  }
}

// ------------------------------------------------------------------ geometry
// Detector coordinate u = x cos + y sin + off, split so that the y part is
// shared by a row.  Single precision uses two fused multiply-adds,
// u = fma(x, cos, fma(y, sin, off)); double precision uses separately rounded
// products and sums, u = (x*cos) + ((y*sin) + off).  The projector and the
// backprojector call exactly these functions, so their weights agree bit for
// bit and P is the exact transpose of P^T up to summation order.
__device__ __forceinline__ float geo_inner(float yf, float s, float off) { return fmaf(yf, s, off); }
__device__ __forceinline__ float geo_outer(float xf, float c, float in) { return fmaf(xf, c, in); }
__device__ __forceinline__ double geo_inner(double yf, double s, double off) {
  return __dadd_rn(__dmul_rn(yf, s), off);
}
__device__ __forceinline__ double geo_outer(double xf, double c, double in) {
  return __dadd_rn(__dmul_rn(xf, c), in);
}

template <typename C>
struct Geo {
  int nx, ny, nz, na, nd;
  C cx, cy, off;            // (nx-1)/2, (ny-1)/2, (nd-1)/2
  const C* cs;              // [na][2] cos, sin
  const C* ex;              // [na][nx] exp(mu x sin) or nullptr (no attenuation)
  const C* ey;              // [na][ny] exp(-mu y cos)
  const C* es;              // [na][nd] vial entry factor (0 off the vial) or nullptr
  double vial_r;            // R
  long long r2i;            // floor(4 R^2): integer vial threshold (-1: no vial)
  const int2* xspan;        // [ny]: inside-vial ix range of row iy (lo > hi: empty)
  const int2* yspan;        // [nx]: inside-vial iy range of column ix
};

// Voxel (ix, iy) inside the vial: x^2 + y^2 <= R^2 evaluated exactly in
// integers, (2ix - nx + 1)^2 + (2iy - ny + 1)^2 <= 4 R^2.
template <typename C>
__device__ __forceinline__ bool in_vial(const Geo<C>& g, int ix, int iy) {
  if (g.r2i < 0) return true;
  const long long a = 2LL * ix - (g.nx - 1), b = 2LL * iy - (g.ny - 1);
  return a * a + b * b <= g.r2i;
}

__device__ __forceinline__ float fl_(float x) { return floorf(x); }
__device__ __forceinline__ double fl_(double x) { return floor(x); }

// floor(u) as a value and as an int.  Single precision avoids the conversion
// unit: adding 1.5*2^23 with round-down lands u + M in [2^23, 2^24), where the
// float spacing is 1, so the sum is exactly M + floor(u) for |u| < 2^22; the
// difference of bit patterns is floor(u) and t - M recovers it as a float.
// The result equals floorf(u) bit for bit.
__device__ __forceinline__ void floor_split(float u, float& fl, int& i) {
  const float t = __fadd_rd(u, 12582912.0f);
  i = __float_as_int(t) - 0x4B400000;
  fl = t - 12582912.0f;
}
__device__ __forceinline__ void floor_split(double u, double& fl, int& i) {
  fl = floor(u);
  i = int(fl);
}


// --------------------------------------------------------------- reductions
// Deterministic block reduction of N doubles per thread: warp shuffles, then
// one pass over the warps in fixed order; thread 0 writes the block partials
// to part[slot * kRedBlocks + blockIdx.x].
// Slots whose bit is set in MAXMASK are reduced with max instead of sum.
template <int N, unsigned MAXMASK = 0u>
__device__ __forceinline__ void block_reduce_store(double (&v)[N], double* part, int slot0) {
  __shared__ double red[kWarps][N > 0 ? N : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double x = v[i];
    const bool mx = (MAXMASK >> i) & 1u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = mx ? fmax(x, y) : x + y;
    }
    if (lane == 0) red[warp][i] = x;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    const bool mx = (MAXMASK >> threadIdx.x) & 1u;
    double s = red[0][threadIdx.x];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) s = mx ? fmax(s, red[w][threadIdx.x]) : s + red[w][threadIdx.x];
    SIPO_DCHECK(isfinite(s) || (mx && s == CUDART_INF), 3);
    part[(slot0 + threadIdx.x) * kRedBlocks + blockIdx.x] = s;
  }
}

// Maximum of one slot over all kRedBlocks partials (non-negative values).
__device__ __forceinline__ double block_max_slot(const double* part, int slot) {
  __shared__ double tmp[kThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) s = fmax(s, part[slot * kRedBlocks + i]);
  tmp[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) tmp[threadIdx.x] = fmax(tmp[threadIdx.x], tmp[threadIdx.x + st]);
    __syncthreads();
  }
  double r = tmp[0];
  __syncthreads();
  return r;
}

// Sum of one slot over all kRedBlocks partials, by one block, fixed order.
__device__ __forceinline__ double block_sum_slot(const double* part, int slot) {
  __shared__ double tmp[kThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) s += part[slot * kRedBlocks + i];
  tmp[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) tmp[threadIdx.x] += tmp[threadIdx.x + st];
    __syncthreads();
  }
  double r = tmp[0];
  __syncthreads();
  return r;
}

}  // namespace sipo
