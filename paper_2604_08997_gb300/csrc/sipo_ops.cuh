// sipo_ops.cuh -- projector P_mu, backprojector P_mu^T and the separable PSF K.
//
// Backprojection (Eqs. 2-3, P^T): every voxel sums, over all angles, the two
// linearly interpolated detector taps floor(u) and floor(u)+1.  The operator is
// slice-separable (z is the rotation axis), so one weight pair per
// (x, y, angle) serves the whole z column: the lanes first compute the weights
// of 32 angles at once into a per-warp table, then the warp applies them with
// lanes holding z, each sinogram row one coalesced load of the warp's z segment.
//
// Projection (P, the exact transpose): gather form.  For each ray (angle, bin)
// the kernel walks the dominant axis of the ray direction and, on each row or
// column, evaluates the three candidate voxels whose interpolation can reach
// the bin, with weights equal bit for bit to the backprojector's.  The lanes
// evaluate 32 lines at once and the warp then streams the compacted taps.  No
// atomics; each output is written once.
//
// Both kernels run a grid-stride loop over tiles on a fixed grid of
// kRedBlocks blocks so that fused reductions have a fixed number of partials.
#pragma once

#include "sipo_solver.cuh"

namespace sipo {

enum FpMode : int { kFpStore = 0, kFpPrimal = 1, kFpPrimalCheck = 2, kFpResid = 3, kFpCert = 4, kFpCertZ = 5 };
enum BpMode : int { kBpStore = 0, kBpDual = 1 };


// --------------------------------------------------------------- projector
// Smallest integer >= x without the conversion unit (via floor_split of -x),
// as an int and as a float.
__device__ __forceinline__ void ceil_split(float x, float& cf, int& ci) {
  float f;
  int i;
  floor_split(-x, f, i);
  cf = -f;
  ci = -i;
}
__device__ __forceinline__ void ceil_split(double x, double& cf, int& ci) {
  cf = ceil(x);
  ci = int(cf);
}
__device__ __forceinline__ int ceil_int(float x) {
  float f;
  int i;
  ceil_split(x, f, i);
  return i;
}
__device__ __forceinline__ int ceil_int(double x) { return int(ceil(x)); }

// Candidate window: the voxels whose detector coordinate on the walked row is
// within 1 of bin j lie strictly inside (xc - h, xc + h), h = 1/|cos| <= sqrt 2
// (exact arithmetic).  With the FP32 rounding of u and of xc (< 1e-4) the
// widened window (xc - h - 1e-3, xc + h + 1e-3) is narrower than 3, so the
// three integers from ceil(xc - h - 1e-3) contain every voxel with a non-zero
// weight; each candidate's weight is then the backprojector's weight of the
// same u, so P stays the transpose.
constexpr float kCandEps = 1e-3f;

// Weight of the voxel with detector coordinate u in bin j (jm = j - 1).  The
// backprojector gives bin floor(u) the weight 1 - (u - floor u) and bin
// floor(u) + 1 the weight u - floor u.
//   FAST = false: that rule, literally.
//   FAST = true (j >= 2): max(0, 1 - |u - j|), the same float bit for bit.
// For |u - j| < 1 and j >= 2, u lies in [j/2, 2j], so u - j is exact
// (Sterbenz).  If u >= j, floor u = j and both forms round 1 - (u - j).  If
// u < j, floor u = j - 1 and the exact value of 1 - (j - u) is u - (j - 1),
// which the backprojector computes exactly, so it is representable and the
// rounding of 1 - (j - u) returns it.  If |u - j| >= 1 the rounded |u - j| is
// >= 1 too and the weight is 0, as it is in the backprojector.
template <bool FAST, typename C>
__device__ __forceinline__ C tap_weight(C u, C jf, C jm) {
  if constexpr (FAST) {
    const C t = C(1) - fabs(u - jf);
    return t > C(0) ? t : C(0);
  } else {
    C flo;
    int i0;
    floor_split(u, flo, i0);
    const C wv = u - flo;
    return (flo == jf) ? (C(1) - wv) : ((flo == jm) ? wv : C(0));
  }
}

// Column flags packed as bits for the projector's candidate test.  rows: for
// each y, bit (x + kNbPad) of word array [y][words] says whether column (y, x)
// may hold a non-zero input; cols: the same indexed [x][words] by y.  The pad
// of kNbPad zero bits on both ends lets the three-candidate window be read
// without bounds checks (the walk is clipped to spans within the grid).
constexpr int kNbPad = 32;
struct NeedBits {
  const uint32_t* rows;  // nullptr: use the vial spans instead
  const uint32_t* cols;
  int wr, wc;            // words per row / per column
  __device__ __forceinline__ unsigned window(const uint32_t* base, int line, int start) const {
    const int w = base == rows ? wr : wc;
    int b = start + kNbPad;
    b = b < 0 ? 0 : (b > 32 * w - 35 ? 32 * w - 35 : b);
    const uint32_t* p = base + (size_t)line * w + (b >> 5);
    const unsigned long long pair = (unsigned long long)__ldg(p) | ((unsigned long long)__ldg(p + 1) << 32);
    return unsigned(pair >> (b & 31)) & 7u;
  }
};

// One ray (angle k, bin j) of the projector, walked along y when
// |cos| >= |sin| (ROWS: on row iy the bin is reached from x near
// (j - inner) / cos) and along x otherwise (on column ix from y near
// (j - off - x cos) / sin); three candidates per line from the window start.
//
// The warp handles the ray's lines 32 at a time: lane l evaluates line
// r0 + l (window, flags, weights), the non-zero taps of the 32 lines are
// compacted in line order into the warp's tap list in shared memory (column
// index and weight), and the whole warp then streams that list, four taps per
// step, each tap a coalesced load of the warp's z segment of one voxel column
// and ZL fused multiply-adds.  Taps are applied in the order of the serial
// walk (line by line, candidates in increasing order), so the sums do not
// depend on how lines are split over lanes.
constexpr int kTapList = 96;  // 32 lines x 3 candidates

template <typename C>
struct TapList {
  int col[kTapList];
  C w[kTapList];
};

template <bool ROWS, bool FAST, typename C>
__device__ __forceinline__ int fp_line_taps(const Geo<C>& g, const NeedBits& nb, bool use_bits, int k, C jf,
                                            C c, C s, C inv_a, C h, int line, int (&col)[3], C (&wt)[3]) {
  const C jm = jf - C(1);
  C cf;
  int i0;
  C inner = C(0), xf = C(0);
  if constexpr (ROWS) {
    inner = geo_inner(C(line) - g.cy, s, g.off);
    ceil_split((jf - inner) * inv_a + g.cx - h, cf, i0);
  } else {
    xf = C(line) - g.cx;
    ceil_split((jf - g.off - xf * c) * inv_a + g.cy - h, cf, i0);
  }
  unsigned okm;
  if (use_bits) {
    okm = nb.window(ROWS ? nb.rows : nb.cols, line, i0);
  } else {
    const int2 sp = ROWS ? g.xspan[line] : g.yspan[line];
    okm = 0u;
#pragma unroll
    for (int m = 0; m < 3; ++m) okm |= unsigned(i0 + m >= sp.x && i0 + m <= sp.y) << m;
  }
  int nt = 0;
  if (okm == 0u) return 0;
  const C f0 = ROWS ? cf - g.cx : cf - g.cy;
  C eline = C(1);
  if (g.ex) eline = ROWS ? g.ey[(size_t)k * g.ny + line] : g.ex[(size_t)k * g.nx + line];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const C u = ROWS ? geo_outer(f0 + C(m), c, inner) : geo_outer(xf, c, geo_inner(f0 + C(m), s, g.off));
    C t = tap_weight<FAST>(u, jf, jm);
    t = ((okm >> m) & 1u) ? t : C(0);
    const int ix = ROWS ? i0 + m : line, iy = ROWS ? line : i0 + m;
    if (g.ex && t != C(0))
      t = ROWS ? t * (g.ex[(size_t)k * g.nx + ix] * eline) : t * (eline * g.ey[(size_t)k * g.ny + iy]);
    col[m] = iy * g.nx + ix;
    wt[m] = t;
    nt += t != C(0);
  }
  return nt;
}

// acc += w * v elementwise; single precision in packed pairs (__ffma2_rn:
// two z values per instruction, each rounded like fmaf).
template <typename C, int ZL>
__device__ __forceinline__ void fma_z(C (&acc)[ZL], C w, const C (&v)[ZL]) {
  if constexpr (sizeof(C) == 4 && ZL % 2 == 0) {
    const float2 ww = make_float2(w, w);
#pragma unroll
    for (int i = 0; i < ZL; i += 2) {
      const float2 a = __ffma2_rn(ww, make_float2(v[i], v[i + 1]), make_float2(acc[i], acc[i + 1]));
      acc[i] = a.x;
      acc[i + 1] = a.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < ZL; ++i) acc[i] = fma(w, v[i], acc[i]);
  }
}

template <bool ROWS, bool FAST, typename SI, typename C, int ZL>
__device__ __forceinline__ void fp_walk(const Geo<C>& g, const SI* vz, const NeedBits& nb, bool use_bits, int k,
                                        C jf, C c, C s, int lo, int hi, TapList<C>& tl, C (&acc)[ZL]) {
  const int lane = threadIdx.x & 31;
  const C a = ROWS ? c : s;
  const C inv_a = C(1) / a, h = C(1) / fabs(a) + C(kCandEps);
  for (int r0 = lo; r0 <= hi; r0 += 32) {
    int col[3] = {0, 0, 0};
    C wt[3] = {C(0), C(0), C(0)};
    int nt = 0;
    if (r0 + lane <= hi)
      nt = fp_line_taps<ROWS, FAST, C>(g, nb, use_bits, k, jf, c, s, inv_a, h, r0 + lane, col, wt);
    // exclusive prefix of the tap counts over the lanes = list positions
    int incl = nt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) continue;
    int pos = incl - nt;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      if (wt[m] != C(0)) {
        tl.col[pos] = col[m];
        tl.w[pos] = wt[m];
        ++pos;
      }
    }
    __syncwarp();
    int t = 0;
#ifdef SIPO_CHECKED
    for (int q = lane; q < total; q += 32) SIPO_DCHECK((unsigned(tl.col[q]) < unsigned(g.nx * g.ny)), 0);
#endif
    for (; t + 4 <= total; t += 4) {
      C v[4][ZL];
#pragma unroll
      for (int u = 0; u < 4; ++u) load_z<SI, C, ZL>(vz + (size_t)tl.col[t + u] * g.nz, v[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) fma_z<C, ZL>(acc, tl.w[t + u], v[u]);
    }
    for (; t < total; ++t) {
      C v[ZL];
      load_z<SI, C, ZL>(vz + (size_t)tl.col[t] * g.nz, v);
      fma_z<C, ZL>(acc, tl.w[t], v);
    }
    __syncwarp();
  }
}

// SI: element type read from `vol`; O: element type written by kFpStore.
// act_col: per (angle, bin) flag of rays with an active z (solver modes skip
// the others); nb: packed per-column flags of voxels whose input can be
// non-zero (the solver's dual combination vanishes on the other columns), or
// rows == nullptr to gather every in-vial voxel; rspan: per-ray walked span
// meeting such columns (nullptr: the whole ray).
//
// Tiles (angle, 8 consecutive bins, z segment) are numbered with the angle
// fastest, so the grid-stride loop gives every block a mix of central bins
// (long rays) and outer bins (short rays) and the blocks finish together.
template <typename SI, typename S, typename C, int ZL, int MODE, typename O>
__global__ void __launch_bounds__(kThreads)
k_project(const Geo<C> g, const SI* __restrict__ vol, const Bufs<S, C> b, O* __restrict__ out,
          const uint8_t* __restrict__ act_col, const NeedBits nb, const int2* __restrict__ rspan) {
  const bool use_bits = nb.rows != nullptr;
  if (MODE != kFpStore && b.st->done) return;
  constexpr int ZC = 32 * ZL;
  constexpr int NR = MODE == kFpPrimalCheck ? 2 : (MODE == kFpResid ? 4 : (MODE == kFpCert ? 1 : 0));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nzc = (g.nz + ZC - 1) / ZC;
  const int njb = (g.nd + kWarps - 1) / kWarps;
  const long long ntiles = (long long)g.na * njb * nzc;
  double red[NR > 0 ? NR : 1] = {};
  StepScalars<C> sc{};
  if (MODE == kFpPrimal || MODE == kFpPrimalCheck) sc = read_scalars<C>(b.st);
  __shared__ __align__(16) TapList<C> taps[kWarps];
  // slice-mode certificate: per-z maxima of the block (dynamic shared memory,
  // nz entries), merged into b.cert_kz after the tile loop
  extern __shared__ __align__(16) unsigned long long kz_block[];
  if constexpr (MODE == kFpCertZ) {
    for (int z = threadIdx.x; z < g.nz; z += blockDim.x) kz_block[z] = 0ull;
    __syncthreads();
  }

  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int k = int(t % g.na);
    const long long t1 = t / g.na;
    const int tz = int(t1 % nzc);
    const int jb = int(t1 / nzc);
    const int j = jb * kWarps + warp;
    const int z0 = tz * ZC + lane * ZLayout<C, ZL>::G;
    if (j >= g.nd) continue;
    if (MODE != kFpStore && act_col != nullptr && !act_col[(size_t)k * g.nd + j]) continue;
    const C esj = g.es ? g.es[(size_t)k * g.nd + j] : C(1);
    C acc[ZL];
#pragma unroll
    for (int i = 0; i < ZL; ++i) acc[i] = C(0);
    // The whole warp walks the ray (the walk uses warp shuffles); a lane past
    // the end of a ragged z column reads the column's first group instead and
    // never stores its result.
    if (esj != C(0)) {
      const C c = g.cs[2 * k], s = g.cs[2 * k + 1];
      const C jf = C(j);
      const C sj = jf - g.off;
      C H = C(0);
      if (g.r2i >= 0) {
        C a = fabs(sj) - C(1.5);
        a = a > C(0) ? a : C(0);
        const C R = C(g.vial_r);
        H = R * R - a * a;
        H = (H > C(0) ? sqrt(H) : C(0)) + C(1.5);
      }
      const SI* vz = vol + (z0 < g.nz ? z0 : 0);
      const bool rows = fabs(c) >= fabs(s);
      int lo = 0, hi = (rows ? g.ny : g.nx) - 1;
      if (g.r2i >= 0) {
        // walked-axis extent of the ray's chord through the vial (+1 margin)
        const C mid = rows ? sj * s + g.cy : sj * c + g.cx;
        const C half = (rows ? fabs(c) : fabs(s)) * H + C(1);
        lo = max(0, -ceil_int(-(mid - half)));
        hi = min(hi, ceil_int(mid + half));
      }
      if (rspan) {
        const int2 r = rspan[(size_t)k * g.nd + j];
        lo = max(lo, r.x);
        hi = min(hi, r.y);
      }
      TapList<C>& tl = taps[warp];
      if (rows) {
        if (j >= 2) fp_walk<true, true, SI, C, ZL>(g, vz, nb, use_bits, k, jf, c, s, lo, hi, tl, acc);
        else fp_walk<true, false, SI, C, ZL>(g, vz, nb, use_bits, k, jf, c, s, lo, hi, tl, acc);
      } else {
        if (j >= 2) fp_walk<false, true, SI, C, ZL>(g, vz, nb, use_bits, k, jf, c, s, lo, hi, tl, acc);
        else fp_walk<false, false, SI, C, ZL>(g, vz, nb, use_bits, k, jf, c, s, lo, hi, tl, acc);
      }
#pragma unroll
      for (int i = 0; i < ZL; ++i) acc[i] *= esj;
    }
    if (z0 >= g.nz) continue;
    const size_t base = ((size_t)k * g.nd + j) * g.nz + z0;
    SIPO_DCHECK((z0 + z_offset<C, ZL>(ZL - 1) < g.nz), 0);
    if constexpr (MODE == kFpStore) {
      store_z<O, C, ZL>(out + base, acc);
    } else if constexpr (MODE == kFpPrimal) {
      primal_update<S, C, ZL, false>(b, sc, base, acc, red);
    } else if constexpr (MODE == kFpPrimalCheck) {
      primal_update<S, C, ZL, true>(b, sc, base, acc, red);
    } else if constexpr (MODE == kFpResid) {
      resid_update<S, C, ZL>(b, base, acc, red);
    } else if constexpr (MODE == kFpCert) {
      cert_update<S, C, ZL>(b, base, acc, red);
    } else {
      cert_update_z<S, C, ZL>(b, base, z0, acc, kz_block);
    }
  }
  if constexpr (MODE == kFpCertZ) {
    __syncthreads();
    for (int z = threadIdx.x; z < g.nz; z += blockDim.x)
      if (kz_block[z] != 0ull) atomicMax(b.cert_kz + z, kz_block[z]);
  }
  if constexpr (MODE == kFpPrimalCheck) block_reduce_store<2>(red, b.part, kSlFpX);
  if constexpr (MODE == kFpResid) block_reduce_store<4, kResidMaxMask>(red, b.part, kSlRd2);
  if constexpr (MODE == kFpCert) block_reduce_store<1, 1u>(red, b.part, kSlCertK);
}

// ----------------------------------------------------------- backprojector
// Per-angle interpolation data of a warp's NV voxels, computed by the lanes
// for kBpChunk angles at once (lane l: angle k0 + l): for voxel v, the first
// tap i0 = floor(u) and the weights w0 (bin i0) and w1 (bin i0 + 1),
// attenuation and vial factors included.  Voxels without their flag keep
// their i0 (so the detector window below still moves monotonically) and get
// zero weights; their sums are never stored.
template <typename C> struct alignas(2 * sizeof(C) >= 16 ? 8 : 16) BpEnt {
  C w0, w1;
  int i0, pad;
};
template <typename C> constexpr int bp_chunk() { return sizeof(C) == 8 ? 16 : 32; }

template <typename C, int NV>
struct BpTable {
  BpEnt<C> e[NV][bp_chunk<C>()];
};

template <typename C, int NV>
__device__ __forceinline__ void bp_fill(const Geo<C>& g, int k, C yf, C xf0, int iy, int tx0, unsigned mask,
                                        BpTable<C, NV>& tb, int slot) {
  const C c = g.cs[2 * k], s = g.cs[2 * k + 1];
  const C inner = geo_inner(yf, s, g.off);
  const C eyv = g.ex ? g.ey[(size_t)k * g.ny + iy] : C(1);
  const C* esk = g.es ? g.es + (size_t)k * g.nd : nullptr;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const C u = geo_outer(xf0 + C(v), c, inner);
    C flo;
    int i0;
    floor_split(u, flo, i0);
    C w0 = C(0), w1 = C(0);
    if ((mask >> v) & 1u) {
      const C wv = u - flo;
      const C e = g.ex ? g.ex[(size_t)k * g.nx + tx0 + v] * eyv : C(1);
      w0 = (C(1) - wv) * e;
      w1 = wv * e;
      if (esk) {
        w0 = unsigned(i0) < unsigned(g.nd) ? w0 * esk[i0] : C(0);
        w1 = unsigned(i0 + 1) < unsigned(g.nd) ? w1 * esk[i0 + 1] : C(0);
      }
    }
    BpEnt<C> en;
    en.w0 = w0;
    en.w1 = w1;
    en.i0 = i0;
    en.pad = 0;
    tb.e[v][slot] = en;
  }
}

// One angle (table column kk) for the NV voxels of a warp's row segment.
// Voxels are visited in increasing detector coordinate (left to right when
// cos >= 0, right to left otherwise); u then never decreases and floor(u)
// advances by 0 or 1 from one voxel to the next (|cos| <= 1), so a two-row
// window (rows cur and cur + 1, ZL values per lane each) slides along the
// detector and each sinogram row is loaded once per angle instead of once per
// voxel.  Rows off the detector are zero.
template <typename SI, typename C, int ZL>
__device__ __forceinline__ void bp_load_row(const Geo<C>& g, const SI* srow, int r, C (&t)[ZL]) {
  if (unsigned(r) < unsigned(g.nd)) {
    load_z<SI, C, ZL>(srow + (size_t)r * g.nz, t);
  } else {
#pragma unroll
    for (int i = 0; i < ZL; ++i) t[i] = C(0);
  }
}

template <typename SI, typename C, int ZL, int NV, bool FWD>
__device__ __forceinline__ void bp_angle(const Geo<C>& g, const SI* srow, const BpTable<C, NV>& tb, int kk,
                                         C (&acc)[NV][ZL]) {
  int cur = -2147483647;
  C r0[ZL], r1[ZL];  // rows cur and cur + 1
#pragma unroll
  for (int i = 0; i < ZL; ++i) { r0[i] = C(0); r1[i] = C(0); }
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const int v = FWD ? q : NV - 1 - q;
    const BpEnt<C> en = tb.e[v][kk];
    const int i0 = en.i0;
    if (i0 != cur) {
      if (i0 == cur + 1) {
#pragma unroll
        for (int i = 0; i < ZL; ++i) r0[i] = r1[i];
      } else {
        bp_load_row<SI, C, ZL>(g, srow, i0, r0);
      }
      bp_load_row<SI, C, ZL>(g, srow, i0 + 1, r1);
      cur = i0;
    }
#pragma unroll
    for (int i = 0; i < ZL; ++i) acc[v][i] = fma(en.w1, r1[i], fma(en.w0, r0[i], acc[v][i]));
  }
}


// Tile: NV voxel columns along x per warp, one row per warp (8 rows per
// block), ZL z values per lane.  need: per (iy, ix) column flag (nullptr:
// every column); columns without it are skipped (and left unwritten in
// kBpStore mode unless need is nullptr).  Angles go in chunks (32 for FP32,
// 16 for FP64): the lanes fill the warp's BpTable for the chunk, then the warp
// applies the chunk's angles in order, so every voxel sums its angles in
// increasing order.
template <typename SI, typename S, typename C, int ZL, int NV, int MINB, int MODE, typename O>
__global__ void __launch_bounds__(kThreads, MINB)
k_backproject(const Geo<C> g, const SI* __restrict__ sino, const Bufs<S, C> b, O* __restrict__ out,
              const uint8_t* __restrict__ need) {
  if (MODE != kBpStore && b.st->done) return;
  constexpr int ZC = 32 * ZL;
  constexpr int NR = MODE == kBpDual ? 2 : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntx = (g.nx + NV - 1) / NV, nty = (g.ny + kWarps - 1) / kWarps;
  const int nzc = (g.nz + ZC - 1) / ZC;
  const long long ntiles = (long long)ntx * nty * nzc;
  double red[NR > 0 ? NR : 1] = {};
  StepScalars<C> sc{};
  if (MODE != kBpStore) sc = read_scalars<C>(b.st);
  // per warp: the angle table, reused after the angle loop to stage the
  // accumulators when they fit, so that the fused epilogue need not keep them
  // in registers
  constexpr size_t kStageBytes = size_t(NV) * ZL * 32 * sizeof(C);
  constexpr bool kStage = MODE != kBpStore && kStageBytes <= 4096;
  constexpr size_t kWarpBytes = sizeof(BpTable<C, NV>) > (kStage ? kStageBytes : 0) ? sizeof(BpTable<C, NV>)
                                                                                   : kStageBytes;
  __shared__ __align__(16) unsigned char smem_warp[kWarps][kWarpBytes];
  BpTable<C, NV>& tb = *reinterpret_cast<BpTable<C, NV>*>(smem_warp[warp]);

  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int tz = int(t % nzc);
    const long long t1 = t / nzc;
    const int tx = int(t1 % ntx);
    const int ty = int(t1 / ntx);
    const int iy = ty * kWarps + warp;
    const int z0 = tz * ZC + lane * ZLayout<C, ZL>::G;
    if (iy >= g.ny) continue;
    const int2 sp = g.xspan[iy];
    unsigned mask = 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int ix = tx * NV + v;
      if (ix < g.nx && ix >= sp.x && ix <= sp.y && (need == nullptr || need[(size_t)iy * g.nx + ix]))
        mask |= 1u << v;
    }
    C acc[NV][ZL];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int i = 0; i < ZL; ++i) acc[v][i] = C(0);
    // the whole warp takes part (table fill + shuffle-free broadcast reads);
    // a lane past the end of a ragged z column reads the column's first
    // group and never stores its result
    if (mask != 0u) {
      const C yf = C(iy) - g.cy;
      const C xf0 = C(tx * NV) - g.cx;
      const SI* sz = sino + (z0 < g.nz ? z0 : 0);
      constexpr int KC = bp_chunk<C>();
      for (int k0 = 0; k0 < g.na; k0 += KC) {
        if (lane < KC && k0 + lane < g.na) bp_fill<C, NV>(g, k0 + lane, yf, xf0, iy, tx * NV, mask, tb, lane);
        __syncwarp();
        const int kn = min(KC, g.na - k0);
        for (int kk = 0; kk < kn; ++kk) {
          const int k = k0 + kk;
          const SI* srow = sz + (size_t)k * g.nd * g.nz;
          if (g.cs[2 * k] >= C(0))
            bp_angle<SI, C, ZL, NV, true>(g, srow, tb, kk, acc);
          else
            bp_angle<SI, C, ZL, NV, false>(g, srow, tb, kk, acc);
        }
        __syncwarp();
      }
    }
    using LS = ZLayout<C, ZL>;
    C* stage = reinterpret_cast<C*>(smem_warp[warp]);
    if constexpr (kStage) {
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int q = 0; q < LS::NG; ++q)
#pragma unroll
          for (int i = 0; i < LS::G; ++i) stage[((v * LS::NG + q) * 32 + lane) * LS::G + i] = acc[v][q * LS::G + i];
      __syncwarp();
    }
    if (z0 >= g.nz) {
      __syncwarp();
      continue;
    }
    SIPO_DCHECK((z0 + z_offset<C, ZL>(ZL - 1) < g.nz), 2);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int ix = tx * NV + v;
      if (ix >= g.nx) continue;
      const size_t base = ((size_t)iy * g.nx + ix) * g.nz + z0;
      if constexpr (MODE == kBpStore) {
        if (need == nullptr || ((mask >> v) & 1u)) store_z<O, C, ZL>(out + base, acc[v]);
      } else if ((mask >> v) & 1u) {
        // the epilogue runs group by group to keep its live range short
        using L = ZLayout<C, ZL>;
#pragma unroll
        for (int q = 0; q < L::NG; ++q) {
          C part[L::G];
#pragma unroll
          for (int i = 0; i < L::G; ++i)
            part[i] = kStage ? stage[((v * L::NG + q) * 32 + lane) * L::G + i] : acc[v][q * L::G + i];
          dual_update<S, C, L::G, false>(b, sc, base + q * L::kStride, part, red);
        }
      }
    }
    __syncwarp();
  }
  if constexpr (MODE == kBpDual) block_reduce_store<2>(red, b.part, kSlSBand);
}

// ------------------------------------------ backprojector with row patterns
// Single-precision form of k_backproject with the same tiles, z layout,
// angle order and epilogues, and sums equal bit for bit.  Per angle the lanes
// write, for the warp's four voxels (x order), the first detector row
// b = min floor(u), the offsets floor(u_v) - b packed two bits each (the
// pattern) and the weights, each one twice (a float pair for the packed
// multiply-add), with zero weight on every tap whose bin is off the detector.
// u = fma(x, cos, inner) is monotone in x, so with |cos| <= 1 the offsets
// move by 0 or 1 from one voxel to the next: 15 patterns.  Each pattern has a
// body whose row indices are compile-time constants: the angle's two to five
// rows are loaded at once into named registers, clamped to the detector (a
// clamped row only meets zero weights, and 0 * x leaves a sum unchanged), and
// every voxel applies its two rows with packed FP32 multiply-adds
// (__ffma2_rn, two z values per instruction, each rounded like fmaf).  A
// pattern outside the 15 takes a generic body that loads each voxel's rows.
struct alignas(16) Bp2Ent {
  float4 w[4];  // voxel v: (w0, w0, w1, w1)
  int b, pat, pad0, pad1;
  int4 i0;      // floor(u) per voxel (read by the generic body only)
};
constexpr int kBp2Chunk = 32;
constexpr int kBp2Generic = 0xff;
constexpr int kBp2NV = 4;

__host__ __device__ constexpr int bp2_off(int pat, int v) { return (pat >> (2 * v)) & 3; }
__host__ __device__ constexpr int bp2_rows(int pat) {
  int m = 0;
  for (int v = 0; v < kBp2NV; ++v) m = bp2_off(pat, v) > m ? bp2_off(pat, v) : m;
  return m + 2;
}

__device__ __forceinline__ void bp2_fill(const Geo<float>& g, int k, float yf, float xf0, int iy, int tx0,
                                         unsigned mask, Bp2Ent& out) {
  const float c = g.cs[2 * k], s = g.cs[2 * k + 1];
  const float inner = geo_inner(yf, s, g.off);
  const float eyv = g.ex ? g.ey[(size_t)k * g.ny + iy] : 1.0f;
  const float* esk = g.es ? g.es + (size_t)k * g.nd : nullptr;
  int i0[kBp2NV];
  float w0[kBp2NV], w1[kBp2NV];
#pragma unroll
  for (int v = 0; v < kBp2NV; ++v) {
    const float u = geo_outer(xf0 + float(v), c, inner);
    float flo;
    floor_split(u, flo, i0[v]);
    float a = 0.0f, bb = 0.0f;
    if ((mask >> v) & 1u) {
      const float wv = u - flo;
      const float e = g.ex ? g.ex[(size_t)k * g.nx + tx0 + v] * eyv : 1.0f;
      a = (1.0f - wv) * e;
      bb = wv * e;
      if (esk) {
        a = unsigned(i0[v]) < unsigned(g.nd) ? a * esk[i0[v]] : 0.0f;
        bb = unsigned(i0[v] + 1) < unsigned(g.nd) ? bb * esk[i0[v] + 1] : 0.0f;
      }
    }
    w0[v] = unsigned(i0[v]) < unsigned(g.nd) ? a : 0.0f;
    w1[v] = unsigned(i0[v] + 1) < unsigned(g.nd) ? bb : 0.0f;
    // a clamped row is only ever met with a zero weight
    SIPO_DCHECK(w0[v] == 0.0f || unsigned(i0[v]) < unsigned(g.nd), 1);
    SIPO_DCHECK(w1[v] == 0.0f || unsigned(i0[v] + 1) < unsigned(g.nd), 1);
  }
  int b = i0[0];
#pragma unroll
  for (int v = 1; v < kBp2NV; ++v) b = min(b, i0[v]);
  bool inc = true, dec = true;
#pragma unroll
  for (int v = 0; v + 1 < kBp2NV; ++v) {
    const int st = i0[v + 1] - i0[v];
    inc = inc && (st == 0 || st == 1);
    dec = dec && (st == 0 || st == -1);
  }
  int pat = 0;
#pragma unroll
  for (int v = 0; v < kBp2NV; ++v) pat |= (i0[v] - b) << (2 * v);
  if (!(inc || dec)) pat = kBp2Generic;
#pragma unroll
  for (int v = 0; v < kBp2NV; ++v) out.w[v] = make_float4(w0[v], w0[v], w1[v], w1[v]);
  out.b = b;
  out.pat = pat;
  out.pad0 = 0;
  out.pad1 = 0;
  out.i0 = make_int4(i0[0], i0[1], i0[2], i0[3]);
}

// acc += w0 * r0 + w1 * r1 elementwise (w0 applied first), packed in pairs.
template <int ZL>
__device__ __forceinline__ void bp2_fma(float (&acc)[ZL], const float4& w, const float (&r0)[ZL],
                                        const float (&r1)[ZL]) {
  if constexpr (ZL % 2 == 0) {
    const float2 wa = make_float2(w.x, w.y), wb = make_float2(w.z, w.w);
#pragma unroll
    for (int i = 0; i < ZL; i += 2) {
      float2 a = make_float2(acc[i], acc[i + 1]);
      a = __ffma2_rn(wa, make_float2(r0[i], r0[i + 1]), a);
      a = __ffma2_rn(wb, make_float2(r1[i], r1[i + 1]), a);
      acc[i] = a.x;
      acc[i + 1] = a.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < ZL; ++i) acc[i] = fmaf(w.z, r1[i], fmaf(w.x, r0[i], acc[i]));
  }
}

template <typename SI, int ZL>
__device__ __forceinline__ void bp2_row(const Geo<float>& g, const SI* srow, int r, float (&t)[ZL]) {
  r = r < 0 ? 0 : (r >= g.nd ? g.nd - 1 : r);
  load_z<SI, float, ZL>(srow + (size_t)r * g.nz, t);
}

template <typename SI, int ZL, int PAT>
__device__ __forceinline__ void bp2_body(const Geo<float>& g, const SI* srow, const Bp2Ent& e,
                                         float (&acc)[kBp2NV][ZL]) {
  constexpr int NR = bp2_rows(PAT);
  float r[NR][ZL];
#pragma unroll
  for (int j = 0; j < NR; ++j) bp2_row<SI, ZL>(g, srow, e.b + j, r[j]);
#pragma unroll
  for (int v = 0; v < kBp2NV; ++v) bp2_fma<ZL>(acc[v], e.w[v], r[bp2_off(PAT, v)], r[bp2_off(PAT, v) + 1]);
}

template <typename SI, int ZL>
__device__ __forceinline__ void bp2_generic(const Geo<float>& g, const SI* srow, const Bp2Ent& e,
                                         float (&acc)[kBp2NV][ZL]) {
  const int i0[kBp2NV] = {e.i0.x, e.i0.y, e.i0.z, e.i0.w};
#pragma unroll
  for (int v = 0; v < kBp2NV; ++v) {
    float r0[ZL], r1[ZL];
    bp2_row<SI, ZL>(g, srow, i0[v], r0);
    bp2_row<SI, ZL>(g, srow, i0[v] + 1, r1);
    bp2_fma<ZL>(acc[v], e.w[v], r0, r1);
  }
}

#define SIPO_BP2_PATTERNS(X)                                                              \
  X(0x00) X(0x40) X(0x50) X(0x90) X(0x54) X(0x94) X(0xA4) X(0xE4)                          \
  X(0x01) X(0x05) X(0x15) X(0x06) X(0x16) X(0x1A) X(0x1B)

// One angle of a warp's four voxels: dispatch on the table entry's pattern.
template <typename SI, int ZL>
__device__ __forceinline__ void bp2_angle(const Geo<float>& g, const SI* srow, const Bp2Ent& e,
                                          float (&acc)[kBp2NV][ZL]) {
  switch (e.pat) {
#define SIPO_BP2_CASE(P) \
  case P:                \
    bp2_body<SI, ZL, P>(g, srow, e, acc); break;
    SIPO_BP2_PATTERNS(SIPO_BP2_CASE)
#undef SIPO_BP2_CASE
    default:
      bp2_generic<SI, ZL>(g, srow, e, acc);
  }
}

// Tile: 4 voxel columns along x per warp, one row per warp (8 rows per
// block), ZL z values per lane; need, modes and epilogues as in
// k_backproject.
template <typename SI, typename S, int ZL, int MINB, int MODE, typename O>
__global__ void __launch_bounds__(kThreads, MINB)
k_backproject2(const Geo<float> g, const SI* __restrict__ sino, const Bufs<S, float> b, O* __restrict__ out,
               const uint8_t* __restrict__ need) {
  using C = float;
  constexpr int NV = kBp2NV;
  if (MODE != kBpStore && b.st->done) return;
  constexpr int ZC = 32 * ZL;
  constexpr int NR = MODE == kBpDual ? 2 : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntx = (g.nx + NV - 1) / NV, nty = (g.ny + kWarps - 1) / kWarps;
  const int nzc = (g.nz + ZC - 1) / ZC;
  const long long ntiles = (long long)ntx * nty * nzc;
  double red[NR > 0 ? NR : 1] = {};
  StepScalars<C> sc{};
  if (MODE != kBpStore) sc = read_scalars<C>(b.st);
  constexpr size_t kTableBytes = sizeof(Bp2Ent) * kBp2Chunk;
  constexpr size_t kStageBytes = size_t(NV) * ZL * 32 * sizeof(C);
  constexpr bool kStage = MODE != kBpStore && kStageBytes <= 4096;
  constexpr size_t kWarpBytes = kTableBytes > (kStage ? kStageBytes : 0) ? kTableBytes : kStageBytes;
  __shared__ __align__(16) unsigned char smem_warp[kWarps][kWarpBytes];
  Bp2Ent* tb = reinterpret_cast<Bp2Ent*>(smem_warp[warp]);

  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int tz = int(t % nzc);
    const long long t1 = t / nzc;
    const int tx = int(t1 % ntx);
    const int ty = int(t1 / ntx);
    const int iy = ty * kWarps + warp;
    const int z0 = tz * ZC + lane * ZLayout<C, ZL>::G;
    if (iy >= g.ny) continue;
    const int2 sp = g.xspan[iy];
    unsigned mask = 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int ix = tx * NV + v;
      if (ix < g.nx && ix >= sp.x && ix <= sp.y && (need == nullptr || need[(size_t)iy * g.nx + ix]))
        mask |= 1u << v;
    }
    C acc[NV][ZL];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int i = 0; i < ZL; ++i) acc[v][i] = C(0);
    // the whole warp takes part; a lane past the end of a ragged z column
    // reads the column's first group and never stores its result
    if (mask != 0u) {
      const C yf = C(iy) - g.cy;
      const C xf0 = C(tx * NV) - g.cx;
      const SI* sz = sino + (z0 < g.nz ? z0 : 0);
      for (int k0 = 0; k0 < g.na; k0 += kBp2Chunk) {
        if (k0 + lane < g.na) bp2_fill(g, k0 + lane, yf, xf0, iy, tx * NV, mask, tb[lane]);
        __syncwarp();
        const int kn = min(kBp2Chunk, g.na - k0);
        for (int kk = 0; kk < kn; ++kk)
          bp2_angle<SI, ZL>(g, sz + (size_t)(k0 + kk) * g.nd * g.nz, tb[kk], acc);
        __syncwarp();
      }
    }
    using LS = ZLayout<C, ZL>;
    C* stage = reinterpret_cast<C*>(smem_warp[warp]);
    if constexpr (kStage) {
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int q = 0; q < LS::NG; ++q)
#pragma unroll
          for (int i = 0; i < LS::G; ++i) stage[((v * LS::NG + q) * 32 + lane) * LS::G + i] = acc[v][q * LS::G + i];
      __syncwarp();
    }
    if (z0 >= g.nz) {
      __syncwarp();
      continue;
    }
    SIPO_DCHECK((z0 + z_offset<C, ZL>(ZL - 1) < g.nz), 2);
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
          for (int i = 0; i < L::G; ++i)
            part[i] = kStage ? stage[((v * L::NG + q) * 32 + lane) * L::G + i] : acc[v][q * L::G + i];
          dual_update<S, C, L::G, false>(b, sc, base + q * L::kStride, part, red);
        }
      }
    }
    __syncwarp();
  }
  if constexpr (MODE == kBpDual) block_reduce_store<2>(red, b.part, kSlSBand);
}

// ----------------------------------------------------------- ray row spans
// For each ray (angle k, bin j): the first and last index along its walked
// axis at which a candidate voxel lies in a flagged column (need).  The span
// tests the window of k_project widened by one candidate on each side, so a
// one-off difference in how the compiler rounds the window start cannot drop
// a row: restricting the walk to the span skips only rows whose taps are all
// zero.  Empty spans are (1, 0).
template <typename C>
__global__ void __launch_bounds__(kThreads)
k_ray_spans(const Geo<C> g, const uint8_t* __restrict__ need, int2* __restrict__ out) {
  const long long n = (long long)g.na * g.nd;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    const int k = int(r / g.nd), j = int(r % g.nd);
    const C c = g.cs[2 * k], s = g.cs[2 * k + 1];
    const C jf = C(j);
    int first = 1, last = 0;
    if (fabs(c) >= fabs(s)) {
      const C inv_c = C(1) / c, h = C(1) / fabs(c) + C(kCandEps);
      for (int iy = 0; iy < g.ny; ++iy) {
        const int2 sp = g.xspan[iy];
        if (sp.x > sp.y) continue;
        const C inner = geo_inner(C(iy) - g.cy, s, g.off);
        const int ix0 = ceil_int((jf - inner) * inv_c + g.cx - h);
        bool hit = false;
        for (int m = -1; m < 4; ++m) {
          const int ix = ix0 + m;
          if (ix >= sp.x && ix <= sp.y && need[(size_t)iy * g.nx + ix]) hit = true;
        }
        if (hit) {
          if (first > last) first = iy;
          last = iy;
        }
      }
    } else {
      const C inv_s = C(1) / s, h = C(1) / fabs(s) + C(kCandEps);
      for (int ix = 0; ix < g.nx; ++ix) {
        const int2 sp = g.yspan[ix];
        if (sp.x > sp.y) continue;
        const C xf = C(ix) - g.cx;
        const int iy0 = ceil_int((jf - g.off - xf * c) * inv_s + g.cy - h);
        bool hit = false;
        for (int m = -1; m < 4; ++m) {
          const int iy = iy0 + m;
          if (iy >= sp.x && iy <= sp.y && need[(size_t)iy * g.nx + ix]) hit = true;
        }
        if (hit) {
          if (first > last) first = ix;
          last = ix;
        }
      }
    }
    out[r] = make_int2(first, last);
  }
}

// ------------------------------------------------------- separable PSF pass
// out = taps (*) in along one axis (0: x, stride nz; 1: y, stride nx*nz;
// 2: z, stride 1), zero outside the grid; taps has 2R+1 entries, applied in
// increasing order.  A thread makes VG consecutive z outputs of one (y, x)
// column (VG = 4 when nz % 4 == 0, else 1).  Along x and y each tap is one
// VG-wide load shared by the thread's outputs and the tap range is clipped to
// the grid; along z the VG + 2R inputs stream through a register window.
template <typename TI, typename C, int VG>
__device__ __forceinline__ void conv_load(const TI* p, C (&v)[VG]) {
  if constexpr (VG == 4 && sizeof(TI) == 4) {
    const uint4 r = __ldg(reinterpret_cast<const uint4*>(p));
    v[0] = __uint_as_float(r.x); v[1] = __uint_as_float(r.y);
    v[2] = __uint_as_float(r.z); v[3] = __uint_as_float(r.w);
  } else if constexpr (VG == 4 && sizeof(TI) == 2) {
    const uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
    v[0] = __uint_as_float(r.x << 16); v[1] = __uint_as_float(r.x & 0xffff0000u);
    v[2] = __uint_as_float(r.y << 16); v[3] = __uint_as_float(r.y & 0xffff0000u);
  } else {
#pragma unroll
    for (int j = 0; j < VG; ++j) v[j] = to_c(p[j]);
  }
}

// x and y passes.  A block covers kConvZ z groups of kConvA consecutive
// positions along the blurred axis (one line of the other in-plane axis): the
// 2R + 1 inputs of neighbouring outputs overlap, so most of each thread's tap
// loads hit the block's own L1 lines instead of L2.
constexpr int kConvZ = 16;
constexpr int kConvA = kThreads / kConvZ;

template <typename TI, typename TO, typename C, int VG>
__global__ void __launch_bounds__(kThreads)
k_conv_xy(const TI* __restrict__ in, TO* __restrict__ out, const C* __restrict__ taps, int R,
          int nx, int ny, int nz, int axis) {
  const int nzg = nz / VG;
  const int na = axis == 0 ? nx : ny, no = axis == 0 ? ny : nx;
  const int nta = (na + kConvA - 1) / kConvA, ntz = (nzg + kConvZ - 1) / kConvZ;
  const long long ntiles = (long long)no * nta * ntz;
  const int tz = threadIdx.x % kConvZ, ta = threadIdx.x / kConvZ;
  const size_t stride = axis == 0 ? (size_t)nz : (size_t)nx * nz;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int zt = int(t % ntz);
    const long long t1 = t / ntz;
    const int at = int(t1 % nta);
    const int o = int(t1 / nta);
    const int a = at * kConvA + ta, zg = zt * kConvZ + tz;
    if (a >= na || zg >= nzg) continue;
    const int ix = axis == 0 ? a : o, iy = axis == 0 ? o : a;
    const size_t cbase = ((size_t)iy * nx + ix) * nz + (size_t)zg * VG;
    const int m0 = max(0, R - a), m1 = min(2 * R, na - 1 - a + R);
    const TI* p = in + cbase + (long long)(m0 - R) * (long long)stride;
    C acc[VG];
#pragma unroll
    for (int j = 0; j < VG; ++j) acc[j] = C(0);
    for (int m = m0; m <= m1; ++m, p += stride) {
      C v[VG];
      conv_load<TI, C, VG>(p, v);
      const C tp = __ldg(taps + m);
#pragma unroll
      for (int j = 0; j < VG; ++j) acc[j] = fma(tp, v[j], acc[j]);
    }
    TO* op = out + cbase;
#pragma unroll
    for (int j = 0; j < VG; ++j) op[j] = from_c<TO>(acc[j]);
  }
}

// z pass: a thread makes VG consecutive z outputs of one column, its VG + 2R
// inputs streaming through a register window; the threads of a block cover
// consecutive z groups of consecutive columns.
template <typename TI, typename TO, typename C, int VG>
__global__ void __launch_bounds__(kThreads)
k_conv_z(const TI* __restrict__ in, TO* __restrict__ out, const C* __restrict__ taps, int R,
         int nx, int ny, int nz) {
  const int nzg = nz / VG;
  const int zt = nzg < kThreads ? nzg : kThreads;  // z groups per block pass
  const int lpb = kThreads / zt;                    // columns per block pass
  const int tz = threadIdx.x % zt, tl = threadIdx.x / zt;
  if (tl >= lpb) return;
  const int ncol = nx * ny;
  for (int colx = blockIdx.x * lpb + tl; colx < ncol; colx += gridDim.x * lpb) {
    const size_t cbase = (size_t)colx * nz;
    const TI* p = in + cbase;
    for (int zg = tz; zg < nzg; zg += zt) {
      const int z0 = zg * VG;
      C acc[VG], w[VG];
#pragma unroll
      for (int j = 0; j < VG; ++j) {
        acc[j] = C(0);
        const int z = z0 - R + j;
        w[j] = (z >= 0 && z < nz) ? to_c(p[z]) : C(0);
      }
      for (int m = 0; m <= 2 * R; ++m) {
        const C tp = __ldg(taps + m);
#pragma unroll
        for (int j = 0; j < VG; ++j) acc[j] = fma(tp, w[j], acc[j]);
#pragma unroll
        for (int j = 0; j + 1 < VG; ++j) w[j] = w[j + 1];
        const int z = z0 - R + m + VG;
        w[VG - 1] = (z >= 0 && z < nz) ? to_c(p[z]) : C(0);
      }
      TO* op = out + cbase + z0;
#pragma unroll
      for (int j = 0; j < VG; ++j) op[j] = from_c<TO>(acc[j]);
    }
  }
}

}  // namespace sipo
