// sipo_ops.cuh -- projector P_mu, backprojector P_mu^T and the separable PSF K.
//
// Backprojection (Eqs. 2-3, P^T): every voxel sums, over all angles, the two
// linearly interpolated detector taps floor(u) and floor(u)+1.  The operator is
// slice-separable (z is the rotation axis), so one weight pair per
// (x, y, angle) serves the whole z column: lanes hold z, the geometry is
// warp-uniform, and each tap is one coalesced 16-byte vector load per lane.
//
// Projection (P, the exact transpose): gather form.  For each ray (angle, bin)
// the kernel walks the dominant axis of the ray direction and, on each row or
// column, evaluates the <= 5 voxels whose interpolation reaches the bin with
// the very same arithmetic as the backprojector, so the weights agree bit for
// bit.  No atomics; each output is written once.
//
// Both kernels run a grid-stride loop over tiles on a fixed grid of
// kRedBlocks blocks so that fused reductions have a fixed number of partials.
#pragma once

#include "sipo_solver.cuh"

namespace sipo {

enum FpMode : int { kFpStore = 0, kFpPrimal = 1, kFpPrimalCheck = 2, kFpResid = 3 };
enum BpMode : int { kBpStore = 0, kBpDual = 1, kBpDualCheck = 2 };


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

// --------------------------------------------------------------- projector
// Smallest integer >= x without the conversion unit (via floor_split of -x).
__device__ __forceinline__ int ceil_int(float x) {
  float f;
  int i;
  floor_split(-x, f, i);
  return -i;
}
__device__ __forceinline__ int ceil_int(double x) { return int(ceil(x)); }

// Candidate window: the voxels whose detector coordinate on the walked row is
// within 1 of bin j lie strictly inside (xc - h, xc + h), h = 1/|cos| <= sqrt 2
// (exact arithmetic).  With the FP32 rounding of u and of xc (< 1e-4) the
// widened window (xc - h - 1e-3, xc + h + 1e-3) is narrower than 3, so the
// three integers from ceil(xc - h - 1e-3) contain every voxel with a non-zero
// weight; each candidate's weight is then computed exactly as the
// backprojector computes it (same u, same floor), so P stays the transpose.
constexpr float kCandEps = 1e-3f;

// SI: element type read from `vol`; O: element type written by kFpStore.
// act_col: per (angle, bin) flag of rays with an active z (solver modes skip
// the others); need: per (y, x) column flag of voxels whose input can be
// non-zero (the solver's dual combination vanishes on exterior columns), or
// nullptr to gather every in-vial voxel.
template <typename SI, typename S, typename C, int ZL, int MODE, typename O>
__global__ void __launch_bounds__(kThreads)
k_project(const Geo<C> g, const SI* __restrict__ vol, const Bufs<S, C> b, O* __restrict__ out,
          const uint8_t* __restrict__ act_col, const NeedBits nb, const int2* __restrict__ rspan) {
  const bool use_bits = nb.rows != nullptr;
  if (MODE != kFpStore && b.st->done) return;
  constexpr int ZC = 32 * ZL;
  constexpr int NR = MODE == kFpPrimalCheck ? 2 : (MODE == kFpResid ? 4 : 0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nzc = (g.nz + ZC - 1) / ZC;
  const int njb = (g.nd + kWarps - 1) / kWarps;
  const long long ntiles = (long long)g.na * njb * nzc;
  double red[NR > 0 ? NR : 1] = {};
  StepScalars<C> sc{};
  if (MODE == kFpPrimal || MODE == kFpPrimalCheck) sc = read_scalars<C>(b.st);

  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int tz = int(t % nzc);
    const long long t1 = t / nzc;
    const int jb = int(t1 % njb);
    const int k = int(t1 / njb);
    const int j = jb * kWarps + warp;
    const int z0 = tz * ZC + lane * ZL;
    if (j >= g.nd) continue;
    if (MODE != kFpStore && act_col != nullptr && !act_col[(size_t)k * g.nd + j]) continue;
    const C esj = g.es ? g.es[(size_t)k * g.nd + j] : C(1);
    C acc[ZL];
#pragma unroll
    for (int i = 0; i < ZL; ++i) acc[i] = C(0);
    if (esj != C(0) && z0 < g.nz) {
      const C c = g.cs[2 * k], s = g.cs[2 * k + 1];
      const C jf = C(j), jm = C(j - 1);
      const C sj = jf - g.off;
      C H = C(0);
      if (g.r2i >= 0) {
        C a = fabs(sj) - C(1.5);
        a = a > C(0) ? a : C(0);
        const C R = C(g.vial_r);
        H = R * R - a * a;
        H = (H > C(0) ? sqrt(H) : C(0)) + C(1.5);
      }
      const SI* vz = vol + z0;
      if (fabs(c) >= fabs(s)) {
        // walk rows iy; on each row the bin is reached from x near (j - inner) / cos
        int lo = 0, hi = g.ny - 1;
        if (g.r2i >= 0) {
          const C yc = sj * s, hy = fabs(c) * H + C(1);
          lo = max(0, -ceil_int(-(yc - hy + g.cy)));
          hi = min(g.ny - 1, ceil_int(yc + hy + g.cy));
        }
        if (rspan) {
          const int2 r = rspan[(size_t)k * g.nd + j];
          lo = max(lo, r.x);
          hi = min(hi, r.y);
        }
        const C inv_c = C(1) / c, h = C(1) / fabs(c) + C(kCandEps);
        C yf = C(lo) - g.cy;
        for (int iy = lo; iy <= hi; ++iy, yf += C(1)) {
          const C inner = geo_inner(yf, s, g.off);
          const C ixc = (jf - inner) * inv_c + g.cx;
          const int ix0 = ceil_int(ixc - h);
          unsigned okm;
          if (use_bits) {
            okm = nb.window(nb.rows, iy, ix0);
          } else {
            const int2 sp = g.xspan[iy];
            okm = 0u;
#pragma unroll
            for (int m = 0; m < 3; ++m) okm |= unsigned(ix0 + m >= sp.x && ix0 + m <= sp.y) << m;
          }
          if (okm == 0u) continue;
          const C xf0 = C(ix0) - g.cx;
          C wt[3];
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const C u = geo_outer(xf0 + C(m), c, inner);
            C flo;
            int i0;
            floor_split(u, flo, i0);
            const C wv = u - flo;
            const C t = (flo == jf) ? (C(1) - wv) : ((flo == jm) ? wv : C(0));
            wt[m] = ((okm >> m) & 1u) ? t : C(0);
          }
          const C eyv = g.ex ? g.ey[(size_t)k * g.ny + iy] : C(1);
          const SI* vrow = vz + ((size_t)iy * g.nx) * g.nz;
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            if (wt[m] == C(0)) continue;
            const int ix = ix0 + m;
            const C w = g.ex ? wt[m] * (g.ex[(size_t)k * g.nx + ix] * eyv) : wt[m];
            C v[ZL];
            load_z<SI, C, ZL>(vrow + (size_t)ix * g.nz, v);
#pragma unroll
            for (int i = 0; i < ZL; ++i) acc[i] = fma(w, v[i], acc[i]);
          }
        }
      } else {
        // walk columns ix; on each column the bin is reached from y near (j - off - x cos) / sin
        int lo = 0, hi = g.nx - 1;
        if (g.r2i >= 0) {
          const C xc = sj * c, hx = fabs(s) * H + C(1);
          lo = max(0, -ceil_int(-(xc - hx + g.cx)));
          hi = min(g.nx - 1, ceil_int(xc + hx + g.cx));
        }
        if (rspan) {
          const int2 r = rspan[(size_t)k * g.nd + j];
          lo = max(lo, r.x);
          hi = min(hi, r.y);
        }
        const C inv_s = C(1) / s, h = C(1) / fabs(s) + C(kCandEps);
        C xf = C(lo) - g.cx;
        for (int ix = lo; ix <= hi; ++ix, xf += C(1)) {
          const C iyc = (jf - g.off - xf * c) * inv_s + g.cy;
          const int iy0 = ceil_int(iyc - h);
          unsigned okm;
          if (use_bits) {
            okm = nb.window(nb.cols, ix, iy0);
          } else {
            const int2 sp = g.yspan[ix];
            okm = 0u;
#pragma unroll
            for (int m = 0; m < 3; ++m) okm |= unsigned(iy0 + m >= sp.x && iy0 + m <= sp.y) << m;
          }
          if (okm == 0u) continue;
          const C yf0 = C(iy0) - g.cy;
          C wt[3];
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const C u = geo_outer(xf, c, geo_inner(yf0 + C(m), s, g.off));
            C flo;
            int i0;
            floor_split(u, flo, i0);
            const C wv = u - flo;
            const C t = (flo == jf) ? (C(1) - wv) : ((flo == jm) ? wv : C(0));
            wt[m] = ((okm >> m) & 1u) ? t : C(0);
          }
          const C exv = g.ex ? g.ex[(size_t)k * g.nx + ix] : C(1);
          const SI* vcol = vz + (size_t)ix * g.nz;
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            if (wt[m] == C(0)) continue;
            const int iy = iy0 + m;
            const C w = g.ex ? wt[m] * (exv * g.ey[(size_t)k * g.ny + iy]) : wt[m];
            C v[ZL];
            load_z<SI, C, ZL>(vcol + (size_t)iy * g.nx * g.nz, v);
#pragma unroll
            for (int i = 0; i < ZL; ++i) acc[i] = fma(w, v[i], acc[i]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < ZL; ++i) acc[i] *= esj;
    }
    if (z0 >= g.nz) continue;
    const size_t base = ((size_t)k * g.nd + j) * g.nz + z0;
    if constexpr (MODE == kFpStore) {
      store_z<O, C, ZL>(out + base, acc);
    } else if constexpr (MODE == kFpPrimal) {
      primal_update<S, C, ZL, false>(b, sc, base, acc, red);
    } else if constexpr (MODE == kFpPrimalCheck) {
      primal_update<S, C, ZL, true>(b, sc, base, acc, red);
    } else {
      resid_update<S, C, ZL>(b, base, acc, red);
    }
  }
  if constexpr (MODE == kFpPrimalCheck) block_reduce_store<2>(red, b.part, kSlFpX);
  if constexpr (MODE == kFpResid) block_reduce_store<4, kResidMaxMask>(red, b.part, kSlRd2);
}

// ----------------------------------------------------------- backprojector
// One angle for the NV voxels of a warp's row segment.  Voxels are visited in
// increasing detector coordinate (left to right when cos >= 0, right to left
// otherwise); u then never decreases and floor(u) advances by 0 or 1 from one
// voxel to the next (|cos| <= 1), so a two-row window (rows cur and cur + 1,
// ZL values per lane each) slides along the detector and each sinogram row is
// loaded once per angle instead of once per voxel.  Rows off the detector are
// zero.  The taps are the same weights as before; only loads are shared.
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
__device__ __forceinline__ void bp_angle(const Geo<C>& g, const SI* srow, const C* exk, const C* esk,
                                         C eyv, C xf0, C c, C inner, unsigned mask, C (&acc)[NV][ZL]) {
  int cur = -2147483647;
  C tA[ZL], tB[ZL];
#pragma unroll
  for (int i = 0; i < ZL; ++i) { tA[i] = C(0); tB[i] = C(0); }
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const int v = FWD ? q : NV - 1 - q;
    if (!((mask >> v) & 1u)) continue;
    const C u = geo_outer(xf0 + C(v), c, inner);
    C flo;
    int i0;
    floor_split(u, flo, i0);
    const C wv = u - flo;
    const C e = exk ? exk[v] * eyv : C(1);
    C w0 = (C(1) - wv) * e, w1 = wv * e;
    if (esk) {
      w0 = unsigned(i0) < unsigned(g.nd) ? w0 * esk[i0] : C(0);
      w1 = unsigned(i0 + 1) < unsigned(g.nd) ? w1 * esk[i0 + 1] : C(0);
    }
    if (i0 != cur) {
      if (i0 == cur + 1) {
#pragma unroll
        for (int i = 0; i < ZL; ++i) tA[i] = tB[i];
      } else {
        bp_load_row<SI, C, ZL>(g, srow, i0, tA);
      }
      bp_load_row<SI, C, ZL>(g, srow, i0 + 1, tB);
      cur = i0;
    }
#pragma unroll
    for (int i = 0; i < ZL; ++i) acc[v][i] = fma(w1, tB[i], fma(w0, tA[i], acc[v][i]));
  }
}


// Tile: NV voxel columns along x per warp, one row per warp (8 rows per
// block), ZL z values per lane.  need: per (iy, ix) column flag (nullptr:
// every column); columns without it are skipped (and left unwritten in
// kBpStore mode unless need is nullptr).
template <typename SI, typename S, typename C, int ZL, int NV, int MINB, int MODE, typename O>
__global__ void __launch_bounds__(kThreads, MINB)
k_backproject(const Geo<C> g, const SI* __restrict__ sino, const Bufs<S, C> b, O* __restrict__ out,
              const uint8_t* __restrict__ need) {
  if (MODE != kBpStore && b.st->done) return;
  constexpr int ZC = 32 * ZL;
  constexpr int NR = MODE == kBpDualCheck ? kCheckSlots : (MODE == kBpDual ? 2 : 0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntx = (g.nx + NV - 1) / NV, nty = (g.ny + kWarps - 1) / kWarps;
  const int nzc = (g.nz + ZC - 1) / ZC;
  const long long ntiles = (long long)ntx * nty * nzc;
  double red[NR > 0 ? NR : 1] = {};
  StepScalars<C> sc{};
  if (MODE != kBpStore) sc = read_scalars<C>(b.st);

  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int tz = int(t % nzc);
    const long long t1 = t / nzc;
    const int tx = int(t1 % ntx);
    const int ty = int(t1 / ntx);
    const int iy = ty * kWarps + warp;
    const int z0 = tz * ZC + lane * ZL;
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
    if (mask != 0u && z0 < g.nz) {
      const C yf = C(iy) - g.cy;
      const C xf0 = C(tx * NV) - g.cx;
      const SI* sz = sino + z0;
      for (int k = 0; k < g.na; ++k) {
        const C c = g.cs[2 * k], s = g.cs[2 * k + 1];
        const C inner = geo_inner(yf, s, g.off);
        const C eyv = g.ex ? g.ey[(size_t)k * g.ny + iy] : C(1);
        const SI* srow = sz + (size_t)k * g.nd * g.nz;
        const C* exk = g.ex ? g.ex + (size_t)k * g.nx + tx * NV : nullptr;
        const C* esk = g.es ? g.es + (size_t)k * g.nd : nullptr;
        if (c >= C(0))
          bp_angle<SI, C, ZL, NV, true>(g, srow, exk, esk, eyv, xf0, c, inner, mask, acc);
        else
          bp_angle<SI, C, ZL, NV, false>(g, srow, exk, esk, eyv, xf0, c, inner, mask, acc);
      }
    }
    if (z0 >= g.nz) continue;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int ix = tx * NV + v;
      if (ix >= g.nx) continue;
      const size_t base = ((size_t)iy * g.nx + ix) * g.nz + z0;
      if constexpr (MODE == kBpStore) {
        if (need == nullptr || ((mask >> v) & 1u)) store_z<O, C, ZL>(out + base, acc[v]);
      } else if ((mask >> v) & 1u) {
        // the epilogue runs on halves of the z-vector to keep its live range short
        constexpr int H = (ZL % 8 == 0) ? ZL / 2 : ZL;
#pragma unroll
        for (int h0 = 0; h0 < ZL; h0 += H) {
          C part[H];
#pragma unroll
          for (int i = 0; i < H; ++i) part[i] = acc[v][h0 + i];
          dual_update<S, C, H, MODE == kBpDualCheck>(b, sc, base + h0, part, red);
        }
      }
    }
  }
  if constexpr (MODE == kBpDual) block_reduce_store<2>(red, b.part, kSlSBand);
  if constexpr (MODE == kBpDualCheck) block_reduce_store<kCheckSlots, kCheckMaxMask>(red, b.part, kSlRp2);
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
// 2: z, stride 1), zero outside the grid; taps has 2R+1 entries.
template <typename TI, typename TO, typename C>
__global__ void __launch_bounds__(kThreads)
k_conv_axis(const TI* __restrict__ in, TO* __restrict__ out, const C* __restrict__ taps, int R,
            int nx, int ny, int nz, int axis) {
  const long long n = (long long)nx * ny * nz;
  const long long stride = axis == 0 ? nz : (axis == 1 ? (long long)nx * nz : 1);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int z = int(idx % nz);
    const long long r = idx / nz;
    const int ix = int(r % nx);
    const int iy = int(r / nx);
    const int a = axis == 0 ? ix : (axis == 1 ? iy : z);
    const int na = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const int m0 = max(0, R - a), m1 = min(2 * R, na - 1 - a + R);
    C s = C(0);
    for (int m = m0; m <= m1; ++m) s = fma(taps[m], to_c(in[idx + (m - R) * stride]), s);
    out[idx] = from_c<TO>(s);
  }
}

}  // namespace sipo
