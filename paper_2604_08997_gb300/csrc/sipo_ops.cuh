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

constexpr int kBpTile = 8;  // backprojector voxel tile: 8 x 8 columns, one row per warp

// --------------------------------------------------------------- projector
// SI: element type read from `vol`; O: element type written by kFpStore.
template <typename SI, typename S, typename C, int ZL, int MODE, typename O>
__global__ void __launch_bounds__(kThreads)
k_project(const Geo<C> g, const SI* __restrict__ vol, const Bufs<S, C> b, O* __restrict__ out,
          const uint8_t* __restrict__ act_col) {
  if (MODE != kFpStore && b.st->done) return;
  constexpr int ZC = 32 * ZL;
  constexpr int NR = MODE == kFpPrimalCheck ? 2 : (MODE == kFpResid ? 3 : 0);
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
    if (esj != C(0)) {
      const C c = g.cs[2 * k], s = g.cs[2 * k + 1];
      const C sj = C(j) - g.off;
      C H = C(0);
      if (g.r2q > 0.0) {
        C a = fabs(sj) - C(1.5);
        a = a > C(0) ? a : C(0);
        const C R = C(g.vial_r);
        H = R * R - a * a;
        H = (H > C(0) ? sqrt(H) : C(0)) + C(1.5);
      }
      if (fabs(c) >= fabs(s)) {
        // walk rows; on row iy the bin is reached from x near (j - inner)/c
        int lo = 0, hi = g.ny - 1;
        if (g.r2q > 0.0) {
          const C yc = sj * s, hy = fabs(c) * H + C(1);
          lo = max(0, int(fl_(yc - hy + g.cy)));
          hi = min(g.ny - 1, int(ceil(yc + hy + g.cy)));
        }
        const C inv_c = C(1) / c, h = C(1) / fabs(c);
        for (int iy = lo; iy <= hi; ++iy) {
          const C yf = C(iy) - g.cy;
          const C inner = geo_inner(yf, s, g.off);
          const C eyv = g.ex ? g.ey[(size_t)k * g.ny + iy] : C(1);
          const C ixc = (C(j) - inner) * inv_c + g.cx;
          const int ixa = int(fl_(ixc - h)) - 1;
#pragma unroll
          for (int m = 0; m < 5; ++m) {
            const int ix = ixa + m;
            if (ix < 0 || ix >= g.nx) continue;
            const C xf = C(ix) - g.cx;
            const C u = geo_outer(xf, c, inner);
            const C flo = fl_(u);
            const int i0 = int(flo);
            const C wv = u - flo;
            C wt = (i0 == j) ? (C(1) - wv) : ((i0 + 1 == j) ? wv : C(0));
            if (wt == C(0)) continue;
            if (!in_vial(g, ix, iy)) continue;
            if (g.ex) wt = wt * (g.ex[(size_t)k * g.nx + ix] * eyv);
            if (z0 < g.nz) {
              C v[ZL];
              load_z<SI, C, ZL>(vol + ((size_t)iy * g.nx + ix) * g.nz + z0, v);
#pragma unroll
              for (int i = 0; i < ZL; ++i) acc[i] = fma(wt, v[i], acc[i]);
            }
          }
        }
      } else {
        // walk columns; on column ix the bin is reached from y near (j - off - x c)/s
        int lo = 0, hi = g.nx - 1;
        if (g.r2q > 0.0) {
          const C xc = sj * c, hx = fabs(s) * H + C(1);
          lo = max(0, int(fl_(xc - hx + g.cx)));
          hi = min(g.nx - 1, int(ceil(xc + hx + g.cx)));
        }
        const C inv_s = C(1) / s, h = C(1) / fabs(s);
        for (int ix = lo; ix <= hi; ++ix) {
          const C xf = C(ix) - g.cx;
          const C exv = g.ex ? g.ex[(size_t)k * g.nx + ix] : C(1);
          const C iyc = (C(j) - g.off - xf * c) * inv_s + g.cy;
          const int iya = int(fl_(iyc - h)) - 1;
#pragma unroll
          for (int m = 0; m < 5; ++m) {
            const int iy = iya + m;
            if (iy < 0 || iy >= g.ny) continue;
            const C yf = C(iy) - g.cy;
            const C u = geo_outer(xf, c, geo_inner(yf, s, g.off));
            const C flo = fl_(u);
            const int i0 = int(flo);
            const C wv = u - flo;
            C wt = (i0 == j) ? (C(1) - wv) : ((i0 + 1 == j) ? wv : C(0));
            if (wt == C(0)) continue;
            if (!in_vial(g, ix, iy)) continue;
            if (g.ex) wt = wt * (exv * g.ey[(size_t)k * g.ny + iy]);
            if (z0 < g.nz) {
              C v[ZL];
              load_z<SI, C, ZL>(vol + ((size_t)iy * g.nx + ix) * g.nz + z0, v);
#pragma unroll
              for (int i = 0; i < ZL; ++i) acc[i] = fma(wt, v[i], acc[i]);
            }
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
  if constexpr (MODE == kFpResid) block_reduce_store<3>(red, b.part, kSlRd2);
}

// ----------------------------------------------------------- backprojector
// need: per (iy, ix) column flag (nullptr: every column); columns without it
// are skipped (and left unwritten in kBpStore mode unless need is nullptr).
template <typename SI, typename S, typename C, int ZL, int MODE, typename O>
__global__ void __launch_bounds__(kThreads)
k_backproject(const Geo<C> g, const SI* __restrict__ sino, const Bufs<S, C> b, O* __restrict__ out,
              const uint8_t* __restrict__ need) {
  if (MODE != kBpStore && b.st->done) return;
  constexpr int ZC = 32 * ZL;
  constexpr int NV = kBpTile;
  constexpr int NR = MODE == kBpDualCheck ? 13 : (MODE == kBpDual ? 2 : 0);
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
    unsigned mask = 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int ix = tx * NV + v;
      if (ix < g.nx && in_vial(g, ix, iy) && (need == nullptr || need[(size_t)iy * g.nx + ix]))
        mask |= 1u << v;
    }
    C acc[NV][ZL];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int i = 0; i < ZL; ++i) acc[v][i] = C(0);
    if (mask != 0u && z0 < g.nz) {
      const C yf = C(iy) - g.cy;
      for (int k = 0; k < g.na; ++k) {
        const C c = g.cs[2 * k], s = g.cs[2 * k + 1];
        const C inner = geo_inner(yf, s, g.off);
        const C eyv = g.ex ? g.ey[(size_t)k * g.ny + iy] : C(1);
        const SI* srow = sino + (size_t)k * g.nd * g.nz + z0;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (!((mask >> v) & 1u)) continue;
          const int ix = tx * NV + v;
          const C xf = C(ix) - g.cx;
          const C u = geo_outer(xf, c, inner);
          const C flo = fl_(u);
          const int i0 = int(flo);
          const C wv = u - flo;
          const C e = g.ex ? g.ex[(size_t)k * g.nx + ix] * eyv : C(1);
          C w0 = (C(1) - wv) * e, w1 = wv * e;
          const bool ok0 = unsigned(i0) < unsigned(g.nd);
          const bool ok1 = unsigned(i0 + 1) < unsigned(g.nd);
          if (g.es) {
            w0 = ok0 ? w0 * g.es[(size_t)k * g.nd + i0] : C(0);
            w1 = ok1 ? w1 * g.es[(size_t)k * g.nd + i0 + 1] : C(0);
          }
          if (ok0) {
            C tv[ZL];
            load_z<SI, C, ZL>(srow + (size_t)i0 * g.nz, tv);
#pragma unroll
            for (int i = 0; i < ZL; ++i) acc[v][i] = fma(w0, tv[i], acc[v][i]);
          }
          if (ok1) {
            C tv[ZL];
            load_z<SI, C, ZL>(srow + (size_t)(i0 + 1) * g.nz, tv);
#pragma unroll
            for (int i = 0; i < ZL; ++i) acc[v][i] = fma(w1, tv[i], acc[v][i]);
          }
        }
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
      } else {
        if ((mask >> v) & 1u) dual_update<S, C, ZL, MODE == kBpDualCheck>(b, sc, base, acc[v], red);
      }
    }
  }
  if constexpr (MODE == kBpDual) block_reduce_store<2>(red, b.part, kSlSBand);
  if constexpr (MODE == kBpDualCheck) block_reduce_store<13>(red, b.part, kSlRp2);
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
