// sipo_solver.cuh -- solver state and the per-element PDHG updates.
//
// The LP (general Eqs. 19-24, Case 1 Eqs. 32-37, Case 2 Eqs. 40-45) is solved
// as  min c^T x  s.t.  G x <= h  over x = (y, u~, v~) with up rows on band and
// gel voxels (d_i <= U_i) and lo rows on gel voxels (d_i >= L_i), d = A^T y.
// Iterates: sinogram y >= 0 (0 on masked rays), scalars u~ >= 0 and v~ >= 1
// (implied bounds), duals lam_up (band and gel up rows) and lam_lo (gel lo rows).
//
// One PDHG step T(z) is split over three kernels:
//   scalar step   u+, v+ from the dual sums (Eqs. 48-49 gradients)
//   projector     g = A (lam_up - lam_lo) (Eq. 51), then y+ = max(0, y - tau g)
//   backprojector d_bar = A^T (2 y+ - y), then the dual prox on every row
// and the restarted Halpern iteration z <- w (2 T(z) - z) + (1 - w) z0 is
// fused into the same epilogues.  Every `check_every` iterations the step
// instead writes T(z) to separate buffers (the dual prox then runs in the
// element-wise k_dual<CHECK> with the FP64 check reductions), evaluates its
// KKT error and the infeasibility tests, and a scalar kernel decides
// termination and restarts before blend kernels form the next iterate.
#pragma once

#include <math_constants.h>

#include "sipo_device.cuh"

namespace sipo {

// Reduction slots (each holds kRedBlocks partials).
enum Slot : int {
  kSlSBand = 0,   // sum_band lam_up of the current iterate          (Eq. 48)
  kSlSGel,        // sum_gel f~ lam_up of the current iterate        (Eq. 49)
  // check-step dual update, k_dual<CHECK> (18 slots, contiguous)
  kSlRp2,         // unscaled primal residual^2 of T(z)
  kSlRp2s,        // preconditioned primal residual^2
  kSlDobL,        // sum_gel L lam_lo+          (dual objective)
  kSlDobU,        // sum_gel f~_U lam_up+       (dual objective, Case 1)
  kSlSBandP,      // sum_band lam_up+
  kSlSGelP,       // sum_gel f~ lam_up+
  kSlFpL,         // ||lam - lam+||^2_row       (fixed-point residual, dual part)
  kSlOmL,         // ||lam+ - lam0||^2_row      (primal-weight update)
  kSlFkL,         // Farkas: sum_gel L dlam_lo
  kSlFkBand,      // Farkas: sum_band dlam_up
  kSlFkGel,       // Farkas: sum_gel f~ dlam_up
  kSlFkUp,        // Farkas: sum_gel f~_U dlam_up
  kSlFkNeg,       // Farkas: max(-dlam, 0) (max-reduced)
  kSlFrL,         // same five for the fixed-point residual direction dlam = lam+ - lam
  kSlFrBand,
  kSlFrGel,
  kSlFrUp,
  kSlFrNeg,
  // projector, check step
  kSlFpX,         // ||y - y+||^2_col
  kSlOmX,         // ||y+ - y0||^2_col
  // projector on q+ (dual residual of T(z))
  kSlRd2,         // ||min(g+, 0)||^2 on active rays
  kSlRd2s,        // preconditioned
  kSlFkG,         // Farkas: max(-(g+ - g0), 0) on active rays (max-reduced)
  kSlFrG,         // Farkas: max(-(g+ - g), 0) on active rays (residual direction, max-reduced)
  // bound-based certificate of the epoch difference (check step)
  kSlCertObj,     // dual objective of the projected candidate
  kSlCertK,       // max over active rays of max(-g^, 0) / b (max-reduced)
  kNumSlots
};

// FP64 scalar state of one solve (device memory, one per context).
struct Scal {
  // problem constants
  double c_u, c_v, band_rhs, col_u, col_v, h_norm, c_norm, kkt_tol;
  int has_u, has_v;
  long long max_iter;
  // scalar iterates
  double u, v, u0, v0, up, vp, ubar, vbar;
  double omega, w;
  long long k, k_in;
  double r0, r_prev;
  int r0_set, done, status, restart, restarts, pad;
  // KKT data of the last check
  double kkt, rel_p, rel_d, rel_gap, rp, rd, pobj, dobj, gap, sband_p, sgel_p;
  // per-check trace: kTraceFields doubles per entry, up to trace_cap entries
  double* trace;
  int trace_cap, trace_n;
  // bound-based infeasibility certificate: B, whether the case has one, and
  // the decision of the current check; cert_slices: evaluated per z-slice
  // (operator without z coupling), cert_z: first slice that carried it (-1)
  double cert_B;
  int cert_on, cert;
  int cert_slices, cert_z;
  // a check found a non-finite residual or objective (the solve stops)
  int numeric, pad2;
};

// Margin of the bound-based certificate: kappa * B <= (1 - kCertMargin) obj.
constexpr double kCertMargin = 1e-3;

// k, kkt, rel_primal, rel_dual, rel_gap, pobj, omega, restarts, and the
// relative violations of the two Farkas candidates (epoch difference, residual
// direction; -1 when the candidate's dual objective is not positive)
constexpr int kTraceFields = 10;
constexpr int kCheckSlots = kSlFpX - kSlRp2;  // check-step dual-update slots
// max-reduced slots among them (Farkas negativity, l_inf) and among the
// projector residual slots (kSlRd2 .. kSlFrG)
constexpr unsigned kCheckMaxMask = (1u << (kSlFkNeg - kSlRp2)) | (1u << (kSlFrNeg - kSlRp2));
constexpr unsigned kResidMaxMask = (1u << (kSlFkG - kSlRd2)) | (1u << (kSlFrG - kSlRd2));

// Device arrays of one solve.  S: storage type of iterates, C: compute type.
template <typename S, typename C>
struct Bufs {
  // sinogram-sized
  S *y, *y0, *yp, *ybar;
  const C* col;         // Pock-Chambolle column abs-sum of each ray (0: masked)
  C *gp, *g0;           // A q+ at the last check / at the last restart
  C* gc;                // A q of the current iterate at the last check
  // volume-sized
  S *lu, *ll, *lu0, *ll0, *lpu, *lpl, *q, *qp;
  C *d, *d0, *dp;       // A^T y (current, anchor, T point) on band and gel
  const C* row;         // A^T 1_act (row abs-sum of A^T over active rays)
  const C* ft;          // normalised lower profile f~ (nullptr: ft_const)
  const uint8_t* lab;   // region labels
  C ft_const;
  C up_ratio;           // Case 1: f~_U / f~_L when fu is null
  const C* fu;          // Case 1: explicit upper profile f~_U per voxel (nullptr: f~ up_ratio)
  int has_u, has_v;
  C band_rhs;           // right side of band rows: 0 (u~ variable) or 1 (Case 2)
  Scal* st;
  double* part;
  // bound-based certificate: b = A 1_rows per ray, the candidate volume,
  // and per z-slice the largest max(-g^, 0) / b as ordered bits (slice mode)
  const C* cert_b;
  C* cert_q;
  unsigned long long* cert_kz;
};

// Halpern weights and steps read once per kernel.
template <typename C>
struct StepScalars {
  C omega, w, ubar, vbar, up, vp;
};

template <typename C>
__device__ __forceinline__ StepScalars<C> read_scalars(const Scal* st) {
  StepScalars<C> s;
  s.omega = C(st->omega);
  s.w = C(st->w);
  s.ubar = C(st->ubar);
  s.vbar = C(st->vbar);
  s.up = C(st->up);
  s.vp = C(st->vp);
  return s;
}

template <typename S, typename C>
__device__ __forceinline__ C rnd(C x) {  // value after a round trip through S
  return to_c(from_c<S>(x));
}

// ------------------------------------------------------------- dual update
// One z-vector of voxels.  CHECK = false: Halpern step fused (writes the next
// iterate and the dual sums of Eqs. 48-49).  CHECK = true: writes T(z) and
// accumulates its residuals, objective pieces and restart distances.
// Reduction accumulators: red[0..1] normal, red[0..kCheckSlots) check.
template <typename S, typename C, int ZL, bool CHECK>
__device__ __forceinline__ void dual_update(const Bufs<S, C>& b, const StepScalars<C>& sc,
                                            size_t base, const C (&dbar)[ZL],
                                            double* red) {
  uint8_t lab[ZL];
  load_labels<C, ZL>(b.lab + base, lab);
  bool any = false;
#pragma unroll
  for (int i = 0; i < ZL; ++i) any |= (lab[i] != kExt);
  if (!any) return;

  C ft[ZL], row[ZL], lu[ZL], ll[ZL], lu0[ZL], ll0[ZL];
  if (b.ft) load_z<C, C, ZL>(b.ft + base, ft);
  else {
#pragma unroll
    for (int i = 0; i < ZL; ++i) ft[i] = b.ft_const;
  }
  load_z<C, C, ZL>(b.row + base, row);
  load_z<S, C, ZL>(b.lu + base, lu);
  load_z<S, C, ZL>(b.ll + base, ll);
  load_z<S, C, ZL>(b.lu0 + base, lu0);
  load_z<S, C, ZL>(b.ll0 + base, ll0);
  const C eo = C(kEta) * sc.omega;
  const C w = sc.w;
  C o_lu[ZL], o_ll[ZL], o_q[ZL], o_d[ZL];
  C dcur[ZL], d0[ZL];
  // sums of this z-vector in the compute type, added to the FP64
  // accumulators once per vector below (in FP32 a sum of ZL terms is within
  // ~ZL ulp; FP64 arithmetic per voxel is slow on this part)
  C acc[CHECK ? kCheckSlots : 2] = {};
  if constexpr (CHECK) load_z<C, C, ZL>(b.d + base, dcur);
  else load_z<C, C, ZL>(b.d0 + base, d0);
#pragma unroll
  for (int i = 0; i < ZL; ++i) {
    const bool band = lab[i] == kBand, gel = lab[i] == kGel;
    if (!band && !gel) {
      o_lu[i] = C(0); o_ll[i] = C(0); o_q[i] = C(0);
      o_d[i] = CHECK ? dcur[i] : d0[i];
      continue;
    }
    const C f = ft[i];
    // constant upper bound of a Case-1 gel row (0 where v~ moves the bound)
    const C fU = (b.has_v || band) ? C(0) : (b.fu ? b.fu[base + z_offset<C, ZL>(i)] : f * b.up_ratio);
    const C extra = band ? (b.has_u ? C(1) : C(0)) : (b.has_v ? f : C(0));
    const C rup = row[i] + extra;
    const C sig_up = rup > C(0) ? eo / rup : C(0);
    const C Ubar = band ? (b.has_u ? sc.ubar : b.band_rhs) : (b.has_v ? sc.vbar * f : fU);
    C lup = lu[i] + sig_up * (dbar[i] - Ubar);
    lup = rnd<S, C>(lup > C(0) ? lup : C(0));
    C llp = C(0);
    if (gel) {
      const C sig_lo = row[i] > C(0) ? eo / row[i] : C(0);
      llp = ll[i] + sig_lo * (f - dbar[i]);
      llp = rnd<S, C>(llp > C(0) ? llp : C(0));
    }
    if constexpr (!CHECK) {
      C lun = rnd<S, C>(w * (C(2) * lup - lu[i]) + (C(1) - w) * lu0[i]);
      C lln = gel ? rnd<S, C>(w * (C(2) * llp - ll[i]) + (C(1) - w) * ll0[i]) : C(0);
      o_lu[i] = lun;
      o_ll[i] = lln;
      o_q[i] = lun - lln;
      o_d[i] = w * dbar[i] + (C(1) - w) * d0[i];
      if (band) acc[0] += lun;
      else acc[1] += f * lun;
    } else {
      const C dp = C(0.5) * (dbar[i] + dcur[i]);
      o_lu[i] = lup;
      o_ll[i] = llp;
      o_q[i] = lup - llp;
      o_d[i] = dp;
      const C Ucur = band ? (b.has_u ? sc.up : b.band_rhs) : (b.has_v ? sc.vp * f : fU);
      const C eu = dp > Ucur ? dp - Ucur : C(0);
      acc[0] += eu * eu;
      if (rup > C(0)) acc[1] += eu * eu / rup;
      const C dlu = lup - lu0[i];
      const C du = lu[i] - lup;
      acc[6] += rup * du * du;
      acc[7] += rup * dlu * dlu;
      acc[12] = acc[12] > -dlu ? acc[12] : -dlu;
      if (band) {
        acc[4] += lup;
        acc[9] += dlu;
      } else {
        const C el = f > dp ? f - dp : C(0);
        acc[0] += el * el;
        if (row[i] > C(0)) acc[1] += el * el / row[i];
        const C dll = llp - ll0[i];
        const C dl = ll[i] - llp;
        acc[2] += f * llp;
        acc[3] += fU * lup;
        acc[5] += f * lup;
        acc[6] += row[i] * dl * dl;
        acc[7] += row[i] * dll * dll;
        acc[8] += f * dll;
        acc[10] += f * dlu;
        acc[11] += fU * dlu;
        acc[12] = acc[12] > -dll ? acc[12] : -dll;
        const C rl = llp - ll[i];
        acc[13] += f * rl;
        acc[15] += f * (lup - lu[i]);
        acc[16] += fU * (lup - lu[i]);
        acc[17] = acc[17] > -rl ? acc[17] : -rl;
      }
      const C ru = lup - lu[i];
      if (band) acc[14] += ru;
      acc[17] = acc[17] > -ru ? acc[17] : -ru;
    }
  }
  if constexpr (CHECK) {
#pragma unroll
    for (int j = 0; j < kCheckSlots; ++j) {
      if ((kCheckMaxMask >> j) & 1u) red[j] = fmax(red[j], double(acc[j]));
      else red[j] += double(acc[j]);
    }
  } else {
    red[0] += double(acc[0]);
    red[1] += double(acc[1]);
  }
  if constexpr (!CHECK) {
    store_z<S, C, ZL>(b.lu + base, o_lu);
    store_z<S, C, ZL>(b.ll + base, o_ll);
    store_z<S, C, ZL>(b.q + base, o_q);
    store_z<C, C, ZL>(b.d + base, o_d);
  } else {
    store_z<S, C, ZL>(b.lpu + base, o_lu);
    store_z<S, C, ZL>(b.lpl + base, o_ll);
    store_z<S, C, ZL>(b.qp + base, o_q);
    store_z<C, C, ZL>(b.dp + base, o_d);
  }
}

// ----------------------------------------------------------- primal update
// One z-vector of rays with g = A q already formed.  CHECK = false: Halpern
// step fused; CHECK = true: writes y+ and the restart distances (red[0..1]).
template <typename S, typename C, int ZL, bool CHECK>
__device__ __forceinline__ void primal_update(const Bufs<S, C>& b, const StepScalars<C>& sc,
                                              size_t base, const C (&g)[ZL], double* red) {
  C col[ZL], y[ZL], y0[ZL], yb[ZL], yo[ZL];
  load_z<C, C, ZL>(b.col + base, col);
  bool any = false;
#pragma unroll
  for (int i = 0; i < ZL; ++i) any |= col[i] > C(0);
  if (!any) return;  // every ray of the vector is masked: y, y_bar stay 0
  load_z<S, C, ZL>(b.y + base, y);
  load_z<S, C, ZL>(b.y0 + base, y0);
  const C w = sc.w;
  C a0 = C(0), a1 = C(0);  // restart distances of this z-vector (compute type)
#pragma unroll
  for (int i = 0; i < ZL; ++i) {
    const C tau = col[i] > C(0) ? C(kEta) / (sc.omega * col[i]) : C(0);
    C yp = y[i] - tau * g[i];
    yp = rnd<S, C>(yp > C(0) ? yp : C(0));
    yb[i] = rnd<S, C>(C(2) * yp - y[i]);
    if constexpr (!CHECK) {
      yo[i] = w * yb[i] + (C(1) - w) * y0[i];
    } else {
      yo[i] = yp;
      const C dx = y[i] - yp, dz = yp - y0[i];
      a0 += col[i] * dx * dx;
      a1 += col[i] * dz * dz;
    }
  }
  if constexpr (CHECK) {
    red[0] += double(a0);
    red[1] += double(a1);
  }
  store_z<S, C, ZL>(b.ybar + base, yb);
  if constexpr (!CHECK) {
    store_z<S, C, ZL>(b.y + base, yo);
  } else {
    store_z<S, C, ZL>(b.yp + base, yo);
    store_z<C, C, ZL>(b.gc + base, g);
  }
}

// Bound-based certificate: largest max(-g^, 0) / b over active rays (red[0];
// +inf where a violated ray has b = 0).
template <typename S, typename C, int ZL>
__device__ __forceinline__ void cert_update(const Bufs<S, C>& b, size_t base, const C (&g)[ZL], double* red) {
  C col[ZL], bb[ZL];
  load_z<C, C, ZL>(b.col + base, col);
  load_z<C, C, ZL>(b.cert_b + base, bb);
#pragma unroll
  for (int i = 0; i < ZL; ++i) {
    if (col[i] > C(0) && g[i] < C(0)) {
      // the ratio in the compute type (its rounding is far inside the
      // certificate's relative margin; FP64 division is slow on this part)
      red[0] = fmax(red[0], bb[i] > C(0) ? double(-g[i] / bb[i]) : CUDART_INF);
    }
  }
}

// Slice mode: the same ratio per z value, folded with an atomic maximum into
// the block's shared array kz[nz] (the bit patterns of non-negative doubles,
// +inf included, order like the values, so the maximum does not depend on
// the order of the updates).
template <typename S, typename C, int ZL>
__device__ __forceinline__ void cert_update_z(const Bufs<S, C>& b, size_t base, int z0, const C (&g)[ZL],
                                              unsigned long long* kz) {
  C col[ZL], bb[ZL];
  load_z<C, C, ZL>(b.col + base, col);
  load_z<C, C, ZL>(b.cert_b + base, bb);
#pragma unroll
  for (int i = 0; i < ZL; ++i) {
    if (col[i] > C(0) && g[i] < C(0)) {
      const double v = bb[i] > C(0) ? double(-g[i] / bb[i]) : CUDART_INF;
      atomicMax(kz + z0 + z_offset<C, ZL>(i), (unsigned long long)__double_as_longlong(v));
    }
  }
}

// Dual residual of T(z) on active rays from g+ = A q+ (red[0..3]).
template <typename S, typename C, int ZL>
__device__ __forceinline__ void resid_update(const Bufs<S, C>& b, size_t base, const C (&g)[ZL],
                                             double* red) {
  C col[ZL], g0[ZL], gc[ZL];
  load_z<C, C, ZL>(b.col + base, col);
  load_z<C, C, ZL>(b.g0 + base, g0);
  load_z<C, C, ZL>(b.gc + base, gc);
  // sums of one z-vector in the compute type, folded into FP64 once per
  // vector (as in the check-step dual update)
  C a0 = C(0), a1 = C(0), a2 = -CUDART_INF_F, a3 = -CUDART_INF_F;
#pragma unroll
  for (int i = 0; i < ZL; ++i) {
    if (col[i] > C(0)) {
      const C m = g[i] < C(0) ? g[i] : C(0);
      a0 += m * m;
      a1 += m * m / col[i];
      const C d0 = g0[i] - g[i], dc = gc[i] - g[i];
      a2 = a2 > d0 ? a2 : d0;
      a3 = a3 > dc ? a3 : dc;
    }
  }
  red[0] += double(a0);
  red[1] += double(a1);
  red[2] = fmax(red[2], double(a2));
  red[3] = fmax(red[3], double(a3));
  store_z<C, C, ZL>(b.gp + base, g);
}

}  // namespace sipo
