// sipo_kernels.cuh -- setup, scalar, blend and post-solve kernels.
//
// Setup builds the domain partition of Sec. 2.2 (Fig. 2) with exact integer
// logic: gel = {f_T != 0}; band = non-gel voxels within Euclidean distance
// <= W of the gel (a windowed squared-distance transform, three separable
// passes that are exact for every distance <= W) or inside the support of
// K f_T (a box dilation by the PSF radii); exterior otherwise or outside the
// vial.  The scalar kernels carry the FP64 logic of the restarted Halpern
// PDHG (step sizes, u~/v~ updates of Eqs. 48-49, KKT of Sec. 6.1, restarts,
// primal weight, infeasibility test).
#pragma once

#include "sipo_solver.cuh"

namespace sipo {

constexpr double kBetaSufficient = 0.2;
constexpr double kBetaNecessary = 0.8;
constexpr double kBetaArtificial = 0.36;
constexpr double kOmegaSmoothing = 0.5;
constexpr double kInfeasTol = 1e-6;
constexpr int kDistInf = 0x3fffffff;

// ------------------------------------------------------------ target stats
struct TargetStats {
  unsigned long long n_gel, n_bad;
  unsigned int min_bits, max_bits;  // float bit patterns of non-negative values
};

__global__ void k_target_stats(const float* __restrict__ f, long long n, TargetStats* out) {
  unsigned long long gel = 0, bad = 0;
  unsigned int mn = 0x7f800000u, mx = 0u;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = f[i];
    if (!(v >= 0.0f) || isinf(v)) { ++bad; continue; }   // NaN, negative or infinite
    if (v != 0.0f) {
      ++gel;
      const unsigned int b = __float_as_uint(v);
      mn = min(mn, b);
      mx = max(mx, b);
    }
  }
  atomicAdd(&out->n_gel, gel);
  atomicAdd(&out->n_bad, bad);
  atomicMin(&out->min_bits, mn);
  atomicMax(&out->max_bits, mx);
}

// Explicit Case-1 bounds: over the gel voxels (f_T > 0) counts those whose
// lower bound is not positive and finite or whose upper bound is below it or
// not finite, and the float bit range of the lower bound (for f_crit).
__global__ void k_bound_stats(const float* __restrict__ fT, const float* __restrict__ fL,
                              const float* __restrict__ fU, long long n, TargetStats* out) {
  unsigned long long bad = 0;
  unsigned int mn = 0x7f800000u, mx = 0u;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (!(fT[i] > 0.0f)) continue;
    const float lo = fL[i], hi = fU[i];
    if (!(lo > 0.0f) || isinf(lo) || !(hi >= lo) || isinf(hi)) { ++bad; continue; }
    const unsigned int b = __float_as_uint(lo);
    mn = min(mn, b);
    mx = max(mx, b);
  }
  atomicAdd(&out->n_bad, bad);
  atomicMin(&out->min_bits, mn);
  atomicMax(&out->max_bits, mx);
}

// ----------------------------------------------------------------- labels
// dist0[v] = 0 on gel, kDistInf elsewhere.
__global__ void k_gel_init(const float* __restrict__ f, long long n, int* __restrict__ dist,
                           uint8_t* __restrict__ lab) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const bool gel = f[i] != 0.0f;
    dist[i] = gel ? 0 : kDistInf;
    lab[i] = gel ? kGel : kExt;
  }
}

// One separable pass of the windowed squared distance:
// out[i] = min_{|m| <= W} (m^2 + in[i + m*stride]) along `axis`.  After the x,
// y and z passes, out = min over gel voxels of the squared Euclidean distance
// whenever that distance is <= W (larger distances stay > W^2).
__global__ void k_dist_pass(const int* __restrict__ in, int* __restrict__ out, int W, int nx,
                            int ny, int nz, int axis) {
  const long long n = (long long)nx * ny * nz;
  const long long stride = axis == 0 ? nz : (axis == 1 ? (long long)nx * nz : 1);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int z = int(idx % nz);
    const long long r = idx / nz;
    const int ix = int(r % nx), iy = int(r / nx);
    const int a = axis == 0 ? ix : (axis == 1 ? iy : z);
    const int na = axis == 0 ? nx : (axis == 1 ? ny : nz);
    int best = kDistInf;
    for (int m = max(-W, -a); m <= min(W, na - 1 - a); ++m) {
      const int v = in[idx + m * stride];
      if (v < kDistInf) best = min(best, v + m * m);
    }
    out[idx] = best;
  }
}

// Box dilation pass: out[i] = any(in[i + m*stride]), |m| <= R.
__global__ void k_dilate_pass(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int R,
                              int nx, int ny, int nz, int axis) {
  const long long n = (long long)nx * ny * nz;
  const long long stride = axis == 0 ? nz : (axis == 1 ? (long long)nx * nz : 1);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int z = int(idx % nz);
    const long long r = idx / nz;
    const int ix = int(r % nx), iy = int(r / nx);
    const int a = axis == 0 ? ix : (axis == 1 ? iy : z);
    const int na = axis == 0 ? nx : (axis == 1 ? ny : nz);
    uint8_t any = 0;
    for (int m = max(-R, -a); m <= min(R, na - 1 - a); ++m) any |= in[idx + m * stride];
    out[idx] = any ? 1 : 0;
  }
}

__global__ void k_gel_mask(const uint8_t* __restrict__ lab, uint8_t* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = lab[i] == kGel ? 1 : 0;
}

// Final labels: band = non-gel & (dist^2 <= W^2 | psf support | band-free),
// inside the vial.
template <typename C>
__global__ void k_labels_final(uint8_t* __restrict__ lab, const int* __restrict__ dist,
                               const uint8_t* __restrict__ psf_sup, int W, int band_free,
                               Geo<C> g) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    if (lab[idx] == kGel) continue;
    const long long r = idx / g.nz;
    const int ix = int(r % g.nx), iy = int(r / g.nx);
    bool band = band_free != 0;
    if (!band && W >= 0 && dist[idx] <= W * W) band = true;
    if (!band && psf_sup != nullptr && psf_sup[idx]) band = true;
    lab[idx] = (band && in_vial(g, ix, iy)) ? kBand : kExt;
  }
}

// Column flag: any non-exterior voxel along z of (iy, ix).
__global__ void k_need_cols(const uint8_t* __restrict__ lab, uint8_t* __restrict__ need, int nx,
                            int ny, int nz) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < (long long)nx * ny;
       c += (long long)gridDim.x * blockDim.x) {
    uint8_t any = 0;
    for (int z = 0; z < nz; ++z) any |= lab[c * nz + z] != kExt;
    need[c] = any;
  }
}

// 2-D box dilation of a column flag (PSF reach in x and y).
__global__ void k_dilate_cols(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int nx,
                              int ny, int Rx, int Ry) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < (long long)nx * ny;
       c += (long long)gridDim.x * blockDim.x) {
    const int ix = int(c % nx), iy = int(c / nx);
    uint8_t any = 0;
    for (int a = max(0, iy - Ry); a <= min(ny - 1, iy + Ry) && !any; ++a)
      for (int b = max(0, ix - Rx); b <= min(nx - 1, ix + Rx); ++b) any |= in[(size_t)a * nx + b];
    out[c] = any;
  }
}

// Normalised lower profile f~ on gel (Sec. 2.5, Eq. 31, Eq. 39).
template <typename C>
__global__ void k_ft(const float* __restrict__ f, const uint8_t* __restrict__ lab, double mult,
                     C* __restrict__ ft, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    ft[i] = lab[i] == kGel ? C(double(f[i]) * mult) : C(0);
}

template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ in, TO* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = from_c<TO>(to_c(in[i]));
}

// A caller's primal point times `scale` (> 0) projected onto the primal
// domain of Eqs. 23-24: y >= 0 on active rays (positive column sum), 0 on the
// others.  A NaN fails the comparison and is dropped like a negative value.
template <typename S, typename C>
__global__ void k_import_primal(const C* __restrict__ in, const C* __restrict__ col, S* __restrict__ out,
                                C scale, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const C v = in[i] * scale;
    out[i] = from_c<S>(col[i] > C(0) && v > C(0) ? v : C(0));
  }
}

// A caller's dual point projected onto the dual domain: lam_up >= 0 on band
// and gel rows, lam_lo >= 0 on gel rows, 0 elsewhere (Eqs. 20-22); stored in
// the iterate type, and q = lam_up - lam_lo of the stored values in C.
template <typename S, typename C>
__global__ void k_import_dual(const C* __restrict__ in_up, const C* __restrict__ in_lo,
                              const uint8_t* __restrict__ lab, S* __restrict__ up, S* __restrict__ lo,
                              C* __restrict__ q, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint8_t l = lab[i];
    const C a = in_up[i], b = in_lo[i];
    const S su = from_c<S>(l != kExt && a > C(0) ? a : C(0));
    const S sl = from_c<S>(l == kGel && b > C(0) ? b : C(0));
    up[i] = su;
    lo[i] = sl;
    q[i] = to_c(su) - to_c(sl);
  }
}

// Indicator volume 1_band + 2 * 1_gel (column abs-sums of G, Pock-Chambolle).
template <typename C>
__global__ void k_row_indicator(const uint8_t* __restrict__ lab, C* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = lab[i] == kGel ? C(2) : (lab[i] == kBand ? C(1) : C(0));
}

// Active rays: mask = [P f_T] > 0; ones = mask as C; per (angle, bin) flag.
template <typename C>
__global__ void k_mask(const C* __restrict__ pf, uint8_t* __restrict__ mask, C* __restrict__ ones,
                       long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const bool a = pf[i] > C(0);
    mask[i] = a ? 1 : 0;
    ones[i] = a ? C(1) : C(0);
  }
}

__global__ void k_act_cols(const uint8_t* __restrict__ mask, uint8_t* __restrict__ act, long long nrays,
                           int nz) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrays;
       r += (long long)gridDim.x * blockDim.x) {
    uint8_t any = 0;
    for (int z = 0; z < nz; ++z) any |= mask[r * nz + z];
    act[r] = any;
  }
}

template <typename C>
__global__ void k_apply_mask(C* __restrict__ col, const uint8_t* __restrict__ mask, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!mask[i]) col[i] = C(0);
}

// Setup sums (FP64 partials per block, summed on the host):
// 0 |band|, 1 |gel|, 2 sum_gel f~, 3 sum_gel f~^2, 4 sum_gel f~_U^2,
// 5 sum U0^2 / row_up over up rows, 6 sum_gel f~^2 / row_lo, 7 sum_gel f~_U,
// with f~_U the Case-1 upper profile (fu, or f~ up_ratio when fu is null).
template <typename C>
__global__ void k_setup_sums(const uint8_t* __restrict__ lab, const C* __restrict__ ft, C ft_const,
                             const C* __restrict__ fu, const C* __restrict__ row, double up_ratio, int has_u,
                             int has_v, int kase, long long n, double* __restrict__ part) {
  double v[8] = {};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint8_t l = lab[i];
    if (l == kExt) continue;
    const double f = ft ? double(ft[i]) : double(ft_const);
    const double r = double(row[i]);
    if (l == kBand) {
      v[0] += 1.0;
      const double rup = r + (has_u ? 1.0 : 0.0);
      const double U0 = has_u ? 0.0 : 1.0;
      if (rup > 0) v[5] += U0 * U0 / rup;
    } else {
      v[1] += 1.0;
      v[2] += f;
      v[3] += f * f;
      const double fU = fu ? double(fu[i]) : f * up_ratio;
      v[4] += fU * fU;
      v[7] += fU;
      const double rup = r + (has_v ? f : 0.0);
      const double U0 = has_v ? 0.0 : fU;
      if (rup > 0) v[5] += U0 * U0 / rup;
      if (r > 0) v[6] += f * f / r;
    }
  }
  (void)kase;
  block_reduce_store<8>(v, part, 0);
}

// ---------------------------------------------------------- scalar kernels
// One block.  Gradient step of the scalars from the dual sums (Eqs. 48-49),
// extrapolation, Halpern weight; outside check steps also the Halpern blend.
template <bool CHECK>
__global__ void __launch_bounds__(kThreads) k_scalar_step(Scal* st, const double* part) {
  if (st->done) return;
  const double Sb = block_sum_slot(part, kSlSBand);
  const double Sg = block_sum_slot(part, kSlSGel);
  if (threadIdx.x != 0) return;
  const double om = st->omega;
  double up = st->u, vp = st->v;
  if (st->has_u && st->col_u > 0) {
    up = st->u - kEta / (om * st->col_u) * (st->c_u - Sb);
    if (up < 0.0) up = 0.0;
  }
  if (st->has_v && st->col_v > 0) {
    vp = st->v - kEta / (om * st->col_v) * (st->c_v - Sg);
    if (vp < 1.0) vp = 1.0;
  }
  st->up = up;
  st->vp = vp;
  st->ubar = 2.0 * up - st->u;
  st->vbar = 2.0 * vp - st->v;
  const double w = (double(st->k_in) + 1.0) / (double(st->k_in) + 2.0);
  st->w = w;
  if (!CHECK) {
    st->u = w * st->ubar + (1.0 - w) * st->u0;
    st->v = w * st->vbar + (1.0 - w) * st->v0;
    st->k_in += 1;
    st->k += 1;
  }
}

// One block.  KKT of T(z) (Sec. 6.1), termination, Farkas test, restart
// decision and primal-weight update, then the scalar Halpern blend.
__global__ void __launch_bounds__(kThreads) k_scalar_check(Scal* st, const double* part) {
  if (st->done) return;
  double s[kNumSlots];
  for (int i = kSlRp2; i <= kSlFrG; ++i) {
    const bool mx = i == kSlFkNeg || i == kSlFrNeg || i == kSlFkG || i == kSlFrG;
    s[i] = mx ? block_max_slot(part, i) : block_sum_slot(part, i);
  }
  if (threadIdx.x != 0) return;
  const double up = st->up, vp = st->vp, u = st->u, v = st->v, u0 = st->u0, v0 = st->v0;
  double om = st->omega;
  const double SbP = s[kSlSBandP], SgP = s[kSlSGelP];
  double rd2 = s[kSlRd2], rd2s = s[kSlRd2s];
  double pobj = 0.0, dobj = s[kSlDobL];
  if (st->has_u) {
    const double r = fmin(st->c_u - SbP, 0.0);
    rd2 += r * r;
    if (st->col_u > 0) rd2s += r * r / st->col_u;
    pobj += st->c_u * up;
  } else {
    dobj -= st->band_rhs * SbP;
  }
  if (st->has_v) {
    const double r = st->c_v - SgP;
    const double m = fmin(r, 0.0);
    rd2 += m * m;
    if (st->col_v > 0) rd2s += m * m / st->col_v;
    dobj += fmax(r, 0.0);
    pobj += st->c_v * vp;
  } else {
    dobj -= s[kSlDobU];
  }
  const double rp = sqrt(s[kSlRp2]), rd = sqrt(rd2);
  const double rel_p = rp / (1.0 + st->h_norm), rel_d = rd / (1.0 + st->c_norm);
  const double gap = fabs(pobj - dobj);
  const double rel_gap = gap / (1.0 + fabs(pobj) + fabs(dobj));
  st->rp = rp; st->rd = rd; st->rel_p = rel_p; st->rel_d = rel_d; st->gap = gap;
  st->rel_gap = rel_gap; st->pobj = pobj; st->dobj = dobj;
  st->kkt = fmax(rel_p, fmax(rel_d, rel_gap));
  st->sband_p = SbP; st->sgel_p = SgP;
  if (!isfinite(rel_p) || !isfinite(rel_d) || !isfinite(rel_gap)) {
    // NaN or infinity in the iterates: no status can be decided from them
    st->numeric = 1;
    st->status = 3;
    st->done = 1;
    return;
  }
  // Farkas candidates (primal infeasibility, Secs. 2.7.1-2.7.2): the dual
  // difference since the last restart, and the dual part of the fixed-point
  // residual T(z) - z (which tends to the infimal displacement of PDHG).
  auto farkas = [&](double L, double band, double gel, double up, double g2, double neg) {
    double obj = L, ru = 0.0, rv = 0.0;
    if (st->has_u) ru = -band;
    else obj -= st->band_rhs * band;
    if (st->has_v) { rv = -gel; obj += fmax(rv, 0.0); }
    else obj -= up;
    if (!(obj > 0.0)) return -1.0;
    // l_inf violation of the ray's conditions relative to its dual objective
    const double viol = fmax(fmax(g2, neg), fmax(-fmin(ru, 0.0), -fmin(rv, 0.0)));
    return viol / obj;
  };
  const double fe = farkas(s[kSlFkL], s[kSlFkBand], s[kSlFkGel], s[kSlFkUp], s[kSlFkG], s[kSlFkNeg]);
  const double fr = farkas(s[kSlFrL], s[kSlFrBand], s[kSlFrGel], s[kSlFrUp], s[kSlFrG], s[kSlFrNeg]);
  if (st->trace && st->trace_n < st->trace_cap) {
    double* e = st->trace + (size_t)st->trace_n * kTraceFields;
    e[0] = double(st->k); e[1] = st->kkt; e[2] = rel_p; e[3] = rel_d; e[4] = rel_gap;
    e[5] = pobj; e[6] = om; e[7] = double(st->restarts); e[8] = fe; e[9] = fr;
    st->trace_n += 1;
  }
  int status = -1;
  if (rel_p <= st->kkt_tol && rel_d <= st->kkt_tol && rel_gap <= st->kkt_tol) {
    status = 0;
  } else if (st->k > 0 && ((fe >= 0.0 && fe <= kInfeasTol) || (fr >= 0.0 && fr <= kInfeasTol) ||
                            st->cert)) {
    status = 1;
  }
  if (status < 0 && st->k >= st->max_iter) status = 3;
  if (status >= 0) {
    st->status = status;
    st->done = 1;
    return;
  }
  const double r = sqrt(om * (s[kSlFpX] + st->col_u * (u - up) * (u - up) +
                              st->col_v * (v - vp) * (v - vp)) + s[kSlFpL] / om);
  int restart = 0;
  if (!st->r0_set) {
    st->r0 = r;
    st->r0_set = 1;
  } else if (r <= kBetaSufficient * st->r0 || (r <= kBetaNecessary * st->r0 && r > st->r_prev) ||
             double(st->k_in) >= kBetaArtificial * double(st->k)) {
    restart = 1;
  }
  st->r_prev = r;
  if (restart) {
    const double ex2 = s[kSlOmX] + st->col_u * (up - u0) * (up - u0) + st->col_v * (vp - v0) * (vp - v0);
    const double el2 = s[kSlOmL];
    // the first restart sets omega to the measured ratio, later ones smooth
    const double th = st->restarts == 0 ? 1.0 : kOmegaSmoothing;
    if (ex2 > 1e-30 && el2 > 1e-30) om = exp(th * 0.5 * log(el2 / ex2) + (1.0 - th) * log(om));
    st->omega = om;
    st->u = up; st->v = vp; st->u0 = up; st->v0 = vp;
    st->k_in = 0;
    st->r0 = r;
    st->r_prev = r;
    st->restarts += 1;
  } else {
    const double w = st->w;
    st->u = w * (2.0 * up - u) + (1.0 - w) * u0;
    st->v = w * (2.0 * vp - v) + (1.0 - w) * v0;
    st->k_in += 1;
  }
  st->restart = restart;
  st->k += 1;
}

// ------------------------------------------- bound-based certificate
// Primal infeasibility by Farkas' lemma with a bound on the rays (a reading of
// the infeasibility diagnostic of Secs. 2.7.1-2.7.2).  The constant upper rows
// bound every feasible ray set: Case 2, sum_band d <= |band|; Case 1,
// sum_gel d <= sum_gel f~_U.  With b = A 1_rows (those rows) and B that sum,
// a candidate lam^ >= 0 without lam_up on the rows whose bound moves with a
// free scalar (gel in Case 2, band in Case 1) satisfies, for every feasible y,
// y^T A(lam^_up - lam^_lo) <= -obj, while y^T g^ >= -kappa B with
// kappa = max over active rays of max(-g^_j, 0) / b_j.  obj > kappa B thus
// proves infeasibility; the test asks for kappa B <= (1 - kCertMargin) obj.

// rows indicator (1 on the bounding rows, else 0) for b = A 1_rows
template <typename C>
__global__ void __launch_bounds__(kThreads) k_cert_rows(const uint8_t* __restrict__ lab, C* __restrict__ out,
                                                        int kase, long long n) {
  const uint8_t rows = kase == 2 ? kBand : kGel;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = lab[i] == rows ? C(1) : C(0);
}

// The epoch difference lam+ - lam0 projected onto the certificate's support,
// lam^_up - lam^_lo written to cert_q, and the FP64 partials of its dual
// objective obj = sum_gel L lam^_lo - sum_const-up U lam^_up.
template <typename S, typename C>
__global__ void __launch_bounds__(kThreads) k_cert_vol(Bufs<S, C> b, long long n) {
  if (b.st->done) return;
  const bool case2 = b.has_v != 0;
  double red[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint8_t l = b.lab[i];
    C qv = C(0);
    if (l == kGel) {
      const C f = b.ft ? b.ft[i] : b.ft_const;
      const C dlo = to_c(b.lpl[i]) - to_c(b.ll0[i]);
      const C llh = dlo > C(0) ? dlo : C(0);
      red[0] += double(f) * double(llh);
      C luh = C(0);
      if (!case2) {
        const C dup = to_c(b.lpu[i]) - to_c(b.lu0[i]);
        luh = dup > C(0) ? dup : C(0);
        const C fU = b.fu ? b.fu[i] : f * b.up_ratio;
        red[0] -= double(fU) * double(luh);
      }
      qv = luh - llh;
    } else if (l == kBand && case2) {
      const C dup = to_c(b.lpu[i]) - to_c(b.lu0[i]);
      const C luh = dup > C(0) ? dup : C(0);
      red[0] -= double(b.band_rhs) * double(luh);
      qv = luh;
    }
    b.cert_q[i] = qv;
  }
  block_reduce_store<1>(red, b.part, kSlCertObj);
}

// One block: the decision from the partials of k_cert_vol and of the
// projector's certificate mode.
__global__ void __launch_bounds__(kThreads) k_cert_decide(Scal* st, const double* part) {
  if (st->done) return;
  const double obj = block_sum_slot(part, kSlCertObj);
  const double kappa = block_max_slot(part, kSlCertK);
  if (threadIdx.x != 0) return;
  st->cert = (obj > 0.0 && kappa * st->cert_B <= (1.0 - kCertMargin) * obj) ? 1 : 0;
}

// ----------------------------------- bound-based certificate, slice by slice
// Without a PSF extent along z the operator maps each z-slice's rays to that
// slice's voxels only (slice-separable forward model, Sec. 2.3), so the
// Farkas bound above holds per slice: obj_z > kappa_z B_z for one slice z
// proves infeasibility.  The per-z sums below use a fixed grid: block b
// covers a contiguous range of (y, x) columns, thread t the z values
// t, t + blockDim.x, ...; each block writes one partial per z and the
// decision sums them in block order, so the result does not depend on timing.
constexpr int kCertBlocks = 304;  // fixed (block-order sums), 2 per SM of a GB300
constexpr int kCertMaxZ = 4096;   // slice mode needs nz <= this (shared maxima)

__device__ __forceinline__ void cert_col_range(long long ncol, long long& c0, long long& c1) {
  const long long per = (ncol + gridDim.x - 1) / gridDim.x;
  c0 = blockIdx.x * per;
  c1 = c0 + per < ncol ? c0 + per : ncol;
}

// B_z: per slice, the sum of the constant upper bounds of the bounding rows
// (Case 2: band rows, bound 1; Case 1: gel rows, bound f~_U).
template <typename C>
__global__ void __launch_bounds__(kThreads)
k_cert_bz(const uint8_t* __restrict__ lab, const C* __restrict__ ft, C ft_const, const C* __restrict__ fu,
          double up_ratio, int kase, long long ncol, int nz, double* __restrict__ partz) {
  long long c0, c1;
  cert_col_range(ncol, c0, c1);
  for (int z = threadIdx.x; z < nz; z += blockDim.x) {
    double acc = 0.0;
    for (long long c = c0; c < c1; ++c) {
      const long long i = c * nz + z;
      const uint8_t l = lab[i];
      if (kase == 2) {
        if (l == kBand) acc += 1.0;
      } else if (l == kGel) {
        const double f = ft ? double(ft[i]) : double(ft_const);
        acc += fu ? double(fu[i]) : f * up_ratio;
      }
    }
    partz[(size_t)blockIdx.x * nz + z] = acc;
  }
}

// out[z] = sum over blocks of partz (block order).
__global__ void __launch_bounds__(kThreads)
k_cert_zsum(const double* __restrict__ partz, int nblocks, int nz, double* __restrict__ out) {
  for (int z = blockIdx.x * blockDim.x + threadIdx.x; z < nz; z += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nblocks; ++b) acc += partz[(size_t)b * nz + z];
    out[z] = acc;
  }
}

// The candidate of k_cert_vol, written to cert_q, with its dual objective
// summed per slice into partz[block][z].
template <typename S, typename C>
__global__ void __launch_bounds__(kThreads) k_cert_vol_z(Bufs<S, C> b, long long ncol, int nz, double* partz) {
  if (b.st->done) return;
  const bool case2 = b.has_v != 0;
  long long c0, c1;
  cert_col_range(ncol, c0, c1);
  for (int z = threadIdx.x; z < nz; z += blockDim.x) {
    double acc = 0.0;
    for (long long c = c0; c < c1; ++c) {
      const long long i = c * nz + z;
      const uint8_t l = b.lab[i];
      C qv = C(0);
      if (l == kGel) {
        const C f = b.ft ? b.ft[i] : b.ft_const;
        const C dlo = to_c(b.lpl[i]) - to_c(b.ll0[i]);
        const C llh = dlo > C(0) ? dlo : C(0);
        acc += double(f) * double(llh);
        C luh = C(0);
        if (!case2) {
          const C dup = to_c(b.lpu[i]) - to_c(b.lu0[i]);
          luh = dup > C(0) ? dup : C(0);
          const C fU = b.fu ? b.fu[i] : f * b.up_ratio;
          acc -= double(fU) * double(luh);
        }
        qv = luh - llh;
      } else if (l == kBand && case2) {
        const C dup = to_c(b.lpu[i]) - to_c(b.lu0[i]);
        const C luh = dup > C(0) ? dup : C(0);
        acc -= double(b.band_rhs) * double(luh);
        qv = luh;
      }
      b.cert_q[i] = qv;
    }
    partz[(size_t)blockIdx.x * nz + z] = acc;
  }
}

// One block: per slice obj_z (block partials of k_cert_vol_z), kappa_z (the
// projector's maxima) and B_z; the decision and the first slice that carries
// it.  The maxima are cleared for the next check.
__global__ void __launch_bounds__(kThreads)
k_cert_decide_z(Scal* st, const double* __restrict__ partz, int nblocks, int nz, unsigned long long* kz,
                const double* __restrict__ Bz) {
  __shared__ int first;
  if (threadIdx.x == 0) first = 0x7fffffff;
  __syncthreads();
  const bool live = !st->done;
  for (int z = threadIdx.x; z < nz; z += blockDim.x) {
    if (live) {
      double obj = 0.0;
      for (int b = 0; b < nblocks; ++b) obj += partz[(size_t)b * nz + z];
      const double kappa = __longlong_as_double((long long)kz[z]);
      if (obj > 0.0 && kappa * Bz[z] <= (1.0 - kCertMargin) * obj) atomicMin(&first, z);
    }
    kz[z] = 0ull;
  }
  __syncthreads();
  if (threadIdx.x == 0 && live) {
    st->cert = first != 0x7fffffff ? 1 : 0;
    st->cert_z = st->cert ? first : -1;
  }
}

// --------------------------------------------------------- blend kernels
// After a check step: next iterate = T(z) (restart) or the Halpern blend.
template <typename S, typename C, int ZL>
__global__ void __launch_bounds__(kThreads) k_blend_sino(Bufs<S, C> b, long long nvec) {
  if (b.st->done) return;
  const int restart = b.st->restart;
  const C w = C(b.st->w);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvec;
       i += (long long)gridDim.x * blockDim.x) {
    const size_t base = size_t(i) * ZL;
    C col[ZL];
    load_z<C, C, ZL>(b.col + base, col);
    bool any = false;
#pragma unroll
    for (int k = 0; k < ZL; ++k) any |= col[k] > C(0);
    if (!any) continue;
    C yp[ZL];
    load_z<S, C, ZL>(b.yp + base, yp);
    if (restart) {
      store_z<S, C, ZL>(b.y + base, yp);
      store_z<S, C, ZL>(b.y0 + base, yp);
      C gp[ZL];
      load_z<C, C, ZL>(b.gp + base, gp);
      store_z<C, C, ZL>(b.g0 + base, gp);
    } else {
      C y[ZL], y0[ZL];
      load_z<S, C, ZL>(b.y + base, y);
      load_z<S, C, ZL>(b.y0 + base, y0);
#pragma unroll
      for (int k = 0; k < ZL; ++k) y[k] = w * (C(2) * yp[k] - y[k]) + (C(1) - w) * y0[k];
      store_z<S, C, ZL>(b.y + base, y);
    }
  }
}

template <typename S, typename C, int ZL>
__global__ void __launch_bounds__(kThreads) k_blend_vol(Bufs<S, C> b, long long nvec) {
  if (b.st->done) return;
  const int restart = b.st->restart;
  const C w = C(b.st->w);
  double red[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvec;
       i += (long long)gridDim.x * blockDim.x) {
    const size_t base = size_t(i) * ZL;
    uint8_t lab[ZL];
    bool any = false;
#pragma unroll
    for (int k = 0; k < ZL; ++k) { lab[k] = b.lab[base + k]; any |= lab[k] != kExt; }
    if (!any) continue;
    C pu[ZL], pl[ZL], dp[ZL], ft[ZL];
    load_z<S, C, ZL>(b.lpu + base, pu);
    load_z<S, C, ZL>(b.lpl + base, pl);
    load_z<C, C, ZL>(b.dp + base, dp);
    if (b.ft) load_z<C, C, ZL>(b.ft + base, ft);
    else {
#pragma unroll
      for (int k = 0; k < ZL; ++k) ft[k] = b.ft_const;
    }
    C nu[ZL], nl[ZL], nd[ZL], nq[ZL];
    if (restart) {
#pragma unroll
      for (int k = 0; k < ZL; ++k) { nu[k] = pu[k]; nl[k] = pl[k]; nd[k] = dp[k]; }
      store_z<S, C, ZL>(b.lu0 + base, pu);
      store_z<S, C, ZL>(b.ll0 + base, pl);
      store_z<C, C, ZL>(b.d0 + base, dp);
    } else {
      C lu[ZL], ll[ZL], lu0[ZL], ll0[ZL], d[ZL], d0[ZL];
      load_z<S, C, ZL>(b.lu + base, lu);
      load_z<S, C, ZL>(b.ll + base, ll);
      load_z<S, C, ZL>(b.lu0 + base, lu0);
      load_z<S, C, ZL>(b.ll0 + base, ll0);
      load_z<C, C, ZL>(b.d + base, d);
      load_z<C, C, ZL>(b.d0 + base, d0);
#pragma unroll
      for (int k = 0; k < ZL; ++k) {
        nu[k] = rnd<S, C>(w * (C(2) * pu[k] - lu[k]) + (C(1) - w) * lu0[k]);
        nl[k] = rnd<S, C>(w * (C(2) * pl[k] - ll[k]) + (C(1) - w) * ll0[k]);
        nd[k] = w * (C(2) * dp[k] - d[k]) + (C(1) - w) * d0[k];
      }
    }
#pragma unroll
    for (int k = 0; k < ZL; ++k) {
      if (lab[k] == kExt) { nu[k] = C(0); nl[k] = C(0); }
      nq[k] = nu[k] - nl[k];
      if (lab[k] == kBand) red[0] += double(nu[k]);
      else if (lab[k] == kGel) red[1] += double(ft[k]) * double(nu[k]);
    }
    store_z<S, C, ZL>(b.lu + base, nu);
    store_z<S, C, ZL>(b.ll + base, nl);
    store_z<C, C, ZL>(b.d + base, nd);
    store_z<S, C, ZL>(b.q + base, nq);
  }
  block_reduce_store<2>(red, b.part, kSlSBand);
}

// Stand-alone dual update from a stored d_bar: used when the PSF sits between
// P^T and the prox, and by every check step (whose FP64 reductions would spill
// registers inside the backprojector).
template <typename S, typename C, int ZL, bool CHECK>
__global__ void __launch_bounds__(kThreads) k_dual(Bufs<S, C> b, const C* __restrict__ dbar,
                                                   long long nvec) {
  if (b.st->done) return;
  const StepScalars<C> sc = read_scalars<C>(b.st);
  constexpr int NR = CHECK ? kCheckSlots : 2;
  double red[NR] = {};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvec;
       i += (long long)gridDim.x * blockDim.x) {
    const size_t base = size_t(i) * ZL;
    C db[ZL];
    load_z<C, C, ZL>(dbar + base, db);
    dual_update<S, C, ZL, CHECK>(b, sc, base, db, red);
  }
  block_reduce_store<NR, CHECK ? kCheckMaxMask : 0u>(red, b.part, CHECK ? kSlRp2 : kSlSBand);
}

// --------------------------------------------------------- post-solve
// Per block: 0 min_gel d/f~T, 1 max_gel d/f~T, 2 max_band d, 3 min_gel d,
// 4 sum_gel d f_T, 5 sum_gel d^2, 6 min_gel d / f~ (recovered scale s),
// 7 max_gel d / f~ (maximum relative dose of the LP).
template <typename C>
__global__ void __launch_bounds__(kThreads)
k_metrics(const C* __restrict__ d, const uint8_t* __restrict__ lab, const float* __restrict__ fT,
          const C* __restrict__ ft, C ft_const, double f_crit, long long n, double* __restrict__ part) {
  double mn_r = 1e300, mx_r = -1e300, mx_b = -1e300, mn_d = 1e300, sdf = 0.0, sdd = 0.0;
  double mn_s = 1e300, mx_s = -1e300;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint8_t l = lab[i];
    if (l == kBand) {
      mx_b = fmax(mx_b, double(d[i]));
    } else if (l == kGel) {
      const double dv = double(d[i]);
      const double ftT = double(fT[i]) / f_crit;
      const double r = dv / ftT;
      mn_r = fmin(mn_r, r);
      mx_r = fmax(mx_r, r);
      mn_d = fmin(mn_d, dv);
      sdf += dv * double(fT[i]);
      sdd += dv * dv;
      const double fl = ft ? double(ft[i]) : double(ft_const);
      mn_s = fmin(mn_s, dv / fl);
      mx_s = fmax(mx_s, dv / fl);
    }
  }
  __shared__ double sh[kThreads];
  double vals[8] = {mn_r, mx_r, mx_b, mn_d, sdf, sdd, mn_s, mx_s};
  for (int q = 0; q < 8; ++q) {
    sh[threadIdx.x] = vals[q];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) {
        const double a = sh[threadIdx.x], c = sh[threadIdx.x + st];
        sh[threadIdx.x] = (q == 0 || q == 3 || q == 6) ? fmin(a, c)
                          : (q == 4 || q == 5) ? a + c : fmax(a, c);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) part[q * kRedBlocks + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

// < a, b > per block (for the PSF sigma gradient).
template <typename C>
__global__ void __launch_bounds__(kThreads) k_dot(const C* __restrict__ a, const C* __restrict__ b,
                                                  long long n, double* __restrict__ part) {
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[0] += double(a[i]) * double(b[i]);
  block_reduce_store<1>(v, part, 0);
}

}  // namespace sipo
