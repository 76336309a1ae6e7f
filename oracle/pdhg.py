"""Oracle restarted Halpern PDHG for the SiPO LP (FP64, CPU, explicit sparse A).

Test infrastructure only (like the whole oracle package): never imported by the product path.

The paper solves the LP with a matrix-free primal-dual hybrid gradient method
driven by the KKT conditions (Sec. 2.8, Sec. 6.1) and gives no further recipe.
The readings implemented here (and by the GPU solver) are published methods:

* The PDHG step T (Chambolle-Pock, primal first, primal extrapolation) on
  min_x max_{lam>=0} c^T x + lam^T (G x - h), x = (y, u~, v~):
      g      = A (lam_up - lam_lo)                         [Eq. 51]
      y+     = max(0, y - tau_y g)        (tau_y = 0 on masked rays)
      u+     = max(0, u - tau_u (c_u - sum_band lam_up))   [Eq. 48]
      v+     = max(1, v - tau_v (c_v - sum_gel f~ lam_up)) [Eq. 49]
      y_bar  = 2 y+ - y,  u_bar = 2 u+ - u,  v_bar = 2 v+ - v
      d_bar  = A^T y_bar                                   [Eqs. 2-3]
      lam_up+ = max(0, lam_up + sigma_up (d_bar - U(u_bar, v_bar)))
      lam_lo+ = max(0, lam_lo + sigma_lo (L - d_bar))
* Diagonal Pock-Chambolle preconditioning (alpha = 1): tau = eta / (omega *
  column abs-sum of G), sigma = eta * omega / row abs-sum, eta = 0.99, with a
  primal weight omega.
* Reflected Halpern iteration with restarts (restarted Halpern PDHG, Lu & Yang
  2024): z <- w (2 T(z) - z) + (1 - w) z0, w = (k+1)/(k+2), k counted from the
  last restart point z0.
* Every `check_every` iterations: the KKT error of T(z) in the unscaled
  problem decides termination (relative primal residual, relative dual
  residual and relative gap all <= tol); the fixed-point residual
  r = ||z - T(z)|| (preconditioned norm weighted by omega) decides restarts:
  sufficient decay r <= 0.2 r0, necessary decay r <= 0.8 r0 without progress
  since the previous check, or an artificial restart when the epoch reaches
  36% of all iterations.  A restart moves z and z0 to T(z) and updates omega
  towards ||lam - lam0|| / ||x - x0|| (scaled norms): the first restart sets
  it to that ratio (omega0 = ||c|| / ||h|| can be two orders of magnitude off,
  e.g. in Case 1), later ones by log-smoothing (0.5).
* Primal infeasibility (Secs. 2.7.1-2.7.2 treat an infeasible LP as a
  diagnostic): at each check two candidate directions are tested as a Farkas
  ray -- the dual difference lam+ - lam0 since the last restart, and the dual
  part of the fixed-point residual T(z) - z, which tends to the infimal
  displacement vector of PDHG (Applegate, Diaz, Lu & Lubin 2021).  A ray's
  reduced costs G^T dlam must be non-negative on every primal column, the ray
  non-negative, and its dual objective positive; the largest violation
  (l_inf) relative to the objective <= 1e-6.
* A bound-based certificate (a reading: Farkas' lemma applied to this LP with
  an a-priori bound on the rays) tests the first candidate exactly.  Project
  it onto the support a certificate may have -- lam >= 0, and no lam_up on the
  rows whose bound moves with a free scalar (band rows in Case 1, where u~ is
  free upward; gel rows in Case 2, where v~ is) -- and apply A to it exactly:
  g^ = A (lam^_up - lam^_lo).  For every feasible y,
      y^T g^ <= -obj,   obj = sum_gel L lam^_lo - sum_const-up U lam^_up,
  and the constant upper rows bound the rays: sum_j y_j b_j <= B with
  b = A 1_rows, B = sum_rows U over those rows (Case 2: band rows with U = 1;
  Case 1: gel rows with U = f~_U).  So y^T g^ >= -kappa B with
  kappa = max_j max(-g^_j, 0) / b_j over active rays, and obj > kappa B proves
  that no feasible y exists.  The test asks for obj > 0 and
  kappa B <= (1 - 1e-3) obj, the margin covering rounding of g^.  The
  general case has no constant upper rows (every LP of that form is
  feasible) and no such test.
* Slice by slice (a reading of the slice-separable forward model of
  Sec. 2.3): when the PSF has no z extent, A maps the rays of slice z only to
  the voxels of slice z, so both inequalities above hold for each slice on
  its own -- y_z^T g^_z <= -obj_z and y_z^T g^_z >= -kappa_z B_z, with obj_z,
  kappa_z and B_z the same quantities restricted to slice z.  One slice with
  obj_z > kappa_z B_z (margin as above) proves the whole LP infeasible.  This
  test implies the whole-volume one (if obj > kappa B then some slice has
  obj_z > kappa_z B_z), and it is not diluted by feasible slices: a single
  infeasible slice among many feasible ones carries the certificate alone.
"""
from __future__ import annotations

import math

import numpy as np

from .lp import CASE1, CASE2, LPData, kkt, metrics, up_bound
from .operators import Operators

OPTIMAL, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE, ITER_LIMIT = 0, 1, 2, 3

ETA = 0.99
BETA_SUFFICIENT = 0.2
BETA_NECESSARY = 0.8
BETA_ARTIFICIAL = 0.36
OMEGA_SMOOTHING = 0.5
INFEAS_TOL = 1e-6
CERT_MARGIN = 1e-3


class Preconditioner:
    """Pock-Chambolle (alpha = 1) column and row abs-sums of the LP matrix G."""

    def __init__(self, lp: LPData, ops: Operators):
        band, gel = lp.band, lp.gel
        g = ops.geo
        ind = band.astype(np.float64) + 2.0 * gel.astype(np.float64)
        col = ops.A(ind.reshape(g.vol_shape)).ravel()
        self.col_y = np.where(lp.active, col, 0.0)
        self.col_u = float(band.sum()) if lp.has_u else 0.0
        self.col_v = float(np.sum(lp.ft[gel])) if lp.has_v else 0.0
        row = ops.AT(lp.active.astype(np.float64).reshape(g.sino_shape)).ravel()
        up = row.copy()
        if lp.has_u:
            up[band] += 1.0
        if lp.has_v:
            up[gel] += lp.ft[gel]
        self.row_up = np.where(band | gel, up, 0.0)
        self.row_lo = np.where(gel, row, 0.0)

    @staticmethod
    def inv(a):
        out = np.zeros_like(a)
        nz = a > 0
        out[nz] = 1.0 / a[nz]
        return out


def _scaled_residuals(lp, pc, d, g, u, v, lam_up, lam_lo):
    """Squared primal and dual residuals in the preconditioned space."""
    band, gel = lp.band, lp.gel
    U = up_bound(lp, u, v)
    iu = Preconditioner.inv(pc.row_up)
    il = Preconditioner.inv(pc.row_lo)
    m = band | gel
    rp2 = np.sum(np.maximum(d[m] - U[m], 0.0) ** 2 * iu[m])
    rp2 += np.sum(np.maximum(lp.lower[gel] - d[gel], 0.0) ** 2 * il[gel])
    ic = Preconditioner.inv(pc.col_y)
    rd2 = np.sum(np.minimum(g[lp.active], 0.0) ** 2 * ic[lp.active])
    if lp.has_u:
        rd2 += min(lp.c_u - lam_up[band].sum(), 0.0) ** 2 / pc.col_u
    if lp.has_v:
        rd2 += min(lp.c_v - np.sum(lp.ft[gel] * lam_up[gel]), 0.0) ** 2 / pc.col_v
    return rp2, rd2


def _farkas(lp, pc, dq_g, dlam_up, dlam_lo):
    """True if the dual difference is (approximately) a primal-infeasibility ray."""
    band, gel = lp.band, lp.gel
    obj = np.sum(lp.lower[gel] * dlam_lo[gel])
    if lp.has_u:
        ru = -dlam_up[band].sum()
    else:
        obj -= lp.band_rhs() * dlam_up[band].sum()
        ru = 0.0
    sgel = np.sum(lp.ft[gel] * dlam_up[gel])
    if lp.has_v:
        rv = -sgel
        obj += max(rv, 0.0)
    else:
        obj -= np.sum(lp.upper[gel] * dlam_up[gel])
        rv = 0.0
    if not obj > 0:
        return False
    viol = max(np.max(np.maximum(-dq_g[lp.active], 0.0), initial=0.0),
               -min(ru, 0.0), -min(rv, 0.0),
               np.max(np.maximum(-dlam_up, 0.0), initial=0.0),
               np.max(np.maximum(-dlam_lo, 0.0), initial=0.0))
    return viol / obj <= INFEAS_TOL


def certificate_data(lp: LPData, ops: Operators):
    """(b, B, B_z) of the bound-based certificate: b = A 1_rows on every ray,
    B = sum of the constant upper bounds over those rows (Case 2: band rows,
    bound 1; Case 1: gel rows, bound f~_U) and B_z the same sum per z-slice;
    None for the general case."""
    g = ops.geo
    if lp.case == CASE2:
        rows = lp.band
        U = rows.astype(np.float64)
    elif lp.case == CASE1:
        rows = lp.gel
        U = np.where(rows, lp.upper, 0.0)
    else:
        return None
    b = ops.A(rows.astype(np.float64).reshape(g.vol_shape)).ravel()
    B_z = U.reshape(g.vol_shape).sum(axis=(0, 1))
    return b, float(U.sum()), B_z


def slices_decoupled(ops: Operators) -> bool:
    """True when A maps each z-slice's rays to that slice's voxels only: the
    parallel-beam operator is slice-separable (Sec. 2.3) and only a PSF with a
    z extent couples slices."""
    return ops.geo.nz > 1 and ops.geo.psf_radii()[2] == 0


def certificate(lp: LPData, ops: Operators, dlam_up, dlam_lo, b, B, B_z=None, per_slice=True):
    """True if the projected dual difference proves primal infeasibility
    (bound-based Farkas test of the module docstring), slice by slice when
    the operator does not couple z-slices."""
    band, gel = lp.band, lp.gel
    lu = np.zeros(lp.labels.size)
    ll = np.zeros(lp.labels.size)
    ll[gel] = np.maximum(dlam_lo[gel], 0.0)
    if lp.case == CASE2:
        lu[band] = np.maximum(dlam_up[band], 0.0)
        objv = lp.lower * ll - lu
    else:
        lu[gel] = np.maximum(dlam_up[gel], 0.0)
        objv = lp.lower * ll - lp.upper * lu
    objv = np.where(gel | band, objv, 0.0)
    g = ops.A((lu - ll).reshape(ops.geo.vol_shape)).ravel()
    act = lp.active
    viol = np.where(act, np.maximum(-g, 0.0), 0.0)
    bad = (viol > 0) & (b <= 0)
    ratio = np.where(viol > 0, viol / np.where(b > 0, b, 1.0), 0.0)
    if per_slice and B_z is not None and slices_decoupled(ops):
        geo = ops.geo
        obj_z = objv.reshape(geo.vol_shape).sum(axis=(0, 1))
        kappa_z = ratio.reshape(geo.sino_shape).max(axis=(0, 1))
        bad_z = bad.reshape(geo.sino_shape).any(axis=(0, 1))
        ok = (obj_z > 0) & ~bad_z & (kappa_z * B_z <= (1.0 - CERT_MARGIN) * obj_z)
        return bool(ok.any())
    obj = float(objv.sum())
    if not obj > 0 or bad.any():
        return False
    kappa = float(ratio.max(initial=0.0))
    return kappa * B <= (1.0 - CERT_MARGIN) * obj


def primal_start(lp: LPData, ops: Operators, y, u=None, v=None):
    """A caller's primal point made admissible as a starting point: y projected
    onto y >= 0 on the active rays and 0 elsewhere (the primal domain of
    Eqs. 23-24); u~ and v~ as given when admissible (u~ >= 0, v~ >= 1), else
    the smallest values the point allows: u~ = max of A^T y over band rows,
    v~ = max of A^T y / f~ over gel rows (the band and gel upper rows of
    Eqs. 20-21, 33-34, 41-42), clamped to the implied bounds u~ >= 0, v~ >= 1.
    Returns (y, u, v)."""
    y = np.where(lp.active & (np.asarray(y, np.float64).ravel() > 0), np.asarray(y, np.float64).ravel(), 0.0)
    d = ops.AT(y.reshape(ops.geo.sino_shape)).ravel()
    if lp.has_u and not (u is not None and math.isfinite(u) and u >= 0):
        u = max(0.0, float(d[lp.band].max(initial=0.0)))
    if lp.has_v and not (v is not None and math.isfinite(v) and v >= 1):
        gel = lp.gel
        v = max(1.0, float(np.max(d[gel] / lp.ft[gel])))
    return y, (float(u) if lp.has_u else 0.0), (float(v) if lp.has_v else 1.0)


def dual_point(lp: LPData, lam_up, lam_lo):
    """A caller's dual point projected onto the dual domain (Eqs. 20-22):
    lam_up >= 0 on band and gel rows, lam_lo >= 0 on gel rows, 0 elsewhere."""
    up = np.asarray(lam_up, np.float64).ravel()
    lo = np.asarray(lam_lo, np.float64).ravel()
    up = np.where((lp.band | lp.gel) & (up > 0), up, 0.0)
    lo = np.where(lp.gel & (lo > 0), lo, 0.0)
    return up, lo


def solve(lp: LPData, ops: Operators, kkt_tol=1e-4, max_iter=10000,
          check_every=64, omega0=None, verbose=False, history=None, start=None, dual_start=None):
    """Run the restarted Halpern PDHG; returns a dict with status, T(z) and KKT data.

    `iters` counts PDHG steps; the returned point is T(z) at the last check.
    `start` = (y, u, v) starts from that primal point (made admissible by
    `primal_start`; None entries for u, v ask for the smallest admissible)
    with zero duals, instead of from y = 0, u~ = 0, v~ = 1; `dual_start` =
    (lam_up, lam_lo) adds a dual point (made admissible by `dual_point`).
    """
    geo = ops.geo
    pc = Preconditioner(lp, ops)
    band, gel = lp.band, lp.gel
    m_up = band | gel
    S = lp.active.size
    V = lp.labels.size
    inv_col = Preconditioner.inv(pc.col_y)
    inv_up = Preconditioner.inv(pc.row_up)
    inv_lo = Preconditioner.inv(pc.row_lo)
    if omega0 is None:
        omega = initial_omega(lp, pc)
    else:
        omega = float(omega0)

    def AT(s):
        return ops.AT(s.reshape(geo.sino_shape)).ravel()

    def A(vv):
        return ops.A(vv.reshape(geo.vol_shape)).ravel()

    cert = certificate_data(lp, ops)
    y, u, v = np.zeros(S), 0.0, 1.0
    if start is not None:
        y, u, v = primal_start(lp, ops, *start)
    lam_up, lam_lo = np.zeros(V), np.zeros(V)
    if dual_start is not None:
        lam_up, lam_lo = dual_point(lp, *dual_start)
    y0, u0, v0, lam_up0, lam_lo0 = y.copy(), u, v, lam_up.copy(), lam_lo.copy()
    g0 = A(lam_up - lam_lo) if dual_start is not None else np.zeros(S)
    k_in = 0
    r0 = None
    r_prev = None
    restarts = 0
    k = 0
    while True:
        # one PDHG step T(z)
        g = A(lam_up - lam_lo)
        y_p = np.maximum(0.0, y - ETA * inv_col / omega * g)
        S_band = lam_up[band].sum()
        S_gel = np.sum(lp.ft[gel] * lam_up[gel])
        u_p = max(0.0, u - ETA / (omega * pc.col_u) * (lp.c_u - S_band)) if lp.has_u else u
        v_p = max(1.0, v - ETA / (omega * pc.col_v) * (lp.c_v - S_gel)) if lp.has_v else v
        y_bar = 2.0 * y_p - y
        d_bar = AT(y_bar)
        U = up_bound(lp, 2.0 * u_p - u, 2.0 * v_p - v)
        lam_up_p = np.where(m_up, np.maximum(0.0, lam_up + ETA * omega * inv_up * (d_bar - U)), 0.0)
        lam_lo_p = np.where(gel, np.maximum(0.0, lam_lo + ETA * omega * inv_lo * (lp.lower - d_bar)), 0.0)
        restart = False
        if k % check_every == 0 or k == max_iter:
            d_p = AT(y_p)
            g_p = A(lam_up_p - lam_lo_p)
            info = kkt(lp, d_p, g_p, u_p, v_p, lam_up_p, lam_lo_p)
            if history is not None:
                history.append(dict(k=k, omega=omega, restarts=restarts, **info))
            if verbose:
                print(f"k={k} kkt={info['kkt']:.3e} p={info['rel_primal']:.2e} "
                      f"d={info['rel_dual']:.2e} gap={info['rel_gap']:.2e} "
                      f"obj={info['pobj']:.6f} omega={omega:.3e}")
            status = None
            if (info["rel_primal"] <= kkt_tol and info["rel_dual"] <= kkt_tol
                    and info["rel_gap"] <= kkt_tol):
                status = OPTIMAL
            elif k > 0 and (_farkas(lp, pc, g_p - g0, lam_up_p - lam_up0, lam_lo_p - lam_lo0)
                            or _farkas(lp, pc, g_p - g, lam_up_p - lam_up, lam_lo_p - lam_lo)
                            or (cert is not None
                                and certificate(lp, ops, lam_up_p - lam_up0, lam_lo_p - lam_lo0, *cert))):
                status = PRIMAL_INFEASIBLE
            elif k == max_iter:
                status = ITER_LIMIT
            if status is not None:
                out = dict(status=status, iters=k, y=y_p, u=u_p, v=v_p, lam_up=lam_up_p,
                           lam_lo=lam_lo_p, d=d_p, g=g_p, omega=omega, restarts=restarts,
                           info=info, obj=info["pobj"])
                out["metrics"] = metrics(lp, d_p)
                return out
            dx2 = np.sum(pc.col_y * (y - y_p) ** 2) + pc.col_u * (u - u_p) ** 2 \
                + pc.col_v * (v - v_p) ** 2
            dl2 = np.sum(pc.row_up * (lam_up - lam_up_p) ** 2) \
                + np.sum(pc.row_lo * (lam_lo - lam_lo_p) ** 2)
            r = math.sqrt(omega * dx2 + dl2 / omega)
            if r0 is None:
                r0 = r
            elif (r <= BETA_SUFFICIENT * r0 or (r <= BETA_NECESSARY * r0 and r > r_prev)
                  or k_in >= BETA_ARTIFICIAL * k):
                restart = True
            r_prev = r
        if restart:
            ex2 = np.sum(pc.col_y * (y_p - y0) ** 2) + pc.col_u * (u_p - u0) ** 2 \
                + pc.col_v * (v_p - v0) ** 2
            el2 = np.sum(pc.row_up * (lam_up_p - lam_up0) ** 2) \
                + np.sum(pc.row_lo * (lam_lo_p - lam_lo0) ** 2)
            if ex2 > 1e-30 and el2 > 1e-30:
                th = 1.0 if restarts == 0 else OMEGA_SMOOTHING
                omega = math.exp(th * 0.5 * math.log(el2 / ex2) + (1.0 - th) * math.log(omega))
            y, u, v, lam_up, lam_lo = y_p, u_p, v_p, lam_up_p, lam_lo_p
            y0, u0, v0 = y_p.copy(), u_p, v_p
            lam_up0, lam_lo0 = lam_up_p.copy(), lam_lo_p.copy()
            g0 = g_p
            k_in = 0
            r0 = r
            r_prev = r
            restarts += 1
        else:
            w = (k_in + 1.0) / (k_in + 2.0)
            y = w * y_bar + (1.0 - w) * y0
            u = w * (2.0 * u_p - u) + (1.0 - w) * u0
            v = w * (2.0 * v_p - v) + (1.0 - w) * v0
            lam_up = w * (2.0 * lam_up_p - lam_up) + (1.0 - w) * lam_up0
            lam_lo = w * (2.0 * lam_lo_p - lam_lo) + (1.0 - w) * lam_lo0
            k_in += 1
        k += 1


def initial_omega(lp: LPData, pc: Preconditioner) -> float:
    """omega0 = ||c|| / ||h|| in the preconditioned space (1 if either is 0)."""
    gel = lp.gel
    m_up = lp.band | gel
    inv_up = Preconditioner.inv(pc.row_up)
    inv_lo = Preconditioner.inv(pc.row_lo)
    c_hat2 = (lp.c_u ** 2 / pc.col_u if lp.has_u else 0.0) + \
             (lp.c_v ** 2 / pc.col_v if lp.has_v else 0.0)
    U0 = up_bound(lp, 0.0, 0.0)
    h_hat2 = np.sum(U0[m_up] ** 2 * inv_up[m_up]) + np.sum(lp.lower[gel] ** 2 * inv_lo[gel])
    return math.sqrt(c_hat2 / h_hat2) if c_hat2 > 0 and h_hat2 > 0 else 1.0
