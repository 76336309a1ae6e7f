"""Dense two-phase tableau simplex with Bland's rule (oracle, tiny LPs only).

Test infrastructure only (like the whole oracle package): never imported by the product path.

Used to pin the PDHG oracle: on tiny instances the LP of Eqs. 19-24
(general), 32-37 (Case 1) or 40-45 (Case 2) is written out as a dense matrix
and solved exactly (up to rounding) by the textbook simplex method.  Bland's
smallest-index rule prevents cycling on these highly degenerate LPs.

The LP is taken as the paper states it: u~ and v~ are free variables (no
implied bounds), so agreement with the PDHG (which adds u~ >= 0, v~ >= 1)
also checks that those bounds do not move the optimum.
"""
from __future__ import annotations

import numpy as np

from .lp import LPData
from .operators import Operators

TOL = 1e-10
PIVOT_TOL = 1e-9
FEAS_TOL = 1e-9


def _pivot(T, basis, r, c):
    T[r] /= T[r, c]
    for i in range(T.shape[0]):
        if i != r and T[i, c] != 0.0:
            T[i] -= T[i, c] * T[r]
    basis[r] = c


def _run(T, basis, cost, allowed, max_iter):
    """Minimise cost over the columns in `allowed`; returns 'optimal'/'unbounded'."""
    m = T.shape[0]
    for _ in range(max_iter):
        cb = cost[basis]
        red = cost[:-1] - cb @ T[:, :-1]          # reduced costs
        enter = -1
        for j in np.flatnonzero(allowed):
            if red[j] < -TOL:
                enter = j
                break
        if enter < 0:
            return "optimal"
        col = T[:, enter]
        rows = np.flatnonzero(col > PIVOT_TOL)
        if rows.size == 0:
            return "unbounded"
        ratios = T[rows, -1] / col[rows]
        best = ratios.min()
        tied = rows[ratios <= best + TOL * max(1.0, abs(best))]
        leave = tied[np.argmin([basis[i] for i in tied])]
        _pivot(T, basis, leave, enter)
    raise RuntimeError("simplex iteration limit")


def simplex_ineq(G, h, c, max_iter=200000):
    """min c^T x  s.t.  G x <= h, x >= 0.  Returns (status, x, objective).

    Rows with h_i >= 0 start with their slack in the basis; rows with h_i < 0
    are negated (-G_i x - s_i = -h_i) and start with an artificial variable.
    Phase 1 minimises the sum of artificials, phase 2 the objective.
    """
    G = np.array(G, dtype=np.float64)
    h = np.array(h, dtype=np.float64)
    c = np.array(c, dtype=np.float64)
    m, n = G.shape
    neg = np.flatnonzero(h < 0)
    na = neg.size
    T = np.zeros((m, n + m + na + 1))
    T[:, :n] = G
    T[:, n:n + m] = np.eye(m)
    T[:, -1] = h
    T[neg] *= -1.0
    basis = np.arange(n, n + m)
    for a, r in enumerate(neg):
        T[r, n + m + a] = 1.0
        basis[r] = n + m + a
    ntot = n + m + na
    if na:
        cost1 = np.zeros(ntot + 1)
        cost1[n + m:ntot] = 1.0
        _run(T, basis, cost1, np.ones(ntot, dtype=bool), max_iter)
        if T[:, -1] @ cost1[basis] > 1e-9 * max(1.0, np.abs(h).max()):
            return "infeasible", None, None
        # an artificial still basic (at level zero) leaves through the largest
        # entry of its row; a row with no usable entry is redundant and keeps it
        for r in range(m):
            if basis[r] >= n + m:
                j = int(np.argmax(np.abs(T[r, :n + m])))
                if abs(T[r, j]) > 1e-9:
                    _pivot(T, basis, r, j)
    cost2 = np.zeros(ntot + 1)
    cost2[:n] = c
    allowed = np.zeros(ntot, dtype=bool)
    allowed[:n + m] = True
    status = _run(T, basis, cost2, allowed, max_iter)
    if status != "optimal":
        return status, None, None
    x = np.zeros(ntot)
    x[basis] = T[:, -1]
    # The tableau carries the rounding of every pivot; a pivot on a near-zero
    # entry can push the vertex off the feasible set, and such a vertex is not
    # an optimum: refuse it rather than report its objective.
    scale = max(1.0, np.abs(h).max())
    if x.min() < -FEAS_TOL * scale or (G @ x[:n] - h).max() > FEAS_TOL * scale:
        raise RuntimeError("simplex lost primal feasibility")
    return "optimal", x[:n], float(c @ x[:n])


def dense_lp(lp: LPData, ops: Operators):
    """The LP as dense data: variables (y_active, u+, u-, v+, v-), rows G x <= h."""
    if ops.geo.nz != 1:
        raise ValueError("dense LP only for single slices")
    PT = ops.PT.toarray()
    if any(s > 0 for s in ops.geo.psf_sigma):
        raise ValueError("dense LP only without PSF")
    act = np.flatnonzero(lp.active)
    M = PT[:, act]                      # A^T restricted to active rays
    band = np.flatnonzero(lp.band)
    gel = np.flatnonzero(lp.gel)
    ny = act.size
    n = ny + 4
    rows, rhs = [], []
    for i in band:
        r = np.zeros(n)
        r[:ny] = M[i]
        if lp.has_u:
            r[ny], r[ny + 1] = -1.0, 1.0
            rhs.append(0.0)
        else:
            rhs.append(1.0)
        rows.append(r)
    for i in gel:
        r = np.zeros(n)
        r[:ny] = M[i]
        if lp.has_v:
            r[ny + 2], r[ny + 3] = -lp.ft[i], lp.ft[i]
            rhs.append(0.0)
        else:
            rhs.append(lp.upper[i])
        rows.append(r)
    for i in gel:
        r = np.zeros(n)
        r[:ny] = -M[i]
        rows.append(r)
        rhs.append(-lp.lower[i])
    G = np.array(rows)
    h = np.array(rhs)
    c = np.zeros(n)
    if lp.has_u:
        c[ny], c[ny + 1] = lp.c_u, -lp.c_u
    if lp.has_v:
        c[ny + 2], c[ny + 3] = lp.c_v, -lp.c_v
    return G, h, c, act


def solve_dense(lp: LPData, ops: Operators):
    """Exact optimum of the LP by simplex; returns (status, objective, y_full)."""
    G, h, c, act = dense_lp(lp, ops)
    status, x, obj = simplex_ineq(G, h, c)
    if status != "optimal":
        return status, None, None
    y = np.zeros(lp.active.size)
    y[act] = x[:act.size]
    return status, obj, y
