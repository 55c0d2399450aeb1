"""FP64 CPU oracle of the linear feasibility projection (Sec. II, eq. linfeas).

TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU legs are the only
callers.  It imports nothing from the GPU package.

The projection of a point x0 onto the linear constraints of the ACOPF NLP
(eq. nlp, A x >= b):

    min ||x - x0||^2  s.t.  power balance (eq. opfc5, opfc6) with the branch
    flows of eq. acopf_pf, which are linear in (w, wR, wI);
    bounds on pg, qg (opfc1-2), w (opfc3), theta (opfc4) and theta_ref = 0.

x = [pg(G) | qg(G) | w(B) | theta(B) | wR(L) | wI(L)]; wR and wI are free.
The problem is a strictly convex QP with equality rows E x = e and bounds
lo <= x <= hi.  Its dual function g(mu) = min_{lo<=x<=hi} 1/2 ||x - x0||^2 +
mu'(E x - e) is concave and piecewise quadratic with maximiser mu*; the
primal solution is x(mu) = clamp(x0 - E' mu, lo, hi).  mu* is found by
semismooth Newton on grad g = E x(mu) - e with a backtracking line search on
g, which terminates once the active pattern is right; the result is checked
against the KKT conditions before it is returned.
"""
from __future__ import annotations

import math

import numpy as np


def linear_constraints(model):
    """Equality rows (E, e) of the power balances and the bounds (lo, hi) for
    an oracle.Model, in the variable layout above."""
    g = model.grid
    B, L, G = model.B, model.L, model.G
    Y = model.admittance().T  # [8][L]: gii bii gij bij gji bji gjj bjj
    gii, bii, gij, bij, gji, bji, gjj, bjj = Y
    n = 2 * G + 2 * B + 2 * L
    iw, ith, iR, iI = 2 * G, 2 * G + B, 2 * G + 2 * B, 2 * G + 2 * B + L
    E = np.zeros((2 * B, n))
    e = np.zeros(2 * B)
    for q in range(G):
        i = int(g.gbus[q])
        E[i, q] += 1.0          # sum pg - sum p_ij - gs w = pd
        E[B + i, G + q] += 1.0  # sum qg - sum q_ij + bs w = qd
    for i in range(B):
        E[i, iw + i] -= g.gs[i]
        E[B + i, iw + i] += g.bs[i]
        e[i] = g.pd[i]
        e[B + i] = g.qd[i]
    for l in range(L):
        f, t = int(g.f[l]), int(g.t[l])
        # p_ij = gii w_i + gij wR + bij wI;  q_ij = -bii w_i - bij wR + gij wI
        E[f, iw + f] -= gii[l]; E[f, iR + l] -= gij[l]; E[f, iI + l] -= bij[l]
        E[B + f, iw + f] += bii[l]; E[B + f, iR + l] += bij[l]; E[B + f, iI + l] -= gij[l]
        # p_ji = gjj w_j + gji wR - bji wI;  q_ji = -bjj w_j - bji wR - gji wI
        E[t, iw + t] -= gjj[l]; E[t, iR + l] -= gji[l]; E[t, iI + l] += bji[l]
        E[B + t, iw + t] += bjj[l]; E[B + t, iR + l] += bji[l]; E[B + t, iI + l] += gji[l]
    lo = np.full(n, -np.inf)
    hi = np.full(n, np.inf)
    lo[:G], hi[:G] = g.pmin, g.pmax
    lo[G:2 * G], hi[G:2 * G] = g.qmin, g.qmax
    lo[iw:iw + B], hi[iw:iw + B] = np.asarray(g.vmin) ** 2, np.asarray(g.vmax) ** 2
    lo[ith:ith + B], hi[ith:ith + B] = -2 * math.pi, 2 * math.pi
    ref = np.flatnonzero(np.asarray(g.bus_type) == 3)
    lo[ith + ref] = hi[ith + ref] = 0.0
    return E, e, lo, hi


def project(model, x0, tol=1e-12, max_iter=200):
    """The exact projection of x0; returns (x, mu) with mu the balance
    multipliers.  Raises if the KKT check fails."""
    E, e, lo, hi = linear_constraints(model)
    x0 = np.asarray(x0, dtype=np.float64)
    m = E.shape[0]
    mu = np.zeros(m)

    def primal(mu):
        return np.clip(x0 - E.T @ mu, lo, hi)

    def dual(mu, x):
        return 0.5 * np.sum((x - x0) ** 2) + mu @ (E @ x - e)

    x = primal(mu)
    for _ in range(max_iter):
        gr = E @ x - e
        if np.max(np.abs(gr)) <= tol * (1.0 + np.max(np.abs(e))):
            break
        free = (x0 - E.T @ mu > lo) & (x0 - E.T @ mu < hi)
        H = (E[:, free] @ E[:, free].T)
        H += 1e-14 * (1.0 + np.trace(H) / m) * np.eye(m)
        step = np.linalg.solve(H, gr)  # Newton ascent direction of the concave dual
        g0 = dual(mu, x)
        a = 1.0
        while True:
            mu1 = mu + a * step
            x1 = primal(mu1)
            if dual(mu1, x1) >= g0 + 1e-4 * a * (gr @ step) or a < 1e-12:
                break
            a *= 0.5
        mu, x = mu1, x1
    # KKT: primal feasibility, stationarity x - x0 + E' mu = nu, nu a valid bound multiplier
    nu = x - x0 + E.T @ mu
    scale = 1.0 + np.max(np.abs(x0))
    assert np.max(np.abs(E @ x - e)) <= 1e-9 * (1.0 + np.max(np.abs(e)))
    assert np.all(x >= lo - 1e-12) and np.all(x <= hi + 1e-12)
    inner = (x > lo + 1e-12) & (x < hi - 1e-12)
    assert np.max(np.abs(nu[inner]), initial=0.0) <= 1e-8 * scale
    at_lo = (x <= lo + 1e-12) & ~(x >= hi - 1e-12)
    at_hi = (x >= hi - 1e-12) & ~(x <= lo + 1e-12)
    assert np.all(nu[at_lo] >= -1e-8 * scale) and np.all(nu[at_hi] <= 1e-8 * scale)
    return x, mu
