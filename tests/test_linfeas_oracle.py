"""Pins of the linear feasibility projection oracle (oracle/linfeas.py,
Sec. II eq. linfeas) against routes other than itself: the oracle model's own
nonlinear balance function, scipy's SLSQP on the same problem, and two
properties every projection onto a convex set has (a feasible point is its
own projection; projections are non-expansive)."""
import numpy as np
import pytest

import oracle
from oracle import linfeas as olf
from paper_2310_13143_gb300 import gridgen as gg


def _start(m, rng, scale=0.05):
    x = m.flat_start()
    return x + scale * rng.standard_normal(x.size)


@pytest.mark.parametrize("name", ["syn30", "shunt_tap", "hub41"])
def test_balance_rows_equal_the_model_balance(name):
    g = {"syn30": gg.grid_30bus(), "hub41": gg.hub_grid(40),
         "shunt_tap": gg.grid_30bus().__class__(**{**gg.grid_30bus().__dict__, "gs": np.linspace(0, .03, 30),
                                                   "bs": np.linspace(.05, 0, 30), "tap": np.linspace(.95, 1.05, 41),
                                                   "shift": np.linspace(-.05, .05, 41)})}[name]
    m = oracle.Model(g)
    E, e, lo, hi = olf.linear_constraints(m)
    rng = np.random.default_rng(1)
    for _ in range(3):
        x = _start(m, rng, 0.2)
        _, bal = m.constraints(x)  # the oracle's nonlinear-model balance residual (p then q per bus)
        np.testing.assert_allclose(E @ x - e, np.concatenate([bal[:, 0], bal[:, 1]]), atol=1e-12)


def test_projection_matches_scipy_slsqp():
    from scipy.optimize import minimize

    m = oracle.Model(gg.grid_30bus())
    E, e, lo, hi = olf.linear_constraints(m)
    x0 = _start(m, np.random.default_rng(2))
    x, _ = olf.project(m, x0)
    bnds = [(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b) for a, b in zip(lo, hi)]
    res = minimize(lambda y: np.sum((y - x0) ** 2), np.clip(x0, lo, hi), jac=lambda y: 2 * (y - x0),
                   bounds=bnds, constraints=[{"type": "eq", "fun": lambda y: E @ y - e, "jac": lambda y: E}],
                   method="SLSQP", options=dict(ftol=1e-12, maxiter=3000))
    assert res.success
    np.testing.assert_allclose(x, res.x, atol=1e-9)
    assert np.sum((x - x0) ** 2) <= np.sum((res.x - x0) ** 2) + 1e-12


def test_projection_fixed_point_and_nonexpansive():
    m = oracle.Model(gg.geometric_grid(118, seed=7))
    rng = np.random.default_rng(3)
    a, b = _start(m, rng), _start(m, rng)
    pa, _ = olf.project(m, a)
    pb, _ = olf.project(m, b)
    again, _ = olf.project(m, pa)
    np.testing.assert_allclose(again, pa, atol=1e-10)
    assert np.linalg.norm(pa - pb) <= np.linalg.norm(a - b) * (1 + 1e-9)


def test_bounds_are_the_nlp_bounds():
    """The projection's bounds are those of eq. nlp (opfc1-4 and the
    reference angle): a random value lies inside exactly when the grid's own
    limits admit it; wR and wI are free.  Per-bus voltage bands, so that a
    bound taken from the wrong bus or left unsquared shows."""
    base = gg.grid_30bus()
    g = base.__class__(**{**base.__dict__, "vmin": np.linspace(0.90, 0.96, 30), "vmax": np.linspace(1.10, 1.04, 30)})
    m = oracle.Model(g)
    _, _, lo, hi = olf.linear_constraints(m)
    G, B, L = m.G, m.B, m.L
    rng = np.random.default_rng(41)
    ref = int(np.flatnonzero(g.bus_type == 3)[0])
    blocks = [(0, G, g.pmin, g.pmax, 4.0), (G, G, g.qmin, g.qmax, 2.0),
              (2 * G, B, g.vmin ** 2, g.vmax ** 2, 1.5), (2 * G + B, B, None, None, 8.0)]
    for o, n, bl, bu, span in blocks:
        for k in range(n):
            for val in rng.uniform(-span, span, 50):
                inside = lo[o + k] <= val <= hi[o + k]
                if bl is None:  # angles: [-2 pi, 2 pi], the reference held at 0
                    want = val == 0.0 if k == ref else -2 * np.pi <= val <= 2 * np.pi
                else:
                    want = bl[k] <= val <= bu[k]
                assert inside == want, (o, k, val)
        if bl is None:
            assert lo[o + ref] == hi[o + ref] == 0.0
    assert np.all(np.isinf(lo[2 * G + 2 * B:])) and np.all(np.isinf(hi[2 * G + 2 * B:]))
    assert lo.size == 2 * G + 2 * B + 2 * L
