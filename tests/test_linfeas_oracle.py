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
