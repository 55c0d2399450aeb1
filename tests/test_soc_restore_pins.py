"""Pins of the oracle's second-order correction and feasibility restoration,
the two steps the paper names as future work for Alg. 1 (Sec. II-D).

Second-order correction.  After a rejected step d, the QP is rebuilt at x
with every nonlinear constraint's value replaced by c(x + d) - grad c(x)' d,
so that its linearised constraints at a step d' read
c(x + d) + grad c(x)'(d' - d).  Pinned against that definition with the
constraint values from their own evaluation at x + d and gradients from
central differences (no use of the elimination or the QP's formulas).

Feasibility restoration.  On a stall above the primal tolerance, or when the
violation stops falling, the objective is dropped until the violation is
within tol; a stall during restoration is local infeasibility.  Pinned on a
two-bus grid whose load exceeds its generation by a known amount (the
restoration must end infeasible with the l1 violation equal to the deficit
and both generators at Pmax), and trajectories against the second driver of
Alg. 1 on runs where the correction is accepted and restoration starts and
ends.
"""
import numpy as np
import pytest

import oracle
from paper_2310_13143_gb300 import gridgen as gg
from sqp_alg1 import alg1


def _perturbed(m, rng, scale=0.04):
    x = m.flat_start()
    v = m.split(x)
    v["pg"][:] += scale * rng.standard_normal(m.G)
    v["qg"][:] += scale * rng.standard_normal(m.G)
    v["w"][:] = 1.0 + scale * rng.standard_normal(m.B)
    v["th"][:] = scale * rng.standard_normal(m.B)
    v["th"][np.flatnonzero(m.grid.bus_type == 3)] = 0.0
    v["wr"][:] = 1.0 + scale * rng.standard_normal(m.L)
    v["wi"][:] = scale * rng.standard_normal(m.L)
    return x


def _grad_fd(m, x, rows, h=1e-6):
    """Central differences of the branch constraints c11..c14 (L x 4) at x."""
    n = x.size
    gr = np.zeros((n,) + rows.shape)
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        gr[k] = (m.constraints(x + e)[0] - m.constraints(x - e)[0]) / (2 * h)
    return gr


@pytest.mark.parametrize("name", ["syn30", "syn30_shunt_tap"])
def test_soc_qp_linearises_the_constraint_values_at_x_plus_d(name):
    g = gg.grid_30bus()
    if name == "syn30_shunt_tap":
        g = g.__class__(**{**g.__dict__, "gs": np.linspace(0, 0.03, 30), "bs": np.linspace(0.05, 0, 30),
                           "tap": np.linspace(0.95, 1.05, 41), "shift": np.linspace(-0.05, 0.05, 41)})
    m = oracle.Model(g)
    rng = np.random.default_rng(17)
    x = _perturbed(m, rng)
    d = 0.05 * rng.standard_normal(x.size)
    m.split(d)["th"][np.flatnonzero(g.bus_type == 3)] = 0.0  # the reference angle does not move
    qp = m.build(x, None, 1.0, 1, dsoc=d)
    c_xd = m.constraints(x + d)[0]            # c(x + d), evaluated directly
    c_x = m.constraints(x)[0]
    J = _grad_fd(m, x, c_x)                   # grad c(x) by central differences
    s = m.split(np.arange(x.size))
    for _ in range(3):
        # a step d' through the QP's own elimination at random dbar'
        db = 0.03 * rng.standard_normal((m.L, 4))
        dp = np.zeros(x.size)
        for l in range(m.L):
            i, j = g.f[l], g.t[l]
            dp[s["w"][i]], dp[s["th"][i]], dp[s["w"][j]], dp[s["th"][j]] = db[l]
        dp[s["th"][np.flatnonzero(g.bus_type == 3)]] = 0.0
        dbar = np.stack([dp[s["w"][g.f]], dp[s["th"][g.f]], dp[s["w"][g.t]], dp[s["th"][g.t]]], axis=1)
        dp[s["wr"]] = (qp["aR"] * dbar).sum(1) + qp["bR"]
        dp[s["wi"]] = (qp["aI"] * dbar).sum(1) + qp["bI"]
        lin = c_xd + np.einsum("nlr,n->lr", J, dp - d)
        # opfc11, opfc12: equalities met by the elimination
        np.testing.assert_allclose(lin[:, :2], 0.0, atol=1e-7)
        # line limits: the QP row's slack equals the linearisation at x + d
        G = qp["G"].reshape(m.L, 2, 4)
        slack = qp["grhs"].reshape(m.L, 2) - np.einsum("lec,lc->le", G, dbar)
        on = g.rate > 0
        np.testing.assert_allclose(slack[on], lin[on][:, 2:], rtol=1e-7, atol=1e-7)


def test_soc_qp_without_a_step_is_the_ordinary_qp():
    m = oracle.Model(gg.grid_30bus())
    x = _perturbed(m, np.random.default_rng(3))
    a, b = m.build(x, None, 0.5, 1), m.build(x, None, 0.5, 1, dsoc=np.zeros(x.size))
    for k in ("bR", "bI", "grhs", "gH", "f0", "QH", "F"):
        np.testing.assert_allclose(b[k], a[k], rtol=1e-14, atol=1e-14, err_msg=k)


def test_restoration_certifies_an_overloaded_two_bus_grid():
    """Load 5 p.u. against 2 + 2 p.u. of generation over a lossless line: no
    feasible point exists; the least l1 violation is the 1 p.u. deficit,
    with both generators at Pmax."""
    g = gg.two_bus(lossless=True, pd2=5.0, qd2=0.2, pmax=(2.0, 2.0), rate=10.0)
    m = oracle.Model(g)
    o = oracle.SqpOptions(restore=1, max_sqp=60, rho=1e3, eps=1e-6, max_iter=20000)
    r = m.sqp(o)
    assert r["status"] == 5
    assert r["hist"][:, 12].any()  # the restoration phase ran
    np.testing.assert_allclose(m.split(r["x"])["pg"], [2.0, 2.0], atol=1e-6)
    np.testing.assert_allclose(m.violations(r["x"])[0], 1.0, atol=1e-6)
    # without restoration the same point ends as a plain stall
    assert m.sqp(oracle.SqpOptions(restore=0, max_sqp=60, rho=1e3, eps=1e-6, max_iter=20000))["status"] == 2


RUNS = {
    # the corrected step is accepted
    "soc_accepted": (lambda: gg.grid_30bus(4), dict(delta0=0.25, delta_max=0.5, max_iter=60, mu=1e5, soc=1)),
    # restoration starts on lost progress and hands back to the SQP
    "restore_and_back": (gg.grid_30bus, dict(delta0=0.25, delta_max=0.5, max_iter=60, mu=1e5, restore=1)),
    "restore_back_twice": (lambda: gg.two_bus(lossless=False, rate=1.0),
                           dict(delta0=1.0, delta_max=10.0, max_iter=30, mu=1e3, restore=1)),
    # restoration stalls: locally infeasible with these settings
    "restore_stalls": (gg.grid_30bus, dict(delta0=0.5, delta_max=0.5, max_iter=20, mu=1e2, soc=1, restore=1)),
    # the violation falls, but by less than a tenth over five iterations: restoration starts
    "restore_on_slow_progress": (lambda: gg.geometric_grid(60, seed=3),
                                 dict(delta0=0.25, delta_max=0.5, max_iter=30, mu=1e5, restore=1)),
    # a corrected step whose own QP predicts no reduction: judged against the original step's model
    "soc_original_model": (lambda: gg.two_bus(lossless=False, rate=1.0),
                           dict(delta0=0.25, delta_max=0.5, max_iter=30, mu=1e5, soc=1)),
}


@pytest.mark.parametrize("name", list(RUNS))
def test_trajectory_with_correction_and_restoration_follows_alg1(name):
    make, run = RUNS[name]
    m = oracle.Model(make())
    o = oracle.SqpOptions(eps=1e-4, max_sqp=40, **run)
    r = m.sqp(o)
    h = r["hist"]
    np.testing.assert_array_equal(h, alg1(m, o))
    phases = "".join("R" if v else "." for v in h[:, 12])
    if name == "soc_accepted":
        assert (h[:, 11] == 2).any()
    if name.startswith("restore_and_back") or name == "restore_back_twice":
        assert "R." in phases
    if name == "restore_stalls":
        assert r["status"] == 5 and phases.endswith("R")
    # restoration rows: the merit has no objective part, so the step's model
    # reduction comes from the violation alone (pred <= mu h(x))
    acc = h[:, 6] > 0
    assert (h[acc & (h[:, 12] > 0), 10] > 0).all()
