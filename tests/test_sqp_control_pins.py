"""Pins of the oracle's SQP control logic (Alg. 1; ratio test of Sec. II-C).

Alg. 1 prints the acceptance test (ared = phi_1(x) - phi_1(x + d) > 0 and
ared / (q(0) - q(d)) > 0) and only the inequalities Delta+ >= Delta on
acceptance and Delta+ <= Delta on rejection; the update rules themselves are
carried as comments in the algorithm: Delta+ = 2 Delta (read as capped at
Delta_max) after an accepted step on the trust-region boundary, and
Delta+ = 0.5 min(Delta, |d|_inf) after a rejection.  An accepted interior step
keeps Delta (the printed inequality with equality).

* the decision function on constructed values, against those rules;
* the oracle's full SQP trajectory, row by row, against a second driver of
  Alg. 1 written here from the same rules over the oracle's separately pinned
  building blocks (QP build, ADMM, step, merit, KKT measures), on runs chosen
  so that every branch of the rule occurs;
* invariants of every trajectory row that hold whatever the constants: the
  step respects the trust region (eq. TR), the printed inequalities, and the
  objective moves only on acceptance.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2310_13143_gb300 import gridgen as gg
from sqp_alg1 import alg1

# Runs on the 30-bus grid whose inexact QP solves (few ADMM iterations) and
# small radii make every branch of the rule occur.  Delta0 <= Delta_max, so
# the cap never lowers Delta below Delta0 on an accepted step.
# run A: rejections, boundary growth, the cap, interior steps, and steps
# with ared > 0 but a non-positive model reduction (merit penalty mu = 1e2)
RUN_A = dict(delta0=0.5, delta_max=0.5, max_iter=20, mu=1e2, eps=1e-4, max_sqp=25)
# run B: the paper's mu = 1e5; rejections, growth, the cap and interior steps
RUN_B = dict(delta0=0.25, delta_max=0.5, max_iter=60, mu=1e5, eps=1e-4, max_sqp=25)


@pytest.mark.parametrize("delta,dn,ared,pred,acc,new", [
    (1.0, 1.0, 3.0, 2.0, True, 2.0),        # boundary step accepted: doubled
    (1.0, 0.995, 3.0, 2.0, True, 2.0),      # within the 0.99 Delta boundary band
    (8.0, 8.0, 3.0, 2.0, True, 10.0),       # doubled, capped at Delta_max = 10
    (1.0, 0.5, 3.0, 2.0, True, 1.0),        # interior step accepted: unchanged
    (1.0, 0.98, 3.0, 2.0, True, 1.0),       # just inside the band: unchanged
    (1.0, 0.5, -3.0, 2.0, False, 0.25),     # merit increased: rejected, 0.5 min(Delta, |d|)
    (1.0, 1.0, 3.0, -2.0, False, 0.5),      # ared > 0 but pred < 0: the ratio is negative
    (1.0, 1.0, -3.0, -2.0, False, 0.5),     # ratio positive but ared < 0: rejected
    (1.0, 0.3, 3.0, 0.0, False, 0.15),      # no model reduction
    (1.0, 0.3, float("nan"), 2.0, False, 0.15),
    (1.0, 0.3, 3.0, float("inf"), False, 0.15),
    (0.4, 2.0, -1.0, 1.0, False, 0.2),      # rejected with |d| above Delta: 0.5 Delta
])
def test_trust_region_rule_on_constructed_values(delta, dn, ared, pred, acc, new):
    got_acc, got = oracle.tr_update(oracle.SqpOptions(delta_max=10.0), delta, dn, ared, pred)
    assert got_acc == acc
    assert got == pytest.approx(new, rel=1e-15)


def test_trust_region_rule_keeps_the_printed_inequalities():
    """Alg. 1: accepted => Delta+ >= Delta, rejected => Delta+ <= Delta, on random values."""
    rng = np.random.default_rng(11)
    o = oracle.SqpOptions(delta_max=10.0)
    for _ in range(2000):
        delta = 10 ** rng.uniform(-6, 1)
        dn = delta * rng.uniform(0, 1.0)
        ared, pred = rng.standard_normal(2) * 10 ** rng.uniform(-8, 3, 2)
        acc, nd = oracle.tr_update(o, delta, dn, ared, pred)
        assert acc == (ared > 0 and ared / pred > 0)
        assert (nd >= delta) if acc else (nd <= delta)
        assert nd <= max(delta, o.delta_max)


def _classify(h, delta0, delta_max):
    acc = h[:, 6] > 0
    prev = np.concatenate([[delta0], h[:-1, 7]])
    bound = acc & (h[:, 8] >= 0.99 * prev)
    capped = bound & (h[:, 7] == delta_max) & (2 * prev > delta_max)
    return dict(reject=~acc, grow=bound & ~capped, cap=capped, interior=acc & ~bound,
                ared_pos_pred_nonpos=(h[:, 9] > 0) & (h[:, 10] <= 0))


@pytest.mark.parametrize("run", [RUN_A, RUN_B], ids=["A", "B"])
def test_sqp_trajectory_follows_alg1(run):
    g = gg.grid_30bus()
    m = oracle.Model(g)
    o = oracle.SqpOptions(**run)
    got = m.sqp(o)["hist"]
    want = alg1(m, o)
    assert got.shape == want.shape
    # the same calls in the same order: identical numbers
    np.testing.assert_array_equal(got, want)
    kinds = _classify(got, o.delta0, o.delta_max)
    need = ["reject", "grow", "cap", "interior"] + (["ared_pos_pred_nonpos"] if run is RUN_A else [])
    for k in need:
        assert kinds[k].any(), f"run does not exercise '{k}'"
    # ared > 0 with pred <= 0 is always a rejection
    assert not (kinds["ared_pos_pred_nonpos"] & (got[:, 6] > 0)).any()


@pytest.mark.parametrize("run", [RUN_A, RUN_B, dict(max_sqp=30)], ids=["A", "B", "default"])
def test_sqp_trajectory_invariants(run):
    """Properties of every row that hold whatever the rule's constants."""
    g = gg.grid_30bus()
    m = oracle.Model(g)
    o = oracle.SqpOptions(**run)
    r = m.sqp(o)
    h = r["hist"]
    prev = np.concatenate([[o.delta0], h[:-1, 7]])
    acc = h[:, 6] > 0
    # eq. TR: the step of the QP solved with radius prev respects it
    assert (h[:, 8] <= prev * (1 + 1e-12)).all()
    # Alg. 1's printed inequalities
    assert (h[acc, 7] >= prev[acc]).all() and (h[~acc, 7] <= prev[~acc]).all()
    assert (h[:, 7] <= max(o.delta0, o.delta_max)).all()
    # the iterate, hence the objective, changes only on acceptance
    obj_prev = np.concatenate([[m.objective(m.flat_start())], h[:-1, 0]])
    assert (h[~acc, 0] == obj_prev[~acc]).all()
    assert r["accepted"] == int(acc.sum())
