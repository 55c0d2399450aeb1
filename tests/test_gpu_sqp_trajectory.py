"""The GPU's SQP trajectory (Alg. 1) against the oracle's, iteration by
iteration, in FP64: the same ADMM iteration counts and acceptance decisions,
and the trust-region radius, step norm, actual and predicted merit
reductions (Sec. II-C) to 1e-9 relative.

The FP64 sweep solves every line subproblem exactly (an active set
predicted in FP32, solved and checked in FP64, else the dual active-set
method), as the oracle does by enumeration, so the two follow the same path
up to rounding.  A line subproblem with no feasible point inside its box has
no unique answer -- the GPU treats its rows softly (the paper's augmented
Lagrangian), the oracle takes its least-violating working set -- so rows are
compared up to the first QP whose ADMM met one.

The runs are the ones that make every branch of the trust-region rule occur
on the 30-bus grid (rejections, boundary growth, the cap, interior steps,
ared > 0 with pred <= 0), the default settings on the 30-bus grid, the
benchmark's settings on the 2,000-bus grid, and the pinned runs of the
second-order correction and feasibility restoration (the future-work steps
of Alg. 1), including a grid of the batched workload that stalls without
restoration and is certified locally infeasible with it.
"""
import numpy as np
import pytest

import oracle
from paper_2310_13143_gb300 import binding, gridgen as gg
from sqp_alg1 import alg1
from test_sqp_control_pins import _classify

pytestmark = pytest.mark.gpu

RUNS = {
    "syn30_A": (gg.grid_30bus, dict(delta0=0.5, delta_max=0.5, max_iter=20, mu=1e2, eps=1e-4, max_sqp=25)),
    "syn30_B": (gg.grid_30bus, dict(delta0=0.25, delta_max=0.5, max_iter=60, mu=1e5, eps=1e-4, max_sqp=25)),
    "syn30_default": (gg.grid_30bus, dict(max_sqp=30)),
    "syn2000_bench": (gg.grid_2000bus, dict(tol=1e-4, max_sqp=20, eps=1e-3, max_iter=1000, rho=2e4)),
    # second-order correction and feasibility restoration (pinned oracle runs)
    "soc_accepted": (lambda: gg.grid_30bus(4), dict(delta0=0.25, delta_max=0.5, max_iter=60, mu=1e5, soc=1,
                                                    max_sqp=40)),
    "restore_and_back": (gg.grid_30bus, dict(delta0=0.25, delta_max=0.5, max_iter=60, mu=1e5, restore=1,
                                             max_sqp=40)),
    "restore_on_slow_progress": (lambda: gg.geometric_grid(60, seed=3),
                                 dict(delta0=0.25, delta_max=0.5, max_iter=30, mu=1e5, restore=1, max_sqp=40)),
    # an uneven grid of the batched workload that stalls without restoration
    "uneven240_restore": (lambda: gg.batched_uneven()[256 + 7],
                          dict(tol=1e-4, max_sqp=40, eps=1e-3, max_iter=1000, rho=2e4, soc=1, restore=1)),
}
# branches of the trust-region rule the compared rows must contain
NEED = {"syn30_A": ("reject", "grow", "cap", "interior", "ared_pos_pred_nonpos"),
        "syn30_B": ("reject", "grow", "cap", "interior")}


def _gpu_opts(o: oracle.SqpOptions):
    return binding.default_sqp(mu=o.mu, tol=o.tol, step_tol=o.step_tol, delta0=o.delta0, delta_max=o.delta_max,
                               delta_min=o.delta_min, max_sqp=o.max_sqp, soc=o.soc, restore=o.restore,
                               admm=dict(rho=o.rho, eps=o.eps, eps_dual=0.0, max_iter=o.max_iter,
                                         warm=o.warm_lambda))


# the same runs with the sweep in one thread-block cluster per instance (sweep_stages 4)
CLUSTER_RUNS = ("syn30_A", "syn30_default", "syn2000_bench", "soc_accepted", "restore_and_back")


@pytest.mark.parametrize("name,cluster", [(n, False) for n in RUNS] + [(n, True) for n in CLUSTER_RUNS])
def test_sqp_history_matches_oracle(name, cluster):
    make, run = RUNS[name]
    g = make()
    o = oracle.SqpOptions(**run)
    m = oracle.Model(g)
    line_fail = []
    want = alg1(m, o, line_fail)
    np.testing.assert_array_equal(want, m.sqp(o)["hist"])  # the second loop of Alg. 1 equals the oracle's own
    s = binding.Solver(g, precision="fp64")
    if cluster:
        s.tune(256, 0, 4)
    s.sqp_solve(_gpu_opts(o))
    got = s.get_history(0)
    res = s.get_residuals(0)
    s.close()
    bad = [k for k, n in enumerate(line_fail) if n > 0]
    n = bad[0] if bad else len(want)
    if not bad:
        assert res["sqp_iter"] == len(want) == len(got), (res["sqp_iter"], len(want))
    assert n >= min(len(want), 15), n
    got, want = got[:n], want[:n]
    for k in NEED.get(name, ()):
        assert _classify(want, o.delta0, o.delta_max)[k].any(), f"compared rows do not exercise '{k}'"
    # ADMM iterations per iteration, acceptance, correction outcome and phase: identical
    np.testing.assert_array_equal(got[:, 3], want[:, 3])
    np.testing.assert_array_equal(got[:, 6], want[:, 6])
    np.testing.assert_array_equal(got[:, 12], want[:, 11])
    np.testing.assert_array_equal(got[:, 13], want[:, 12])
    # trust radius after the update and step norm: relative 1e-9
    np.testing.assert_allclose(got[:, 7], want[:, 7], rtol=1e-9, atol=0)
    np.testing.assert_allclose(got[:, 8], want[:, 8], rtol=1e-9, atol=1e-13)
    # merit reductions: relative 1e-9 of the reduction, or 1e-11 of the
    # objective where the reduction itself is tiny (a reduction is the
    # difference of two merit values of the objective's size, and the line
    # subproblems are solved exactly by another method than the oracle's, so
    # the iterates part at the rounding level over the run)
    for col in (9, 10):
        tol = 1e-9 * np.abs(want[:, col]) + 1e-11 * np.abs(want[:, 0])
        assert (np.abs(got[:, col] - want[:, col]) <= tol).all(), (col, got[:, col], want[:, col])
    # objective, primal and dual measures after every iteration
    np.testing.assert_allclose(got[:, 0], want[:, 0], rtol=1e-10)
    acc = want[:, 6] > 0
    np.testing.assert_allclose(got[acc, 1], want[acc, 1], rtol=1e-6, atol=1e-10)
    np.testing.assert_allclose(got[acc, 2], want[acc, 2], rtol=1e-6, atol=1e-10)
    if not bad:
        assert res["result"] == m.sqp(o)["status"]
    if name == "soc_accepted":
        assert (got[:, 12] == 2).any()
    if name.startswith("restore") or name.endswith("restore"):
        assert got[:, 13].any()


def test_restoration_certifies_an_overloaded_two_bus_grid():
    """Load 5 p.u. against 2 + 2 p.u. of generation: the GPU's restoration ends
    'infeasible' at the least l1 violation (the 1 p.u. deficit), generators at
    Pmax, as the oracle's does."""
    g = gg.two_bus(lossless=True, pd2=5.0, qd2=0.2, pmax=(2.0, 2.0), rate=10.0)
    s = binding.Solver(g, precision="fp64")
    s.sqp_solve(binding.default_sqp(restore=1, max_sqp=60, admm=dict(rho=1e3, eps=1e-6, max_iter=20000)))
    res, sol = s.get_residuals(0), s.get_solution(0)
    s.close()
    assert res["result_name"] == "infeasible", res
    np.testing.assert_allclose(sol["pg"], [2.0, 2.0], atol=1e-6)
    x = np.concatenate([sol["pg"], sol["qg"], sol["vm"] ** 2, sol["va"], sol["wr"], sol["wi"]])
    np.testing.assert_allclose(oracle.Model(g).violations(x)[0], 1.0, atol=1e-5)
