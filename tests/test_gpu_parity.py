"""CUDA path vs the FP64 CPU oracle, through the C ABI, on the same seeded inputs.

* QP build (Alg. 1, eq. QPsub): every field, element by element, FP64.
* One ADMM iteration (Alg. 2) from the same random state: every coupling.
  The GPU solves each line subproblem by its augmented Lagrangian to 1e-11;
  the oracle solves it exactly, so the FP64 tolerance is 1e-7 relative to the
  state's scale.
* Converged QP solve: step and recovered multipliers.
* Full SQP: objective relative error <= 1e-5 and primal/dual infeasibility
  <= 1e-4 (the acceptance bar), FP64 and mixed precision.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2310_13143_gb300 import binding, gridgen as gg

pytestmark = pytest.mark.gpu


def _with(g, **kw):
    return g.__class__(**{**g.__dict__, **kw})


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


GRIDS = {
    "syn30": lambda: gg.grid_30bus(),
    "two_bus": lambda: gg.two_bus(lossless=False, rate=1.0),
    "syn30_shunt_tap": lambda: _with(gg.grid_30bus(), gs=np.linspace(0, 0.03, 30), bs=np.linspace(0.05, 0, 30),
                                     tap=np.linspace(0.95, 1.05, 41), shift=np.linspace(-0.05, 0.05, 41)),
    "syn30_nolimits": lambda: _with(gg.grid_30bus(), rate=np.zeros(41), angmin=np.full(41, -7.0),
                                    angmax=np.full(41, 7.0)),
    "syn118": lambda: gg.geometric_grid(118, seed=7),
    "hub41": lambda: gg.hub_grid(40),  # a bus with 40 branch ends (more than one warp task)
}


@pytest.mark.parametrize("name", list(GRIDS))
def test_build_matches_oracle(name):
    g = GRIDS[name]()
    rng = np.random.default_rng(5)
    m = oracle.Model(g)
    x = _perturbed(m, rng)
    pi = 50 * rng.standard_normal(4 * m.L)
    delta, rho = 0.3, 2e4
    ref = m.build(x, pi, delta, 1)
    s = binding.Solver(g)
    s.set_iterate(0, x, pi)
    s.build_qp(delta, rho, True)
    got = s.get_qp(0)
    for key in ("flow", "H", "aR", "aI", "bR", "bI", "QH", "gH", "F", "f0", "lo", "hi", "G", "grhs",
                "gd1", "gd2", "glp", "gup", "glq", "guq", "pdk", "qdk"):
        a, b = np.asarray(got[key]).reshape(-1), np.asarray(ref[key]).reshape(-1)
        b = np.where(np.abs(b) >= 1e29, np.sign(b) * 1e30, b)
        scale = max(1.0, np.abs(b[np.abs(b) < 1e29]).max(initial=0.0))
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * scale, err_msg=key)
    for key in ("alo", "ahi"):
        a, b = got[key], ref[key]
        fin = np.abs(b) < 1e29
        np.testing.assert_allclose(a[fin], b[fin], atol=1e-12)
        assert np.all(np.abs(a[~fin]) >= 1e29)


def _random_state(m, rng, rho):
    st = m.new_state(rho)
    st["zl"][...] = 0.02 * rng.standard_normal(st["zl"].shape)
    st["ll"][...] = 300 * rng.standard_normal(st["ll"].shape)
    st["zg"][...] = 0.02 * rng.standard_normal(st["zg"].shape)
    st["lg"][...] = 300 * rng.standard_normal(st["lg"].shape)
    # bus copies of w and theta are the bus values (one per bus)
    g = m.grid
    zb = 0.01 * rng.standard_normal((m.B, 2))
    zb[np.flatnonzero(g.bus_type == 3), 1] = 0.0
    st["zl"][:, 4], st["zl"][:, 5] = zb[g.f, 0], zb[g.f, 1]
    st["zl"][:, 6], st["zl"][:, 7] = zb[g.t, 0], zb[g.t, 1]
    st["zb"][...] = zb
    return st


def _gpu_state_from(st):
    return {"x": st["xl"], "z": st["zl"], "lam": st["ll"], "xg": st["xg"], "zg": st["zg"], "lg": st["lg"],
            "zb": st["zb"], "nu": st["nu"], "ul": st["ul"]}


@pytest.mark.parametrize("name", ["syn30", "syn30_shunt_tap", "syn118", "two_bus", "hub41"])
@pytest.mark.parametrize("iters", [1, 3])
def test_admm_iterations_match_oracle(name, iters):
    g = GRIDS[name]()
    rng = np.random.default_rng(11)
    rho = 2e4
    m = oracle.Model(g)
    x = _perturbed(m, rng, 0.02)
    pi = 20 * rng.standard_normal(4 * m.L)
    qp = m.build(x, pi, 0.2, 1)
    st = _random_state(m, rng, rho)
    s = binding.Solver(g)
    s.set_iterate(0, x, pi)
    s.build_qp(0.2, rho, True)
    s.set_admm_state(0, _gpu_state_from(st))
    st, _ = m.admm(qp, st, rho=rho, eps=0.0, max_iter=iters)
    s.admm_iterate(iters)
    got = s.get_admm_state(0)
    pairs = [("x", "xl"), ("z", "zl"), ("lam", "ll"), ("xg", "xg"), ("zg", "zg"), ("lg", "lg"), ("zb", "zb"),
             ("nu", "nu")]
    for gk, ok in pairs:
        a, b = got[gk], st[ok]
        scale = max(1.0, np.abs(b).max())
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-7 * scale, err_msg=f"{gk} after {iters} iterations")


def test_converged_qp_step_and_multipliers():
    g = gg.grid_30bus()
    m = oracle.Model(g)
    r = m.sqp(oracle.SqpOptions(max_sqp=2))
    x, pi = r["x"], r["pi"]
    # eps / rho must stay above the line solver's own tolerance (1e-11)
    delta, rho, eps = 0.5, 2e4, 1e-6
    qp = m.build(x, pi, delta, 1)
    st, info = m.admm(qp, rho=rho, eps=eps, max_iter=50000)
    d_ref, pi_ref = m.step(qp, st, x)
    s = binding.Solver(g)
    s.set_iterate(0, x, pi)
    s.admm_solve_qp(delta, binding.default_admm(rho=rho, eps=eps, max_iter=50000, warm=0))
    d, pi_new = s.get_step(0)
    res = s.get_residuals(0)
    assert res["r_inf"] <= eps and res["s_inf"] <= eps
    np.testing.assert_allclose(d, d_ref, atol=1e-6)
    np.testing.assert_allclose(pi_new, pi_ref, atol=1e-3 * max(1.0, np.abs(pi_ref).max()))


def _sqp_compare(g, precision, tol_obj=1e-5, **opt):
    m = oracle.Model(g)
    ref = m.sqp(oracle.SqpOptions(**opt))
    assert ref["status"] == 0
    s = binding.Solver(g, precision=precision)
    o = binding.default_sqp(admm={k: v for k, v in opt.items() if k in ("rho", "eps", "max_iter")},
                            **{k: v for k, v in opt.items() if k in ("tol", "max_sqp", "mu")})
    s.sqp_solve(o)
    res = s.get_residuals(0)
    sol = s.get_solution(0)
    assert res["result_name"] == "converged", res
    assert res["primal"] <= 1e-4 and res["dual"] <= 1e-4, res
    assert abs(sol["obj"] - ref["obj"]) <= tol_obj * abs(ref["obj"]), (sol["obj"], ref["obj"])
    return ref, res, sol


def test_sqp_fp64_30bus_matches_oracle():
    ref, res, sol = _sqp_compare(gg.grid_30bus(), "fp64")
    v = oracle.Model(gg.grid_30bus()).split(ref["x"])
    np.testing.assert_allclose(sol["pg"], v["pg"], atol=1e-3)


def test_sqp_mixed_30bus_matches_oracle():
    _sqp_compare(gg.grid_30bus(), "mixed")


def test_sqp_two_bus_closed_form():
    c2, c1, pd = (0.02, 0.05), (20.0, 22.0), 0.8
    g = gg.two_bus(lossless=True, c2=c2, c1=c1, pd2=pd)
    s = binding.Solver(g)
    s.sqp_solve(binding.default_sqp(tol=1e-7, admm=dict(rho=1e3, eps=1e-8, max_iter=100000)))
    res, sol = s.get_residuals(0), s.get_solution(0)
    assert res["result_name"] == "converged"
    S = 100.0
    p1 = (2 * c2[1] * S * S * pd + c1[1] * S - c1[0] * S) / (2 * S * S * (c2[0] + c2[1]))
    np.testing.assert_allclose(sol["pg"], [p1, pd - p1], atol=1e-6)


def test_batched_instances_match_single_solves():
    grids = [gg.grid_30bus(), gg.grid_30bus(4), gg.grid_30bus(5), gg.two_bus(lossless=False, rate=2.0)]
    s = binding.Solver(grids)
    s.sqp_solve()
    for k, g in enumerate(grids):
        ref = oracle.Model(g).sqp(oracle.SqpOptions())
        res, sol = s.get_residuals(k), s.get_solution(k)
        assert res["result_name"] == "converged", (k, res)
        assert abs(sol["obj"] - ref["obj"]) <= 1e-5 * abs(ref["obj"]), (k, sol["obj"], ref["obj"])


def test_barrier_timeout_is_reported_and_handle_stays_usable():
    g = gg.geometric_grid(2000, seed=2)
    s = binding.Solver(g)
    s.build_qp(1.0, 2e4, True)
    # a one-cycle wait limit makes CTAs give up at the first device-wide barrier
    with pytest.raises(binding.AcopfError) as ei:
        s.admm_iterate(5, binding.default_admm(spin_limit=1))
    assert ei.value.status == 4
    s.admm_iterate(2)  # the context is still usable
    st = s.get_admm_state(0)
    assert np.all(np.isfinite(st["x"]))


def test_residual_balancing_matches_oracle():
    """Adaptive penalty (residual balancing every 2 iterations): the GPU patches
    each line record in place, the oracle rebuilds its QPs; states agree."""
    g = gg.grid_30bus()
    rng = np.random.default_rng(3)
    rho = 2e4
    m = oracle.Model(g)
    x = _perturbed(m, rng, 0.02)
    qp = m.build(x, None, 0.2, 1)
    st = m.new_state(rho)
    s = binding.Solver(g)
    s.set_iterate(0, x, None)
    s.build_qp(0.2, rho, True)
    s.set_admm_state(0, _gpu_state_from(st))
    st, _ = m.admm(qp, st, rho=rho, eps=0.0, max_iter=8, rb_period=2)
    s.admm_iterate(8, binding.default_admm(rb_period=2))
    assert not np.allclose(st["rl"], rho)  # the penalty did change
    got = s.get_admm_state(0)
    for gk, ok in [("x", "xl"), ("z", "zl"), ("lam", "ll"), ("zb", "zb")]:
        a, b = got[gk], st[ok]
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-7 * max(1.0, np.abs(b).max()), err_msg=gk)


@pytest.mark.parametrize("name", ["syn30", "syn118", "syn30_shunt_tap", "hub41"])
@pytest.mark.parametrize("iters", [1, 3])
def test_admm_iterations_mixed_precision(name, iters):
    """FP32 sweep (branch tiles staged in shared memory by bulk copies) against
    the FP64 oracle: FP32 state within 3e-4 of each array's scale."""
    g = GRIDS[name]()
    rng = np.random.default_rng(11)
    rho = 2e4
    m = oracle.Model(g)
    x = _perturbed(m, rng, 0.02)
    pi = 20 * rng.standard_normal(4 * m.L)
    qp = m.build(x, pi, 0.2, 1)
    st = _random_state(m, rng, rho)
    s = binding.Solver(g, precision="mixed")
    s.set_iterate(0, x, pi)
    s.build_qp(0.2, rho, True)
    s.set_admm_state(0, _gpu_state_from(st))
    st, _ = m.admm(qp, st, rho=rho, eps=0.0, max_iter=iters)
    s.admm_iterate(iters)
    got = s.get_admm_state(0)
    for gk, ok in [("x", "xl"), ("z", "zl"), ("lam", "ll"), ("xg", "xg"), ("zg", "zg"), ("lg", "lg"), ("zb", "zb")]:
        a, b = got[gk], st[ok]
        np.testing.assert_allclose(a, b, rtol=0, atol=3e-4 * max(1.0, np.abs(b).max()), err_msg=f"{gk} {iters}")


def test_mixed_sweep_many_tiles_matches_fp64():
    """A grid large enough for many branch tiles per CTA: the FP32 sweep tracks
    the FP64 sweep over 20 iterations."""
    g = gg.geometric_grid(20000, seed=9, nbranch=27000, ngen=4000, nload=12000)
    out = {}
    for prec in ("fp64", "mixed"):
        s = binding.Solver(g, precision=prec)
        s.build_qp(0.5, 2e4, True)
        s.admm_iterate(20)
        out[prec] = s.get_admm_state(0)
        s.close()
    for key in ("x", "z", "zb"):
        a, b = out["mixed"][key], out["fp64"][key]
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-3 * max(1.0, np.abs(b).max()), err_msg=key)


def test_graph_replayed_solve_equals_eager_solve():
    """The CUDA-graph SQP loop replays the same kernels on the same data: every
    instance's result must equal the eager loop's, including instances that
    stop early while others keep going."""
    grids = [gg.grid_30bus(), gg.two_bus(), gg.geometric_grid(118, seed=11)]
    for prec in ("fp64", "mixed"):
        opts = binding.default_sqp(tol=1e-4, max_sqp=30, admm=dict(rho=2e4, max_iter=800, eps=1e-4,
                                                                   eps_dual=5e-3 if prec == "mixed" else 0.0))
        a = binding.Solver(grids, precision=prec)
        a.sqp_solve(opts)
        b = binding.Solver(grids, precision=prec)
        for check in (1, 3):
            b.sqp_solve_graph(opts, check_every=check)
            for k in range(len(grids)):
                ra, rb = a.get_residuals(k), b.get_residuals(k)
                assert ra["sqp_iter"] == rb["sqp_iter"] and ra["admm_iter"] == rb["admm_iter"]
                assert ra["result"] == rb["result"]
                xa, _ = a.get_iterate(k)
                xb, _ = b.get_iterate(k)
                np.testing.assert_array_equal(xa, xb)
        a.close()
        b.close()


def test_autotune_applies_and_caches_a_shape(tmp_path):
    cache = str(tmp_path / "tune.json")
    grids = [gg.grid_30bus()] * 4
    s = binding.Solver(grids, precision="mixed")
    shape, us = s.autotune(cache, iters=20)
    assert shape[0] in (64, 128, 192, 224, 256) and shape[1] in (0, 1) and shape[2] in (0, 1, 2, 3, 4) and us > 0
    import json
    entries = json.load(open(cache))
    assert len(entries) == 1 and entries[0]["block_threads"] == shape[0]
    shape2, us2 = s.autotune(cache, iters=20)
    assert shape2 == shape and us2 == -1.0
    # the tuned handle still solves correctly
    s.sqp_solve(binding.default_sqp(tol=1e-4, admm=dict(rho=2e4, max_iter=1000, eps=1e-4, eps_dual=5e-3)))
    assert all(s.get_residuals(k)["result_name"] == "converged" for k in range(4))
    s.close()


def test_mixed_sweep_launch_shapes_agree():
    """The FP32 sweep reads branch records from shared-memory tiles (one or two
    buffers) or in place from global memory, with any CTA size: the same
    arithmetic on the same values, so the state after a fixed number of
    iterations must be identical.  The resident form (records held in
    registers) and the cluster-per-instance form are separately compiled
    kernels in which the compiler may contract multiply-adds differently:
    they must agree to 1e-4 of each array's scale (FP32 rounding carried
    over 25 iterations)."""
    grids = [gg.geometric_grid(118, seed=7), gg.grid_30bus(), gg.hub_grid(40)]
    ref = None
    for bt, st in [(256, 1), (256, 0), (128, 2), (64, 0), (96, 1), (256, 3), (64, 3), (32, 3), (256, 4), (64, 4)]:
        s = binding.Solver(grids, precision="mixed")
        s.tune(bt, 0, st)
        s.build_qp(1.0, 2e4, True)
        s.admm_iterate(25, binding.default_admm())
        got = [s.get_admm_state(k) for k in range(len(grids))]
        s.close()
        if ref is None:
            ref = got
            continue
        for a, b in zip(ref, got):
            for key in ("x", "z", "lam", "xg", "zg", "lg", "zb", "nu", "ul"):
                if st >= 3:
                    # a kernel of its own: the compiler may fuse multiply-adds differently there
                    np.testing.assert_allclose(a[key], b[key], rtol=0, atol=1e-4 * max(1.0, np.abs(a[key]).max()),
                                               err_msg=f"{bt}:{st}:{key}")
                else:
                    np.testing.assert_array_equal(a[key], b[key], err_msg=f"{bt}:{st}:{key}")


@pytest.mark.parametrize("name", ["syn30", "syn30_shunt_tap", "syn118", "hub41", "two_bus"])
def test_linear_projection_matches_oracle(name):
    """acopf_project_linear (eq. linfeas) against the exact projection of the
    oracle: every instance of a two-instance handle, from perturbed starts."""
    from oracle import linfeas as olf

    g = GRIDS[name]()
    m = oracle.Model(g)
    rng = np.random.default_rng(5)
    starts = [_perturbed(m, rng, 0.05), _perturbed(m, rng, 0.2)]
    s = binding.Solver([g, g], precision="fp64")
    for k, x0 in enumerate(starts):
        s.set_iterate(k, x0)
    it, r, sres = s.project_linear(rho=0.5, eps=1e-10, max_iter=40000)
    assert r <= 1e-10 and sres <= 1e-10, (it, r, sres)
    E, e, lo, hi = olf.linear_constraints(m)
    for k, x0 in enumerate(starts):
        want, _ = olf.project(m, x0)
        got, _ = s.get_iterate(k)
        # the ADMM residual bound 1e-10 leaves the point within ~1e-8 of the projection
        np.testing.assert_allclose(got, want, atol=2e-7)
        assert np.max(np.abs(E @ got - e)) <= 1e-6
        assert np.all(got >= lo - 1e-12) and np.all(got <= hi + 1e-12)
    s.close()


def test_fp64_sweep_resident_records_agree():
    """The FP64 sweep with records held in registers, or with one cluster per
    instance, gives the same state as with records read in place, to the
    rounding of a separately compiled kernel (1e-9 of each array's scale)."""
    grids = [gg.geometric_grid(118, seed=7), gg.grid_30bus(), gg.hub_grid(40)]
    ref = None
    for bt, st in [(256, 0), (256, 3), (64, 3), (256, 4)]:
        s = binding.Solver(grids, precision="fp64")
        s.tune(bt, 0, st)
        s.build_qp(1.0, 2e4, True)
        s.admm_iterate(25, binding.default_admm())
        got = [s.get_admm_state(k) for k in range(len(grids))]
        s.close()
        if ref is None:
            ref = got
            continue
        for a, b in zip(ref, got):
            for key in a:
                if st >= 3:
                    np.testing.assert_allclose(a[key], b[key], rtol=0, atol=1e-9 * max(1.0, np.abs(a[key]).max()),
                                               err_msg=f"{key} threads {bt} mode {st}")
                else:
                    np.testing.assert_array_equal(a[key], b[key], err_msg=f"{key} threads {bt} mode {st}")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cluster_sweep_solves_like_the_device_wide_sweep(prec):
    """Sweep mode 4 (one thread-block cluster per instance, hardware cluster
    barriers, residual maxima combined in distributed shared memory) against
    the device-wide sweep: full SQP solves of a batch whose instances stop
    their QPs at different ADMM iterations, including a 2,000-bus grid that
    spreads over a 16-CTA cluster with several branches per thread."""
    grids = [gg.grid_30bus(), gg.two_bus(), gg.geometric_grid(118, seed=11), gg.hub_grid(40),
             gg.grid_2000bus()]
    opts = binding.default_sqp(tol=1e-4, max_sqp=8, admm=dict(rho=2e4, max_iter=600, eps=1e-4,
                                                              eps_dual=5e-3 if prec == "mixed" else 0.0))
    out = []
    for bt, st in ((256, 0), (128, 4)):
        s = binding.Solver(grids, precision=prec)
        s.tune(bt, 0, st)
        s.sqp_solve_graph(opts, check_every=2)
        out.append([(s.get_residuals(k), s.get_solution(k)["obj"]) for k in range(len(grids))])
        s.close()
    for (ra, oa), (rb, ob) in zip(*out):
        assert ra["result"] == rb["result"], (ra, rb)
        np.testing.assert_allclose(ob, oa, rtol=1e-9 if prec == "fp64" else 1e-6)
        if prec == "fp64":
            assert ra["sqp_iter"] == rb["sqp_iter"]


def test_cluster_sweep_with_state_in_shared_memory():
    """Grids with no bus of more than 32 couplings, a cluster that covers each
    of them: the FP32 cluster sweep keeps the state it exchanges (x one way,
    z and lambda the other) in distributed shared memory and writes it back
    at the end.  Its state after a fixed number of iterations matches the
    device-wide sweep to FP32 rounding, and so does a full SQP solve."""
    grids = [gg.grid_30bus(), gg.two_bus(), gg.geometric_grid(118, seed=11), gg.grid_2000bus()]
    ref = None
    for bt, st in ((256, 0), (256, 4), (224, 4)):
        s = binding.Solver(grids, precision="mixed")
        s.tune(bt, 0, st)
        s.build_qp(1.0, 2e4, True)
        s.admm_iterate(25, binding.default_admm())
        got = [s.get_admm_state(k) for k in range(len(grids))]
        s.close()
        if ref is None:
            ref = got
            continue
        for a, b in zip(ref, got):
            for key in ("x", "z", "lam", "xg", "zg", "lg", "zb", "nu", "ul"):
                np.testing.assert_allclose(b[key], a[key], rtol=0, atol=1e-4 * max(1.0, np.abs(a[key]).max()),
                                           err_msg=f"{bt}:{st}:{key}")
    # enough SQP iterations that no instance sits at the limit: which side of
    # it an FP32 run ends on is a matter of rounding
    opts = binding.default_sqp(tol=1e-4, max_sqp=20, admm=dict(rho=2e4, max_iter=600, eps=1e-4, eps_dual=5e-3))
    out = []
    for st in (0, 4):
        s = binding.Solver(grids, precision="mixed")
        s.tune(256, 0, st)
        s.sqp_solve_graph(opts, check_every=2)
        out.append([(s.get_residuals(k), s.get_solution(k)["obj"]) for k in range(len(grids))])
        s.close()
    for (ra, oa), (rb, ob) in zip(*out):
        assert ra["result"] == rb["result"], (ra, rb)
        np.testing.assert_allclose(ob, oa, rtol=1e-6)


def test_cluster_sweep_with_correction_and_restoration():
    """The cluster forms under the SQP's second-order correction and
    feasibility restoration: in a correction pass only the instances whose
    step was rejected run, so the clusters of the others return at once.  A
    batch with a grid that restoration certifies infeasible, an overloaded
    two-bus grid and the 30-bus grid ends the same in the cluster form as in
    the device-wide form (mixed precision, results to FP32 rounding)."""
    grids = [gg.batched_uneven()[256 + 7], gg.grid_30bus(),
             gg.two_bus(lossless=True, pd2=5.0, qd2=0.2, pmax=(2.0, 2.0), rate=10.0)]
    opts = binding.default_sqp(tol=1e-4, max_sqp=40, soc=1, restore=1,
                               admm=dict(rho=2e4, max_iter=1000, eps=1e-3, eps_dual=5e-3))
    out = []
    for st in (0, 4):
        s = binding.Solver(grids, precision="mixed")
        s.tune(256, 0, st)
        s.sqp_solve_graph(opts, check_every=2)
        out.append([(s.get_residuals(k), s.get_solution(k)["obj"]) for k in range(len(grids))])
        s.close()
    for k, ((ra, oa), (rb, ob)) in enumerate(zip(*out)):
        assert ra["result_name"] == rb["result_name"], (k, ra, rb)
        if ra["result_name"] == "converged":
            np.testing.assert_allclose(ob, oa, rtol=1e-6)
        else:
            np.testing.assert_allclose(rb["primal"], ra["primal"], rtol=1e-3)
