"""Pins of the FP64 CPU oracle against things other than itself.

Each test checks one oracle function against an independent route to the
same quantity: nodal complex-power arithmetic, finite differences of the
constraint functions, closed forms, scipy's solvers, or brute force on tiny
problems.  A dropped term, wrong sign, swapped index or transposed operand in
the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2310_13143_gb300 import gridgen as gg

RNG = np.random.default_rng(1234)


def _perturbed_point(m, scale=0.05, rng=RNG):
    """A point near flat start with w, theta, wR, wI moved independently (so
    that c11 and c12 are not satisfied and every Hessian term is exercised)."""
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


# --------------------------------------------------------------------------
# model: flows (eq. acopf_pf) and balances (opfc5-6) against nodal arithmetic
# --------------------------------------------------------------------------
def _ybus_injections(g, V):
    """Complex bus injections S = V conj(Ybus V) with Ybus assembled from the
    standard pi-model branch stamps (series y, charging b/2 at each end,
    off-nominal tap t e^{j shift} on the from side)."""
    n = g.nbus
    Y = np.zeros((n, n), complex)
    for l in range(g.nbranch):
        y = 1.0 / complex(g.r[l], g.x[l])
        a = g.tap[l] * np.exp(1j * g.shift[l])
        i, j = g.f[l], g.t[l]
        Y[i, i] += (y + 0.5j * g.b[l]) / abs(a) ** 2
        Y[j, j] += y + 0.5j * g.b[l]
        Y[i, j] += -y / np.conj(a)
        Y[j, i] += -y / a
    Y += np.diag(g.gs + 1j * g.bs)
    return V * np.conj(Y @ V)


@pytest.mark.parametrize("tapshift", [False, True])
def test_balance_matches_nodal_injections(tapshift):
    g = gg.grid_30bus()
    if tapshift:
        g = g.__class__(**{**g.__dict__, "tap": 1 + 0.05 * RNG.standard_normal(g.nbranch),
                           "shift": 0.1 * RNG.standard_normal(g.nbranch),
                           "gs": 0.02 * RNG.random(g.nbus), "bs": 0.05 * RNG.random(g.nbus)})
    m = oracle.Model(g)
    vm = 1 + 0.03 * RNG.standard_normal(g.nbus)
    va = 0.1 * RNG.standard_normal(g.nbus)
    V = vm * np.exp(1j * va)
    x = m.flat_start()
    v = m.split(x)
    v["w"][:] = vm ** 2
    v["th"][:] = va
    v["wr"][:] = vm[g.f] * vm[g.t] * np.cos(va[g.f] - va[g.t])
    v["wi"][:] = vm[g.f] * vm[g.t] * np.sin(va[g.f] - va[g.t])
    v["pg"][:] = RNG.random(g.ngen)
    v["qg"][:] = RNG.random(g.ngen)
    c4, bal = m.constraints(x)
    S = _ybus_injections(g, V)
    gen = np.zeros(g.nbus, complex)
    np.add.at(gen, g.gbus, v["pg"] + 1j * v["qg"])
    expect = gen - (g.pd + 1j * g.qd) - S  # balance = generation - load - injection into network
    np.testing.assert_allclose(bal[:, 0], expect.real, atol=1e-12)
    np.testing.assert_allclose(bal[:, 1], expect.imag, atol=1e-12)
    # at a consistent point c11 and c12 vanish (wR, wI = v_i v_j cos/sin)
    np.testing.assert_allclose(c4[:, :2], 0.0, atol=1e-14)


def test_two_bus_lossless_flow_closed_form():
    g = gg.two_bus(lossless=True)
    m = oracle.Model(g)
    x = m.flat_start()
    v = m.split(x)
    d = 0.2
    v["th"][:] = [0.0, -d]
    v["wr"][:] = math.cos(d)
    v["wi"][:] = math.sin(d)
    fl = m.flows(x)[0]
    # p_12 = V1 V2 sin(delta) / x,  p_21 = -p_12,  q_12 = (V1^2 - V1 V2 cos delta) / x
    assert fl[0] == pytest.approx(math.sin(d) / 0.1, rel=1e-14)
    assert fl[2] == pytest.approx(-math.sin(d) / 0.1, rel=1e-14)
    assert fl[1] == pytest.approx((1 - math.cos(d)) / 0.1, rel=1e-12)
    assert fl[3] == pytest.approx((1 - math.cos(d)) / 0.1, rel=1e-12)


# --------------------------------------------------------------------------
# QP build (Alg. 1, eq. QPsub): Hessian, elimination, flow maps, boxes
# --------------------------------------------------------------------------
def _lagrangian_ij(m, x, pi, l):
    c4, _ = m.constraints(x)
    return float(np.dot(pi[4 * l:4 * l + 4], c4[l]))


def _z_index(m, l):
    g = m.grid
    o = np.cumsum([0, m.G, m.G, m.B, m.B, m.L, m.L])
    i, j = g.f[l], g.t[l]
    return [o[2] + i, o[3] + i, o[4] + l, o[5] + l, o[2] + j, o[3] + j]


def test_hessian_matches_finite_differences_of_constraints():
    g = gg.grid_30bus()
    m = oracle.Model(g)
    x = _perturbed_point(m)
    pi = 10 * RNG.standard_normal(4 * m.L)
    qp = m.build(x, pi, 1.0, 1)
    h = 1e-4
    for l in [0, 7, 23, 40]:
        idx = _z_index(m, l)
        H = qp["H"][l].reshape(6, 6)
        Hfd = np.zeros((6, 6))
        for a in range(6):
            for b in range(6):
                def L(da, db):
                    y = x.copy()
                    y[idx[a]] += da
                    y[idx[b]] += db
                    return _lagrangian_ij(m, y, pi, l)
                Hfd[a, b] = (L(h, h) - L(h, -h) - L(-h, h) + L(-h, -h)) / (4 * h * h)
        np.testing.assert_allclose(H, Hfd, atol=2e-5 * (1 + np.abs(H).max()))


def _grad_c(m, x, l, k, h=1e-6):
    idx = _z_index(m, l)
    out = np.zeros(6)
    for a in range(6):
        y1 = x.copy(); y1[idx[a]] += h
        y0 = x.copy(); y0[idx[a]] -= h
        out[a] = (m.constraints(y1)[0][l, k] - m.constraints(y0)[0][l, k]) / (2 * h)
    return out


def test_elimination_satisfies_linearised_c11_c12():
    g = gg.grid_30bus()
    m = oracle.Model(g)
    x = _perturbed_point(m)
    qp = m.build(x, None, 1.0, 1)
    c4, _ = m.constraints(x)
    for l in [0, 5, 17, 33]:
        db = 0.05 * RNG.standard_normal(4)
        dR = qp["aR"][l] @ db + qp["bR"][l]
        dI = qp["aI"][l] @ db + qp["bI"][l]
        z = np.array([db[0], db[1], dR, dI, db[2], db[3]])
        for k in (0, 1):
            lin = c4[l, k] + _grad_c(m, x, l, k) @ z
            assert abs(lin) < 1e-8, (l, k, lin)


def test_flow_maps_match_flow_change():
    g = gg.grid_30bus()
    m = oracle.Model(g)
    x = _perturbed_point(m)
    qp = m.build(x, None, 1.0, 1)
    f0 = m.flows(x)
    for l in [1, 9, 30]:
        db = 0.05 * RNG.standard_normal(4)
        y = x.copy()
        idx = _z_index(m, l)
        dR = qp["aR"][l] @ db + qp["bR"][l]
        dI = qp["aI"][l] @ db + qp["bI"][l]
        for k, val in zip(idx, [db[0], db[1], dR, dI, db[2], db[3]]):
            y[k] += val
        # flows are linear in (w, wR, wI): the change is exact
        np.testing.assert_allclose(qp["F"][l].reshape(4, 4) @ db + qp["f0"][l], m.flows(y)[l] - f0[l], atol=1e-12)
        # Q_H and g_H: the quadratic form of the Hessian along the eliminated direction
        H = qp["H"][l].reshape(6, 6)
        A = np.zeros((6, 4)); A[0, 0] = A[1, 1] = A[4, 2] = A[5, 3] = 1
        A[2] = qp["aR"][l]; A[3] = qp["aI"][l]
        b = np.array([0, 0, qp["bR"][l], qp["bI"][l], 0, 0])
        z = A @ db + b
        lhs = 0.5 * db @ qp["QH"][l].reshape(4, 4) @ db + qp["gH"][l] @ db + 0.5 * b @ H @ b
        assert lhs == pytest.approx(0.5 * z @ H @ z, rel=1e-12, abs=1e-14)


def test_line_limit_rows_are_linearised_limits():
    g = gg.grid_30bus()
    m = oracle.Model(g)
    x = _perturbed_point(m)
    qp = m.build(x, None, 1.0, 1)
    c4, _ = m.constraints(x)
    for l in [2, 11]:
        db = 0.05 * RNG.standard_normal(4)
        idx = _z_index(m, l)
        dR = qp["aR"][l] @ db + qp["bR"][l]
        dI = qp["aI"][l] @ db + qp["bI"][l]
        z = np.array([db[0], db[1], dR, dI, db[2], db[3]])
        for e, k in ((0, 2), (1, 3)):
            lin = c4[l, k] + _grad_c(m, x, l, k) @ z     # c + grad c . d >= 0
            row = qp["G"][l].reshape(2, 4)[e] @ db - qp["grhs"][l, e]  # <= 0
            assert row == pytest.approx(-lin, rel=1e-6, abs=1e-8)


def test_qp_rows_are_the_shifted_nlp_constraints():
    """The QP of eq. QPsub at x, on a grid with shunts, taps and phase shifts:
    the balance rows' right-hand sides are minus the (linear) balances at x;
    a step d lies in a box exactly when x + d meets the NLP's bounds and
    |d| <= delta; and it meets an angle row exactly when x + d meets the
    angle-difference limit.  Membership is tested on random steps, with the
    NLP side evaluated from its own definition."""
    base = gg.grid_30bus()
    g = base.__class__(**{**base.__dict__, "gs": np.linspace(0, 0.03, 30), "bs": np.linspace(0.05, 0, 30),
                          "tap": np.linspace(0.95, 1.05, 41), "shift": np.linspace(-0.05, 0.05, 41),
                          "vmin": np.linspace(0.90, 0.96, 30), "vmax": np.linspace(1.10, 1.04, 30)})
    m = oracle.Model(g)
    rng = np.random.default_rng(23)
    x = _perturbed_point(m, 0.05, rng)
    v = m.split(x)
    # points near the bounds (each bus has its own band), so that both sides of
    # every box are exercised
    v["pg"][::2] = g.pmax[::2] - 0.01
    v["w"][::3] = g.vmin[::3] ** 2 + 0.02
    v["w"][1::3] = g.vmax[1::3] ** 2 - 0.02
    delta = 0.05
    qp = m.build(x, None, delta, 1)
    _, bal = m.constraints(x)
    np.testing.assert_allclose(qp["pdk"], -bal[:, 0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(qp["qdk"], -bal[:, 1], rtol=0, atol=1e-13)

    def same_membership(lo, hi, val, lb, ub, n=400):
        for _ in range(n):
            d = rng.uniform(-2 * delta, 2 * delta)
            in_box = lo - 1e-12 <= d <= hi + 1e-12
            in_nlp = lb - 1e-12 <= val + d <= ub + 1e-12 and abs(d) <= delta + 1e-12
            assert in_box == in_nlp, (lo, hi, val, lb, ub, d)

    for k in range(m.G):
        same_membership(qp["glp"][k], qp["gup"][k], v["pg"][k], g.pmin[k], g.pmax[k], 100)
        same_membership(qp["glq"][k], qp["guq"][k], v["qg"][k], g.qmin[k], g.qmax[k], 100)
    ref = int(np.flatnonzero(g.bus_type == 3)[0])
    for l in range(m.L):
        i, j = g.f[l], g.t[l]
        lo, hi = qp["lo"][l], qp["hi"][l]
        same_membership(lo[0], hi[0], v["w"][i], g.vmin[i] ** 2, g.vmax[i] ** 2, 40)
        same_membership(lo[2], hi[2], v["w"][j], g.vmin[j] ** 2, g.vmax[j] ** 2, 40)
        for e, b in ((1, i), (3, j)):
            if b == ref:  # the reference angle is held at 0
                assert lo[e] == hi[e] == -v["th"][b]
            else:
                same_membership(lo[e], hi[e], v["th"][b], -2 * np.pi, 2 * np.pi, 20)
        for _ in range(40):
            di, dj = rng.uniform(-0.6, 0.6, 2)
            in_row = qp["alo"][l] - 1e-12 <= di - dj <= qp["ahi"][l] + 1e-12
            t = (v["th"][i] + di) - (v["th"][j] + dj)
            assert in_row == (g.angmin[l] - 1e-12 <= t <= g.angmax[l] + 1e-12)


# --------------------------------------------------------------------------
# component updates
# --------------------------------------------------------------------------
def test_generator_update_is_the_boxed_minimiser():
    for _ in range(50):
        gd1, gd2 = RNG.uniform(-3000, 3000), RNG.uniform(100, 2000)
        lp, up = -RNG.random(), RNG.random()
        lq, uq = -RNG.random(), RNG.random()
        z, lam, rho = RNG.standard_normal(2), 1000 * RNG.standard_normal(2), RNG.uniform(1e2, 3e4, 2)
        out = oracle.gen_update(gd1, gd2, lp, up, lq, uq, z, lam, rho)
        grid_p = np.linspace(lp, up, 200001)
        fp = gd1 * grid_p + 0.5 * gd2 * grid_p ** 2 + lam[0] * grid_p + 0.5 * rho[0] * (grid_p - z[0]) ** 2
        grid_q = np.linspace(lq, uq, 200001)
        fq = lam[1] * grid_q + 0.5 * rho[1] * (grid_q - z[1]) ** 2
        assert abs(out[0] - grid_p[np.argmin(fp)]) <= 2 * (up - lp) / 200000
        assert abs(out[1] - grid_q[np.argmin(fq)]) <= 2 * (uq - lq) / 200000


def _random_line_qp(rng, active_limits=True):
    M = rng.standard_normal((4, 4))
    Q = M @ M.T + 0.5 * np.eye(4)
    c = 3 * rng.standard_normal(4)
    lo = -rng.uniform(0.1, 1.0, 4)
    hi = rng.uniform(0.1, 1.0, 4)
    G = rng.standard_normal((2, 4))
    grhs = rng.uniform(0.05, 0.5, 2) if active_limits else np.full(2, 5.0)
    alo, ahi = -rng.uniform(0.05, 0.5), rng.uniform(0.05, 0.5)
    return Q, c, lo, hi, G, grhs, alo, ahi


def test_line_qp_matches_scipy_and_kkt():
    from scipy.optimize import minimize

    rng = np.random.default_rng(7)
    n_active = 0
    for trial in range(60):
        Q, c, lo, hi, G, grhs, alo, ahi = _random_line_qp(rng)
        x, mult, rc = oracle.line_qp(Q, c, lo, hi, G, grhs, alo, ahi, 1)
        assert rc == 0
        cons = [{"type": "ineq", "fun": (lambda y, r=r: grhs[r] - G[r] @ y), "jac": (lambda y, r=r: -G[r])}
                for r in range(2)]
        cons += [{"type": "ineq", "fun": lambda y: ahi - (y[1] - y[3])},
                 {"type": "ineq", "fun": lambda y: (y[1] - y[3]) - alo}]
        res = minimize(lambda y: 0.5 * y @ Q @ y + c @ y, np.clip(np.zeros(4), lo, hi),
                       jac=lambda y: Q @ y + c, bounds=list(zip(lo, hi)), constraints=cons,
                       method="SLSQP", options=dict(ftol=1e-15, maxiter=500))
        f_or = 0.5 * x @ Q @ x + c @ x
        assert f_or <= res.fun + 1e-9 * (1 + abs(res.fun))
        np.testing.assert_allclose(x, res.x, atol=1e-5)
        # KKT: stationarity with the returned multipliers and free bound multipliers
        assert np.all(mult >= -1e-10)
        g = Q @ x + c + mult[0] * G[0] + mult[1] * G[1] + (mult[2] - mult[3]) * np.array([0, 1, 0, -1])
        for v in range(4):
            if x[v] <= lo[v] + 1e-12:
                assert g[v] >= -1e-8
            elif x[v] >= hi[v] - 1e-12:
                assert g[v] <= 1e-8
            else:
                assert abs(g[v]) < 1e-8
        n_active += int(np.any(mult > 1e-9))
    assert n_active > 10  # the limit rows were exercised


def test_line_qp_brute_force_never_beats_it():
    rng = np.random.default_rng(11)
    for _ in range(20):
        Q, c, lo, hi, G, grhs, alo, ahi = _random_line_qp(rng)
        x, mult, rc = oracle.line_qp(Q, c, lo, hi, G, grhs, alo, ahi, 1)
        f_or = 0.5 * x @ Q @ x + c @ x
        Y = rng.uniform(lo, hi, size=(200000, 4))
        ok = (Y @ G.T <= grhs).all(1) & (Y[:, 1] - Y[:, 3] <= ahi) & (Y[:, 1] - Y[:, 3] >= alo)
        Y = Y[ok]
        fy = 0.5 * np.einsum("ij,jk,ik->i", Y, Q, Y) + Y @ c
        assert f_or <= fy.min() + 1e-12


def test_line_update_solves_the_line_subproblem():
    """eq. line_kernel from an ADMM state with a different penalty on every
    coupling: the branch result of one iteration must minimise
    1/2 d'QH d + gH'd + sum over flows and voltage copies of
    lambda (v - z) + rho/2 (v - z)^2 (flows v = F d + f0) over the box, the
    line-limit rows and the angle rows, written out here and solved by SLSQP
    from scratch (the oracle's solution, being exact, can only be better)."""
    from scipy.optimize import minimize

    g = gg.grid_30bus()
    m = oracle.Model(g)
    rng = np.random.default_rng(37)
    x = _perturbed_point(m, 0.05, rng)
    qp = m.build(x, 10 * rng.standard_normal(4 * m.L), 0.3, 1)
    st = m.new_state(rho=2e4)
    st["zl"][...] = 0.05 * rng.standard_normal(st["zl"].shape)
    st["ll"][...] = 300 * rng.standard_normal(st["ll"].shape)
    st["rl"][...] = rng.uniform(1e3, 3e4, st["rl"].shape)
    z0, l0, r0 = np.array(st["zl"]), np.array(st["ll"]), np.array(st["rl"])
    st, _ = m.admm(qp, st, eps=0.0, max_iter=1)
    for l in range(m.L):
        QH, gH = qp["QH"][l].reshape(4, 4), qp["gH"][l]
        F, f0 = qp["F"][l].reshape(4, 4), qp["f0"][l]

        def obj(db):
            df = F @ db + f0
            return (0.5 * db @ QH @ db + gH @ db + l0[l, :4] @ (df - z0[l, :4])
                    + 0.5 * r0[l, :4] @ (df - z0[l, :4]) ** 2 + l0[l, 4:] @ (db - z0[l, 4:])
                    + 0.5 * r0[l, 4:] @ (db - z0[l, 4:]) ** 2)

        Gm, gr = qp["G"][l].reshape(2, 4), qp["grhs"][l]
        cons = [{"type": "ineq", "fun": lambda db, e=e: gr[e] - Gm[e] @ db} for e in range(2) if gr[e] < 1e29]
        cons += [{"type": "ineq", "fun": lambda db: db[1] - db[3] - qp["alo"][l]},
                 {"type": "ineq", "fun": lambda db: qp["ahi"][l] - (db[1] - db[3])}]
        lo, hi = qp["lo"][l], qp["hi"][l]

        def feasible(v):
            return np.all(v >= lo - 1e-12) and np.all(v <= hi + 1e-12) and all(c["fun"](v) >= -1e-9 for c in cons)

        # the best feasible point two independent solvers find from the same start
        start = np.clip(z0[l, 4:], lo, hi)
        found = [minimize(obj, start, method="SLSQP", bounds=list(zip(lo, hi)), constraints=cons,
                          options=dict(ftol=1e-15, maxiter=1000)).x,
                 minimize(obj, start, method="trust-constr", bounds=list(zip(lo, hi)), constraints=cons,
                          options=dict(gtol=1e-12, xtol=1e-14, maxiter=3000)).x]
        best = min(obj(v) for v in found if feasible(v))
        mine = st["xl"][l, 4:]
        assert feasible(mine), l
        assert obj(mine) <= best + 1e-9 * (1 + abs(best)), l
        np.testing.assert_allclose(st["xl"][l, :4], F @ mine + f0, rtol=0, atol=1e-12)


def test_bus_update_solves_its_kkt_system():
    """eq. bus_kernel: the closed form equals a dense solve of the bus QP's KKT system."""
    g = gg.grid_30bus()
    g = g.__class__(**{**g.__dict__, "gs": 0.03 * RNG.random(g.nbus), "bs": 0.05 * RNG.random(g.nbus)})
    m = oracle.Model(g)
    x = _perturbed_point(m)
    qp = m.build(x, None, 1.0, 1)
    st = m.new_state(rho=2e4)
    for k in ("xl", "ll", "xg", "lg"):
        st[k][...] = RNG.standard_normal(st[k].shape)
    st["rl"][...] = RNG.uniform(1e3, 3e4, st["rl"].shape)
    st["rg"][...] = RNG.uniform(1e3, 3e4, st["rg"].shape)
    st, info = m.admm(qp, st, eps=0.0, max_iter=1)  # one full iteration runs the bus update
    # rebuild the bus problem from the state the bus saw: x (line/gen side) unchanged by it,
    # lambda before the multiplier step = lambda_after - rho (x - z)
    lam_l = st["ll"] - st["rl"] * (st["xl"] - st["zl"])
    lam_g = st["lg"] - st["rg"] * (st["xg"] - st["zg"])
    for i in [0, 3, 12, int(np.flatnonzero(g.bus_type == 3)[0])]:
        gens = np.flatnonzero(g.gbus == i)
        ends = [(l, 0) for l in np.flatnonzero(g.f == i)] + [(l, 1) for l in np.flatnonzero(g.t == i)]
        # variables: (p,q) per gen copy, (p,q) per flow copy, d_w
        rho, cvec, A = [], [], []
        for k in gens:
            for a in range(2):
                rho.append(st["rg"][k, a]); cvec.append(lam_g[k, a] + st["rg"][k, a] * st["xg"][k, a])
                A.append([1.0, 0.0] if a == 0 else [0.0, 1.0])
        for l, e in ends:
            for a in range(2):
                s = 2 * e + a
                rho.append(st["rl"][l, s]); cvec.append(lam_l[l, s] + st["rl"][l, s] * st["xl"][l, s])
                A.append([-1.0, 0.0] if a == 0 else [0.0, -1.0])
        rw = sum(st["rl"][l, 4 + 2 * e] for l, e in ends)
        cw = sum(lam_l[l, 4 + 2 * e] + st["rl"][l, 4 + 2 * e] * st["xl"][l, 4 + 2 * e] for l, e in ends)
        rho.append(rw); cvec.append(cw); A.append([-g.gs[i], g.bs[i]])
        Qm = np.diag(rho); Am = np.array(A).T; cv = np.array(cvec)
        n = len(rho)
        K = np.block([[Qm, Am.T], [Am, np.zeros((2, 2))]])
        sol = np.linalg.solve(K, np.concatenate([cv, [qp["pdk"][i], qp["qdk"][i]]]))
        xs = sol[:n]
        k = 0
        for kk in gens:
            assert st["zg"][kk, 0] == pytest.approx(xs[k], rel=1e-10, abs=1e-12); k += 1
            assert st["zg"][kk, 1] == pytest.approx(xs[k], rel=1e-10, abs=1e-12); k += 1
        for l, e in ends:
            assert st["zl"][l, 2 * e] == pytest.approx(xs[k], rel=1e-10, abs=1e-12); k += 1
            assert st["zl"][l, 2 * e + 1] == pytest.approx(xs[k], rel=1e-10, abs=1e-12); k += 1
            assert st["zl"][l, 4 + 2 * e] == pytest.approx(xs[-1], rel=1e-10, abs=1e-12)
        assert st["zb"][i, 0] == pytest.approx(xs[-1], rel=1e-10, abs=1e-12)
        # the angle copies: an unconstrained consensus, the penalty-weighted mean
        # (0 at the reference bus)
        rt = sum(st["rl"][l, 5 + 2 * e] for l, e in ends)
        ct = sum(lam_l[l, 5 + 2 * e] + st["rl"][l, 5 + 2 * e] * st["xl"][l, 5 + 2 * e] for l, e in ends)
        th_want = 0.0 if g.bus_type[i] == 3 else ct / rt
        assert st["zb"][i, 1] == pytest.approx(th_want, rel=1e-10, abs=1e-12)
        for l, e in ends:
            assert st["zl"][l, 5 + 2 * e] == pytest.approx(th_want, rel=1e-10, abs=1e-12)
        np.testing.assert_allclose(st["nu"][i], sol[n:], rtol=1e-9, atol=1e-9)
        # the balance rows hold exactly
        np.testing.assert_allclose(Am @ xs, [qp["pdk"][i], qp["qdk"][i]], atol=1e-11)


def test_admm_residuals_are_their_definitions():
    """Sec. IV-B residuals of one ADMM iteration from random states with
    uneven penalties: r = max |x - z| and s = max rho |z+ - z| over every
    coupling of generators and branches (flows, voltages and angles).  The
    residuals are l_inf norms, so each coupling group is also made the
    largest in turn (large multipliers for r, large penalties for s): a group
    left out of either norm would then show."""
    g = gg.grid_30bus()
    m = oracle.Model(g)
    rng = np.random.default_rng(31)
    qp = m.build(_perturbed_point(m, 0.05, rng), None, 1.0, 1)
    groups = {"gen": ("g", slice(None)), "flow": ("l", [0, 1, 2, 3]), "w": ("l", [4, 6]), "th": ("l", [5, 7])}

    def run(boost=None, what=None):
        st = m.new_state(rho=2e4)
        for k in ("xl", "zl", "ll", "xg", "zg", "lg"):
            st[k][...] = rng.standard_normal(st[k].shape)
        st["rl"][...] = rng.uniform(1e3, 3e4, st["rl"].shape)
        st["rg"][...] = rng.uniform(1e3, 3e4, st["rg"].shape)
        if boost is not None:
            side, cols = groups[boost]
            key = ("l" if what == "r" else "r") + side
            st[key][:, cols] *= 1e6 if what == "r" else 1e4
        z_old = {k: np.array(st[k]) for k in ("zl", "zg")}
        st, info = m.admm(qp, st, eps=0.0, max_iter=1)
        rg_ = {"gen": np.abs(st["xg"] - st["zg"]).max()}
        sg_ = {"gen": (st["rg"] * np.abs(st["zg"] - z_old["zg"])).max()}
        for name in ("flow", "w", "th"):
            cols = groups[name][1]
            rg_[name] = np.abs(st["xl"][:, cols] - st["zl"][:, cols]).max()
            sg_[name] = (st["rl"][:, cols] * np.abs(st["zl"][:, cols] - z_old["zl"][:, cols])).max()
        if boost is not None:
            mine = rg_ if what == "r" else sg_
            assert mine[boost] == max(mine.values()), (boost, what, mine)
        assert info["r"] == pytest.approx(max(rg_.values()), rel=1e-12)
        assert info["s"] == pytest.approx(max(sg_.values()), rel=1e-12)

    run()
    for name in groups:
        run(name, "r")
        run(name, "s")


# --------------------------------------------------------------------------
# ADMM (Alg. 2) against a direct solve of the same QP
# --------------------------------------------------------------------------
def _dense_qp(m, qp, use_angle=1):
    """The eliminated QP (variables pg, qg, w, theta steps) as dense arrays."""
    g = m.grid
    G, B, L = m.G, m.B, m.L
    n = 2 * G + 2 * B
    ipg, iqg = np.arange(G), G + np.arange(G)
    iw, ith = 2 * G + np.arange(B), 2 * G + B + np.arange(B)
    P = np.zeros((n, n)); c = np.zeros(n)
    P[ipg, ipg] = qp["gd2"]; c[ipg] = qp["gd1"]
    Aeq = np.zeros((2 * B, n)); beq = np.zeros(2 * B)
    for k in range(G):
        Aeq[2 * g.gbus[k], ipg[k]] += 1; Aeq[2 * g.gbus[k] + 1, iqg[k]] += 1
    for i in range(B):
        Aeq[2 * i, iw[i]] -= g.gs[i]; Aeq[2 * i + 1, iw[i]] += g.bs[i]
    beq[0::2] = qp["pdk"]; beq[1::2] = qp["qdk"]
    Aub, bub = [], []
    lo = np.zeros(n); hi = np.zeros(n)
    lo[ipg], hi[ipg], lo[iqg], hi[iqg] = qp["glp"], qp["gup"], qp["glq"], qp["guq"]
    const = 0.0
    for l in range(L):
        i, j = g.f[l], g.t[l]
        S = np.zeros((4, n)); S[0, iw[i]] = S[1, ith[i]] = S[2, iw[j]] = S[3, ith[j]] = 1
        P += S.T @ qp["QH"][l].reshape(4, 4) @ S; c += S.T @ qp["gH"][l]
        H = qp["H"][l].reshape(6, 6); bb = np.array([0, 0, qp["bR"][l], qp["bI"][l], 0, 0])
        const += 0.5 * bb @ H @ bb
        F = qp["F"][l].reshape(4, 4)
        for r, (bus, part) in enumerate([(i, 0), (i, 1), (j, 0), (j, 1)]):
            Aeq[2 * bus + part] -= F[r] @ S; beq[2 * bus + part] += qp["f0"][l, r]
        for e in range(2):
            Aub.append(qp["G"][l].reshape(2, 4)[e] @ S); bub.append(qp["grhs"][l, e])
        if use_angle and qp["ahi"][l] < 1e29:
            r = S[1] - S[3]
            Aub.append(r); bub.append(qp["ahi"][l]); Aub.append(-r); bub.append(-qp["alo"][l])
        lo[[iw[i], ith[i], iw[j], ith[j]]] = qp["lo"][l]
        hi[[iw[i], ith[i], iw[j], ith[j]]] = qp["hi"][l]
    return dict(P=P, c=c, const=const, Aeq=Aeq, beq=beq, Aub=np.array(Aub), bub=np.array(bub), lo=lo, hi=hi)


def _admm_objective(m, qp, d, dq):
    v = d
    return 0.5 * v @ dq["P"] @ v + dq["c"] @ v + dq["const"]


@pytest.mark.parametrize("which", ["two_bus", "two_bus_limit"])
def test_admm_qp_matches_bruteforce_active_sets(which):
    """Tiny grid: every working set of the eliminated QP is enumerated; the
    best KKT point's objective must equal ADMM's converged objective."""
    import itertools

    g = gg.two_bus(lossless=False, rate=5.0 if which == "two_bus" else 0.7,
                   c1=(20.0, 22.0) if which == "two_bus" else (20.0, 35.0))
    m = oracle.Model(g)
    x = m.flat_start()
    if which == "two_bus_limit":
        # a loaded operating point, so that the linearised line limit can bind
        v = m.split(x)
        v["th"][1] = -0.075
        v["wr"][0], v["wi"][0] = math.cos(0.075), math.sin(0.075)
        v["pg"][:] = [0.75, 0.1]
    qp = m.build(x, None, 1.5, 1)
    dq = _dense_qp(m, qp)
    ref = int(np.flatnonzero(g.bus_type == 3)[0])
    n = dq["P"].shape[0]
    # inequality rows: bounds (lo/hi) and Aub
    rows, rhs = [], []
    for k in range(n):
        e = np.zeros(n); e[k] = -1; rows.append(e); rhs.append(-dq["lo"][k])
        e = np.zeros(n); e[k] = 1; rows.append(e); rhs.append(dq["hi"][k])
    rows += list(dq["Aub"]); rhs += list(dq["bub"])
    R = np.array(rows); r = np.array(rhs)
    Eq = dq["Aeq"]; be = dq["beq"]
    best = np.inf
    for size in range(0, n - Eq.shape[0] + 1):
        for W in itertools.combinations(range(len(r)), size):
            A = np.vstack([Eq, R[list(W)]]) if W else Eq
            b = np.concatenate([be, r[list(W)]]) if W else be
            K = np.block([[dq["P"], A.T], [A, np.zeros((A.shape[0], A.shape[0]))]])
            rhs_k = np.concatenate([-dq["c"], b])
            # the QP is convex but not strictly (an LP in q, w, theta at pi = 0):
            # any consistent solution of a working set's KKT system is a KKT point
            sol = np.linalg.lstsq(K, rhs_k, rcond=None)[0]
            if np.abs(K @ sol - rhs_k).max() > 1e-9 * (1 + np.abs(rhs_k).max()):
                continue
            v = sol[:n]
            mu = sol[n + Eq.shape[0]:]
            if np.all(R @ v <= r + 1e-9) and np.all(mu >= -1e-9):
                best = min(best, 0.5 * v @ dq["P"] @ v + dq["c"] @ v)
    assert np.isfinite(best)
    st, info = m.admm(qp, rho=1e3, eps=1e-9, max_iter=200000)
    assert info["r"] <= 1e-9 and info["s"] <= 1e-9
    d, _ = m.step(qp, st, x)
    v = np.concatenate([d[:2 * m.G], d[2 * m.G:2 * m.G + 2 * m.B]])
    f_admm = 0.5 * v @ dq["P"] @ v + dq["c"] @ v
    assert f_admm == pytest.approx(best, rel=1e-7, abs=1e-6)
    assert abs(v[2 * m.G + m.B + ref]) < 1e-12


def test_admm_qp_30bus_matches_scipy():
    """30-bus QP at a perturbed point with multipliers: ADMM's converged step
    is feasible for the eliminated QP and its objective matches scipy's."""
    from scipy.optimize import minimize

    g = gg.grid_30bus()
    m = oracle.Model(g)
    x = m.flat_start()
    qp = m.build(x, None, 0.3, 1)
    dq = _dense_qp(m, qp)
    st, info = m.admm(qp, rho=2e4, eps=1e-8, max_iter=100000)
    assert info["r"] <= 1e-8 and info["s"] <= 1e-8
    d, _ = m.step(qp, st, x)
    v = np.concatenate([d[:2 * m.G], d[2 * m.G:2 * m.G + 2 * m.B]])
    assert np.abs(dq["Aeq"] @ v - dq["beq"]).max() < 1e-7
    assert (dq["Aub"] @ v - dq["bub"]).max() < 1e-7
    assert np.all(v >= dq["lo"] - 1e-7) and np.all(v <= dq["hi"] + 1e-7)
    f_admm = 0.5 * v @ dq["P"] @ v + dq["c"] @ v
    cons = [{"type": "eq", "fun": lambda y: dq["Aeq"] @ y - dq["beq"], "jac": lambda y: dq["Aeq"]},
            {"type": "ineq", "fun": lambda y: dq["bub"] - dq["Aub"] @ y, "jac": lambda y: -dq["Aub"]}]
    res = minimize(lambda y: 0.5 * y @ dq["P"] @ y + dq["c"] @ y, v, jac=lambda y: dq["P"] @ y + dq["c"],
                   bounds=list(zip(dq["lo"], dq["hi"])), constraints=cons, method="SLSQP",
                   options=dict(ftol=1e-14, maxiter=1000))
    assert f_admm == pytest.approx(res.fun, rel=1e-6, abs=1e-6)


# --------------------------------------------------------------------------
# merit function and model (Sec. II-C), SQP (Alg. 1)
# --------------------------------------------------------------------------
def test_merit_model_is_second_order_accurate():
    g = gg.grid_30bus()
    m = oracle.Model(g)
    r = m.sqp(oracle.SqpOptions(max_sqp=2))
    x = r["x"]
    qp = m.build(x, r["pi"], 1.0, 1)
    d0 = 1e-2 * RNG.standard_normal(m.n)
    # keep c11, c12 linearisations satisfied so only smooth terms remain
    errs = []
    for s in [1.0, 0.5, 0.25]:
        d = s * d0
        dv = m.split(d)
        for l in range(m.L):
            i, j = g.f[l], g.t[l]
            db = np.array([dv["w"][i], dv["th"][i], dv["w"][j], dv["th"][j]])
            dv["wr"][l] = qp["aR"][l] @ db + qp["bR"][l]
            dv["wi"][l] = qp["aI"][l] @ db + qp["bI"][l]
        phx, phxd, pred = m.merit(qp, x, d, mu=0.0)
        errs.append(abs((phx - phxd) - pred))
    # mu = 0: ared - pred = f-part only (exact quadratic cost) up to the Hessian of
    # the constraints times multipliers, which is second order => error ~ s^3
    assert errs[2] <= errs[0] / 4


def test_merit_and_model_against_their_definitions():
    """The l1 merit phi = f + mu h and the predicted reduction q(0) - q(d)
    (Sec. II-C) on a grid with tight ratings, so that line limits are
    violated at x and in the linearisation.  q(d) = grad f d + d' Hess L d / 2
    + mu m(d), with m(d) the linearised nonlinear constraints plus the linear
    constraints at x + d (the default merit).  Derivatives along d are
    symmetric differences of the objective and the constraint values (exact
    for quadratic f, c11, c13, c14; O(|d|^3) for c12)."""
    base = gg.grid_30bus()
    g = base.__class__(**{**base.__dict__, "rate": 0.25 * base.rate})
    m = oracle.Model(g)
    rng = np.random.default_rng(29)
    x = _perturbed_point(m, 0.05, rng)
    pi = 10 * rng.standard_normal(4 * m.L)
    qp = m.build(x, pi, 1.0, 1)
    d = 1e-3 * rng.standard_normal(m.n)
    mu = 7.0
    P = pi.reshape(m.L, 4)

    def neg(a):
        return np.maximum(0.0, -np.asarray(a))

    def nonlinear(c4):
        return np.abs(c4[:, 0]) + np.abs(c4[:, 1]) + neg(c4[:, 2]) + neg(c4[:, 3])

    def h(y):  # l1 sum of every violation
        c4, bal = m.constraints(y)
        v = m.split(y)
        dth = v["th"][g.f] - v["th"][g.t]
        ref = np.flatnonzero(g.bus_type == 3)
        thn = np.delete(v["th"], ref)
        return (nonlinear(c4).sum() + neg(dth - g.angmin).sum() + neg(g.angmax - dth).sum() + np.abs(bal).sum()
                + neg(v["w"] - g.vmin ** 2).sum() + neg(g.vmax ** 2 - v["w"]).sum() + np.abs(v["th"][ref]).sum()
                + neg(thn + 2 * np.pi).sum() + neg(2 * np.pi - thn).sum() + neg(v["pg"] - g.pmin).sum()
                + neg(g.pmax - v["pg"]).sum() + neg(v["qg"] - g.qmin).sum() + neg(g.qmax - v["qg"]).sum())

    f = m.objective

    def lag(y):
        return f(y) + np.sum(P * m.constraints(y)[0])

    phx, phxd, pred_mu = m.merit(qp, x, d, mu=mu)
    _, _, pred0 = m.merit(qp, x, d, mu=0.0)
    assert phx == pytest.approx(f(x) + mu * h(x), rel=1e-12)
    assert phxd == pytest.approx(f(x + d) + mu * h(x + d), rel=1e-12)
    # quadratic model of the Lagrangian along d
    gd = (f(x + d) - f(x - d)) / 2
    dHd = lag(x + d) + lag(x - d) - 2 * lag(x)
    assert pred0 == pytest.approx(-gd - dHd / 2, rel=1e-7, abs=1e-9)
    # constraint model
    c0, c1, cm = m.constraints(x)[0], m.constraints(x + d)[0], m.constraints(x - d)[0]
    lin = c0 + (c1 - cm) / 2
    assert neg(lin[:, 2:]).sum() > 0  # the linearised limits are violated
    m_d = nonlinear(lin).sum() + (h(x + d) - nonlinear(c1).sum())
    # the symmetric difference of c12 errs by O(|d|^3): 3e-11 of mu h here
    assert abs((pred_mu - pred0) - mu * (h(x) - m_d)) <= 1e-9 * mu * h(x)


def _two_bus_dispatch(c2, c1, pd, S=100.0):
    """Economic dispatch of two generators on a lossless line (closed form)."""
    p1 = (2 * c2[1] * S * S * pd + c1[1] * S - c1[0] * S) / (2 * S * S * (c2[0] + c2[1]))
    return p1, pd - p1


def test_sqp_two_bus_economic_dispatch():
    c2, c1, pd = (0.02, 0.05), (20.0, 22.0), 0.8
    g = gg.two_bus(lossless=True, c2=c2, c1=c1, pd2=pd)
    m = oracle.Model(g)
    r = m.sqp(oracle.SqpOptions(rho=1e3, eps=1e-8, max_iter=100000, tol=1e-7))
    assert r["status"] == 0
    p1, p2 = _two_bus_dispatch(c2, c1, pd)
    v = m.split(r["x"])
    np.testing.assert_allclose(v["pg"], [p1, p2], atol=1e-6)
    S = 100.0
    f = sum(c2[k] * (S * pp) ** 2 + c1[k] * S * pp for k, pp in enumerate((p1, p2)))
    assert r["obj"] == pytest.approx(f, rel=1e-8)


def test_sqp_30bus_matches_scipy_polar_acopf():
    """Independent polar-form ACOPF solved by scipy SLSQP: same objective."""
    from scipy.optimize import minimize

    g = gg.grid_30bus()
    m = oracle.Model(g)
    r = m.sqp(oracle.SqpOptions())
    assert r["status"] == 0 and r["primal"] <= 1e-4 and r["dual"] <= 1e-4
    B, G, S = g.nbus, g.ngen, g.base_mva
    y = 1 / (g.r + 1j * g.x)
    Yff, Yft, Ytf, Ytt = y + 0.5j * g.b, -y, -y, y + 0.5j * g.b
    ref = int(np.flatnonzero(g.bus_type == 3)[0])

    def unpack(z):
        return z[:B], z[B:2 * B], z[2 * B:2 * B + G], z[2 * B + G:]

    def flows(z):
        v, th, _, _ = unpack(z)
        V = v * np.exp(1j * th)
        return V[g.f] * np.conj(Yff * V[g.f] + Yft * V[g.t]), V[g.t] * np.conj(Ytf * V[g.f] + Ytt * V[g.t])

    def eq(z):
        v, th, pg, qg = unpack(z)
        Sf, St = flows(z)
        inj = np.zeros(B, complex)
        np.add.at(inj, g.gbus, pg + 1j * qg)
        inj -= g.pd + 1j * g.qd
        np.add.at(inj, g.f, -Sf)
        np.add.at(inj, g.t, -St)
        return np.concatenate([inj.real, inj.imag, [th[ref]]])

    def ineq(z):
        v, th, _, _ = unpack(z)
        Sf, St = flows(z)
        dth = th[g.f] - th[g.t]
        return np.concatenate([g.rate ** 2 - abs(Sf) ** 2, g.rate ** 2 - abs(St) ** 2, dth - g.angmin, g.angmax - dth])

    v = m.split(r["x"])
    z0 = np.concatenate([np.sqrt(v["w"]), v["th"], v["pg"], v["qg"]])
    res = minimize(lambda z: np.sum(g.c2 * (S * unpack(z)[2]) ** 2 + g.c1 * S * unpack(z)[2]), z0,
                   method="SLSQP", bounds=list(zip(g.vmin, g.vmax)) + [(-2 * np.pi, 2 * np.pi)] * B
                   + list(zip(g.pmin, g.pmax)) + list(zip(g.qmin, g.qmax)),
                   constraints=[{"type": "eq", "fun": eq}, {"type": "ineq", "fun": ineq}],
                   options=dict(maxiter=500, ftol=1e-12))
    assert np.abs(eq(res.x)).max() < 1e-6
    assert r["obj"] == pytest.approx(res.fun, rel=1e-5)


def test_sqp_multipliers_are_marginal_costs():
    """At the 2-bus optimum the power-balance multiplier of each generator bus
    equals minus that generator's marginal cost (stationarity in p_g)."""
    c2, c1, pd = (0.02, 0.05), (20.0, 22.0), 0.8
    g = gg.two_bus(lossless=True, c2=c2, c1=c1, pd2=pd)
    m = oracle.Model(g)
    x = m.flat_start()
    opts = dict(rho=1e3, eps=1e-9, max_iter=200000)
    r = m.sqp(oracle.SqpOptions(tol=1e-8, **opts))
    x = r["x"]
    qp = m.build(x, r["pi"], 0.1, 1)
    st, info = m.admm(qp, **opts)
    v = m.split(x)
    S = 100.0
    mc = 2 * np.array(c2) * S * S * v["pg"] + np.array(c1) * S
    np.testing.assert_allclose(st["nu"][:, 0], -mc, rtol=1e-5)
    p, dd = m.kkt(x, r["pi"], st["nu"].ravel(), st["ul"].ravel())
    assert p < 1e-7 and dd < 1e-6


def test_recovered_line_multipliers_satisfy_stationarity():
    """pi recovery (Sec. IV-B): at a tight 30-bus optimum, the Lagrangian
    f + sum pi c + sum nu bal must be stationary in every branch's wR and wI
    (free variables, no bounds).  The derivatives are central differences of
    the model's constraint values, not the oracle's Jacobians, so an error in
    those Jacobians cannot cancel between the recovery and the check.  All
    four multipliers of a branch enter (one branch has both limits binding);
    flipping the sign of any column breaks the identity by orders of
    magnitude."""
    g = gg.grid_30bus()
    m = oracle.Model(g)
    opts = dict(rho=2e4, eps=1e-9, max_iter=200000)
    r = m.sqp(oracle.SqpOptions(tol=1e-8, **opts))
    assert r["status"] == 0
    x = r["x"]
    qp = m.build(x, r["pi"], 0.1, 1)
    st, info = m.admm(qp, **opts)
    assert info["s"] <= 1e-9
    _, pi = m.step(qp, st, x)
    P = pi.reshape(m.L, 4)
    nu = st["nu"]
    nonzero = (np.abs(P) > 1e-6).sum(axis=0)
    assert nonzero[0] == m.L and np.all(nonzero[1:] >= 1), nonzero
    o = np.cumsum([0, m.G, m.G, m.B, m.B, m.L, m.L])
    h = 1e-6

    def grad_free(pm):
        def lag(y):
            c4, bal = m.constraints(y)
            return np.sum(pm * c4) + np.sum(nu * bal)
        out = []
        for l in range(m.L):
            for i in (o[4] + l, o[5] + l):
                y1 = x.copy(); y1[i] += h
                y0 = x.copy(); y0[i] -= h
                out.append((lag(y1) - lag(y0)) / (2 * h))
        return np.abs(out).max()

    scale = np.abs(P).max() + np.abs(nu).max()
    assert grad_free(P) <= 1e-8 * scale
    for k in range(4):
        Pw = P.copy()
        Pw[:, k] *= -1
        assert grad_free(Pw) >= 1e-2 * scale, k


def test_recovered_multipliers_satisfy_qp_stationarity():
    """pi recovery away from the optimum (Sec. IV-B): at the second SQP
    iterate of the 30-bus grid the QP's step is far from zero, and its
    Lagrangian, d'(Hess of pi_old c) d / 2 + pi_new (c + J d) + nu bal, must
    be stationary in every branch's d_wR and d_wI.  The curvature term is
    the directional derivative of central differences of pi_old c along d,
    the linear terms central differences of the constraint values: no
    Jacobian or Hessian of the oracle enters the check."""
    g = gg.grid_30bus()
    m = oracle.Model(g)
    opts = dict(rho=2e4, eps=1e-10, max_iter=400000)
    r = m.sqp(oracle.SqpOptions(max_sqp=2, **opts))
    x, p_old = r["x"], r["pi"]
    qp = m.build(x, p_old, 0.3, 1)
    st, info = m.admm(qp, **opts)
    assert info["s"] <= 1e-10
    d, p_new = m.step(qp, st, x)
    assert np.abs(d).max() > 0.1  # far from the optimum: the curvature term matters
    P, Po, nu = p_new.reshape(m.L, 4), p_old.reshape(m.L, 4), st["nu"]
    o = np.cumsum([0, m.G, m.G, m.B, m.B, m.L, m.L])
    h, e = 1e-4, 1e-2

    def lin(y):
        c4, bal = m.constraints(y)
        return np.sum(P * c4) + np.sum(nu * bal)

    def curv(y):
        return np.sum(Po * m.constraints(y)[0])

    def dfun(fun, y, i):
        y1 = y.copy(); y1[i] += h
        y0 = y.copy(); y0[i] -= h
        return (fun(y1) - fun(y0)) / (2 * h)

    res, hd = [], []
    for l in range(m.L):
        for i in (o[4] + l, o[5] + l):
            Hd = (dfun(curv, x + e * d, i) - dfun(curv, x - e * d, i)) / (2 * e)
            hd.append(Hd)
            res.append(Hd + dfun(lin, x, i))
    scale = np.abs(P).max() + np.abs(nu).max()
    assert np.abs(hd).max() > 1e-2 * scale
    assert np.abs(res).max() <= 1e-8 * scale


def test_kkt_measures_against_their_definitions():
    """The primal and dual measures of the termination test (Alg. 1) away
    from any optimum, at a point strictly inside every bound with random
    multipliers.  Primal: the largest violation of any constraint, equalities
    in absolute value and inequalities by their negative part.  Dual: the
    l_inf norm of the gradient of f + pi c + nu bal + angle rows (pi = -u on
    angmax - dtheta >= 0 and dtheta - angmin >= 0) over every variable but
    the reference angle, divided by max(1, |grad f|_inf).  Every gradient is
    a central difference of the objective and constraint values, not the
    oracle's Jacobians."""
    g = gg.grid_30bus()
    m = oracle.Model(g)
    rng = np.random.default_rng(17)
    x = _perturbed_point(m, 0.02, rng)
    v = m.split(x)
    margin = 1e-3
    v["pg"][:] = np.clip(v["pg"], g.pmin + margin, g.pmax - margin)
    v["qg"][:] = np.clip(v["qg"], g.qmin + margin, g.qmax - margin)
    v["w"][:] = np.clip(v["w"], g.vmin ** 2 + margin, g.vmax ** 2 - margin)
    ref = int(np.flatnonzero(g.bus_type == 3)[0])
    P = 10 * rng.standard_normal((m.L, 4))
    NU = 10 * rng.standard_normal((m.B, 2))
    UL = rng.standard_normal((m.L, 4))
    primal, _ = m.kkt(x, P.ravel(), NU.ravel(), UL.ravel())

    def neg(a):
        return np.maximum(0.0, -np.asarray(a))

    c4, bal = m.constraints(x)
    dth = v["th"][g.f] - v["th"][g.t]
    th_nonref = np.delete(v["th"], ref)
    viol = np.concatenate([
        np.abs(c4[:, 0]), np.abs(c4[:, 1]), neg(c4[:, 2]), neg(c4[:, 3]),
        neg(dth - g.angmin), neg(g.angmax - dth), np.abs(bal).ravel(),
        neg(v["w"] - g.vmin ** 2), neg(g.vmax ** 2 - v["w"]), [abs(v["th"][ref])],
        neg(th_nonref + 2 * np.pi), neg(2 * np.pi - th_nonref),
        neg(v["pg"] - g.pmin), neg(g.pmax - v["pg"]), neg(v["qg"] - g.qmin), neg(g.qmax - v["qg"])])
    assert primal == pytest.approx(viol.max(), rel=1e-12)

    th0 = np.cumsum([0, m.G, m.G, m.B])[3]
    h = 1e-6

    def fd(fun):
        out = np.zeros(x.size)
        for k in range(x.size):
            y1 = x.copy(); y1[k] += h
            y0 = x.copy(); y0[k] -= h
            out[k] = (fun(y1) - fun(y0)) / (2 * h)
        return out

    gf = fd(m.objective)

    def measure(Pm, NUm, ULm):
        def lag(y):
            cy, by = m.constraints(y)
            vy = m.split(y)
            d = vy["th"][g.f] - vy["th"][g.t]
            ang = -ULm[:, 2] * (g.angmax - d) - ULm[:, 3] * (d - g.angmin)
            return m.objective(y) + np.sum(Pm * cy) + np.sum(NUm * by) + np.sum(ang)
        grad = fd(lag)
        grad[th0 + ref] = 0.0
        return np.abs(grad).max() / max(1.0, np.abs(gf).max())

    # all multipliers at once, then each group alone and large enough that its
    # terms set the maximum (the measure is an l_inf norm)
    Z4, Z2 = np.zeros((m.L, 4)), np.zeros((m.B, 2))
    cases = [(P, NU, UL), (Z4, 1e4 * NU, Z4), (Z4, Z2, 1e4 * UL)]
    for k in range(4):
        Pk = Z4.copy()
        Pk[:, k] = 1e4 * P[:, k]
        cases.append((Pk, Z2, Z4))
    # one branch's four multipliers with its end buses' balance multipliers, of
    # comparable weight: the terms add in the same components, so a wrong sign
    # of any one term changes the maximum (a lone term's sign would not show)
    for n in range(24):
        l = int(rng.integers(m.L))
        Pk, NUk, ULk = Z4.copy(), Z2.copy(), Z4.copy()
        Pk[l] = 1e5 * rng.standard_normal(4)
        NUk[[g.f[l], g.t[l]]] = 3e3 * rng.standard_normal((2, 2))
        ULk[l, 2:] = 1e5 * rng.standard_normal(2)
        cases.append((Pk, NUk, ULk))
    for n, (Pm, NUm, ULm) in enumerate(cases):
        want = measure(Pm, NUm, ULm)
        _, got = m.kkt(x, Pm.ravel(), NUm.ravel(), ULm.ravel())
        assert want > 1e-2, n  # far from stationary: the measure is exercised
        assert got == pytest.approx(want, rel=1e-6), n


def test_sqp_objective_is_invariant_under_relabelling():
    """Renumbering buses and reordering branches describes the same grid, so
    the SQP solution's objective and infeasibility must not change (beyond
    rounding): an index mix-up between bus, branch or generator arrays in the
    oracle would break this."""
    a = gg.geometric_grid(118, seed=11, regional=False)
    b = gg.relabel_regional(a)
    assert not np.array_equal(a.f, b.f)
    ra = oracle.Model(a).sqp(oracle.SqpOptions())
    rb = oracle.Model(b).sqp(oracle.SqpOptions())
    assert abs(ra["obj"] - rb["obj"]) <= 1e-9 * abs(ra["obj"])
    assert rb["primal"] <= 1e-4
