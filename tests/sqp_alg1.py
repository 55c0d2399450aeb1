"""Alg. 1 driven step by step over the oracle's building blocks (QP build,
ADMM, step, merit, KKT measures), with the trust-region rules the algorithm
carries as comments: a second driver of the SQP loop, written from the paper,
against which the oracle's own loop and the GPU's history are checked.  Test
helper (not collected)."""
import math

import numpy as np

import oracle


def alg1(m, o: oracle.SqpOptions, line_fail=None):
    """Rows as the oracle's history: obj primal dual admm_iters r s accept
    delta dnorm ared pred.  line_fail (a list, optional) receives, per
    iteration, how many line subproblems of that QP's ADMM had no feasible
    point."""
    G, B = m.G, m.B
    x = m.flat_start()
    pi = np.zeros(4 * m.L)
    st = m.new_state(o.rho)
    delta = o.delta0
    primal = m.violations(x, o.use_angle)[1]
    dual = 1e30
    rows = []
    for k in range(o.max_sqp):
        qp = m.build(x, pi, delta, o.use_angle)
        m.cold(st, o.rho, 0 if k == 0 else o.warm_lambda)
        st, ai = m.admm(qp, st, rho=o.rho, eps=o.eps, max_iter=o.max_iter, use_angle=o.use_angle)
        if line_fail is not None:
            line_fail.append(ai["line_fail"])
        d, pin = m.step(qp, st, x)
        dn = float(np.abs(d[:2 * G + 2 * B]).max())
        phx, phxd, pred = m.merit(qp, x, d, o.mu, o.use_angle)
        ared = phx - phxd
        # Sec. II-C: ared > 0 and ared / pred > 0 (with ared > 0: pred > 0)
        accept = math.isfinite(ared) and math.isfinite(pred) and ared > 0 and pred > 0
        if accept:
            x = x + d
            pi = pin
            if dn >= 0.99 * delta:
                delta = min(2.0 * delta, o.delta_max)
            primal, dual = m.kkt(x, pi, st["nu"].ravel(), st["ul"].ravel(), o.use_angle)
        else:
            delta = 0.5 * min(delta, dn)
        rows.append([m.objective(x), primal, dual, ai["iters"], ai["r"], ai["s"], float(accept), delta, dn, ared,
                     pred])
        if accept and primal <= o.tol and dual <= o.tol:
            break
        if (accept and dn <= o.step_tol) or delta < o.delta_min:
            break
    return np.array(rows)
