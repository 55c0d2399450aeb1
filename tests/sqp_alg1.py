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
    delta dnorm ared pred soc restoring.  line_fail (a list, optional)
    receives, per iteration, how many line subproblems of that iteration's
    ADMM had no feasible point.

    With o.soc, a rejected step d is corrected once: the QP is rebuilt at x
    with every nonlinear constraint's value taken at x + d (linearised at x),
    and x + d' is judged by the same ratio test against the original step's
    model reduction.  With o.restore, a stall (step or radius below its
    tolerance) above the primal tolerance starts a restoration phase that
    drops the objective (weight 0) until the violation is within tol, then
    the SQP resumes from radius delta0; a stall during restoration is local
    infeasibility (status 5)."""
    G, B = m.G, m.B
    x = m.flat_start()
    pi = np.zeros(4 * m.L)
    st = m.new_state(o.rho)
    delta = o.delta0
    primal = m.violations(x, o.use_angle)[1]
    dual = 1e30
    rows = []
    restoring, fscale = 0, 1.0
    ring, since = [0.0] * 5, 0  # primal of the last five iterations; iterations since a change of phase

    def ratio_ok(ared, pred):  # Sec. II-C: ared > 0 and ared / pred > 0
        return math.isfinite(ared) and math.isfinite(pred) and ared > 0 and pred > 0

    status = 1
    for k in range(o.max_sqp):
        qp = m.build(x, pi, delta, o.use_angle, fscale=fscale)
        m.cold(st, o.rho, 0 if k == 0 else o.warm_lambda)
        st, ai = m.admm(qp, st, rho=o.rho, eps=o.eps, max_iter=o.max_iter, use_angle=o.use_angle)
        fails = ai["line_fail"]
        iters, r_inf, s_inf = ai["iters"], ai["r"], ai["s"]
        d, pin = m.step(qp, st, x)
        dn = float(np.abs(d[:2 * G + 2 * B]).max())
        phx, phxd, pred = m.merit(qp, x, d, o.mu, o.use_angle, fscale)
        ared = phx - phxd
        accept = ratio_ok(ared, pred)
        soc = 0
        if not accept and o.soc and math.isfinite(pred) and pred > 0:
            q2 = m.build(x, pi, delta, o.use_angle, dsoc=d, fscale=fscale)
            m.cold(st, o.rho, o.warm_lambda)
            st, a2 = m.admm(q2, st, rho=o.rho, eps=o.eps, max_iter=o.max_iter, use_angle=o.use_angle)
            fails += a2["line_fail"]
            iters += a2["iters"]
            r_inf, s_inf = a2["r"], a2["s"]
            d2, pin2 = m.step(q2, st, x)
            dn2 = float(np.abs(d2[:2 * G + 2 * B]).max())
            _, phxd2, _ = m.merit(q2, x, d2, o.mu, o.use_angle, fscale)
            soc = 1
            if ratio_ok(phx - phxd2, pred):
                d, pin, dn, ared, accept, soc = d2, pin2, dn2, phx - phxd2, True, 2
        if line_fail is not None:
            line_fail.append(fails)
        if accept:
            x = x + d
            pi = pin
            if dn >= 0.99 * delta:
                delta = min(2.0 * delta, o.delta_max)
            primal, dual = m.kkt(x, pi, st["nu"].ravel(), st["ul"].ravel(), o.use_angle)
        else:
            delta = 0.5 * min(delta, dn)
        rows.append([m.objective(x), primal, dual, iters, r_inf, s_inf, float(accept), delta, dn, ared, pred,
                     float(soc), float(restoring)])
        stall = (accept and dn <= o.step_tol) or delta < o.delta_min
        # no progress: the violation, above 10 tol, has not fallen by a tenth
        # over the last five iterations of the current phase
        older, ring[k % 5] = ring[k % 5], primal
        no_progress = k >= 5 and primal > 10 * o.tol and primal > 0.9 * older and since >= 5
        since += 1
        if not restoring:
            if accept and primal <= o.tol and dual <= o.tol:
                status = 0
                break
            if stall or (o.restore and no_progress):
                if o.restore and primal > o.tol:
                    restoring, fscale, delta, since = 1, 0.0, o.delta0, 0
                    continue
                status = 2
                break
        else:
            if accept and primal <= o.tol:
                restoring, fscale, delta, since = 0, 1.0, o.delta0, 0
                continue
            if stall or no_progress:
                status = 5
                break
    return np.array(rows)
