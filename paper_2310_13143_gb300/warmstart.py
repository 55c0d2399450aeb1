"""Learned warm start of the SQP-ADMM solver (driver over the C ABI).

A network maps a scenario's loads (pd, qd of every bus) to the starting
point of a solve: the NLP point x0, the line multipliers pi, the ADMM
multipliers lambda of the first QP and a log penalty factor per component
(layout of acopf_set_warm_start_device).  The training targets are the
final iterate, multipliers and ADMM state of cold-start solves of sampled
scenarios, computed by the same solver, and penalty factors chosen by
solving each scenario from the network's own predicted start under a few
candidate factors (rho_targets).  A warm-started solve must still pass the
solver's own convergence test, so the cold-start method still decides
whether a prediction was good enough.

Everything numeric runs in the library's kernels (solves, tensor-core
products, Adam, the scatter into the solver); this module only moves arrays
between calls and draws the mini-batch order.
"""
from __future__ import annotations

import numpy as np

from . import binding


def output_width(grid) -> int:
    """5G + 2B + 15L: x0 (2G + 2B + 2L), pi (4L), lambda (8L + 2G), log factor (L + G)."""
    return 5 * grid.ngen + 2 * grid.nbus + 15 * grid.nbranch


def pad8(n: int) -> int:
    return (n + 7) // 8 * 8


def dims_for(grid, hidden=(512, 512, 512)):
    return [pad8(2 * grid.nbus), *hidden, pad8(output_width(grid))]


def loads_matrix(grids, width=None):
    """Network inputs: [pd | qd] per scenario (zero padded to width)."""
    w = width or pad8(2 * grids[0].nbus)
    X = np.zeros((len(grids), w), dtype=np.float32)
    for k, g in enumerate(grids):
        X[k, :g.nbus] = g.pd
        X[k, g.nbus:2 * g.nbus] = g.qd
    return X


def solve_targets(grids, opts, precision="mixed", chunk=256, base_rho=2e4):
    """Cold-start solves of the scenarios, chunk instances per launch.
    Returns (targets [n x padded width] FP32, converged flags, ADMM iterations,
    objectives)."""
    g0 = grids[0]
    B, L, G = g0.nbus, g0.nbranch, g0.ngen
    width = pad8(output_width(g0))
    T = np.zeros((len(grids), width), dtype=np.float32)
    conv = np.zeros(len(grids), dtype=bool)
    iters = np.zeros(len(grids), dtype=np.int64)
    objs = np.zeros(len(grids))
    for c0 in range(0, len(grids), chunk):
        part = grids[c0:c0 + chunk]
        s = binding.Solver(part, precision=precision)
        s.sqp_solve(opts)
        for k in range(len(part)):
            x, pi = s.get_iterate(k)
            st = s.get_admm_state(k)
            r = s.get_residuals(k)
            row = T[c0 + k]
            o = 0
            row[o:o + x.size] = x; o += x.size
            row[o:o + 4 * L] = pi.ravel(); o += 4 * L
            row[o:o + 8 * L] = st["lam"].ravel(); o += 8 * L
            row[o:o + 2 * G] = st["lg"].ravel(); o += 2 * G
            row[o:o + L + G] = 0.0  # the base penalty; rho_targets sets these columns
            conv[c0 + k] = r["result_name"] == "converged"
            iters[c0 + k] = r["admm_iter"]
            objs[c0 + k] = s.get_solution(k)["obj"]
        s.close()
    return T, conv, iters, objs


# candidate penalty factors (branches, generators) of the penalty targets.
# Factors below 0.5 win narrowly on many training scenarios but sit at the
# edge of stability: on held-out scenarios of the 2,000-bus grid a constant
# 0.35 left 21 of 512 warm-started solves unconverged and 0.25 left 124,
# while 0.5 converged all of them with 0.72x the ADMM iterations of 1.
RHO_CHOICES = ((1.0, 1.0), (0.75, 0.75), (0.5, 0.5), (0.5, 1.0), (0.5, 0.75))


def rho_columns(grid):
    """Column range of the per-component log penalty factors (branches, then
    generators) in the output layout."""
    B, L, G = grid.nbus, grid.nbranch, grid.ngen
    o = 2 * G + 2 * B + 2 * L + 4 * L + 8 * L + 2 * G
    return o, o + L, o + L + G


def rho_targets(grids, net, X_dev, T, opts, choices=RHO_CHOICES, chunk=1024, base_rho=2e4, precision="mixed",
                stream_ptr=None):
    """Per-component penalty targets (form 4).  Every scenario is solved from
    the network's predicted start (x0, pi, lambda) under each candidate pair
    of penalty factors -- one for every branch's couplings, one for every
    generator's -- and the pair whose solve converges in the fewest ADMM
    iterations becomes the scenario's target: log factors in T's penalty
    columns (in place).  Returns the chosen pair index per scenario and the
    ADMM iterations of each candidate."""
    import torch

    o0, o1, o2 = rho_columns(grids[0])
    n = len(grids)
    pick = np.zeros(n, dtype=np.int64)
    iters = np.full((n, len(choices)), np.inf)
    if stream_ptr is not None:
        net.set_stream(stream_ptr)
    for c0 in range(0, n, chunk):
        part = grids[c0:c0 + chunk]
        m = len(part)
        pred = torch.zeros((m, net.dims[-1]), device=X_dev.device)
        net.forward(X_dev[c0:c0 + m].data_ptr(), m, pred.data_ptr())
        s = binding.Solver(part, precision=precision)
        if stream_ptr is not None:
            s.set_stream(stream_ptr)
        for j, (fb, fg) in enumerate(choices):
            pred[:, o0:o1] = float(np.log(fb))
            pred[:, o1:o2] = float(np.log(fg))
            s.set_warm_start_device(pred.data_ptr(), net.dims[-1], base_rho=base_rho, use_x=True, use_pi=True,
                                    use_lambda=True, use_rho=True)
            s.sqp_solve_graph(opts, check_every=2)
            for k in range(m):
                r = s.get_residuals(k)
                if converged(r):
                    iters[c0 + k, j] = r["admm_iter"]
        s.close()
    # ties and all-failed rows keep the base penalty (choice 0)
    best = np.argmin(iters, axis=1)
    base_ok = np.isfinite(iters[:, 0])
    keep = ~np.isfinite(iters.min(axis=1)) | (base_ok & (iters[np.arange(n), best] >= iters[:, 0]))
    best[keep] = 0
    pick[:] = best
    for k in range(n):
        fb, fg = choices[pick[k]]
        T[k, o0:o1] = np.log(fb)
        T[k, o1:o2] = np.log(fg)
    return pick, iters


def train(net, X_dev, T_dev, n: int, steps: int, batch: int, lr: float, seed: int, schedule: str = "const"):
    """Mini-batch Adam on rows [0, n) of the device data set (shuffled every
    epoch); schedule "cos" decays the learning rate from lr to 0 along half a
    cosine.  Returns the loss of every step (read back once at the end)."""
    import math

    import torch

    rng = np.random.default_rng(seed)
    dev = X_dev.device
    losses = torch.zeros(steps, dtype=torch.float32, device=dev)
    order = np.concatenate([rng.permutation(n) for _ in range((steps * batch) // n + 1)]).astype(np.int32)
    idx_all = torch.from_numpy(order).to(dev)
    for k in range(steps):
        idx = idx_all[k * batch:(k + 1) * batch]
        lk = lr if schedule == "const" else max(lr * 0.5 * (1.0 + math.cos(math.pi * k / steps)), 1e-7)
        net.train_step(X_dev.data_ptr(), T_dev.data_ptr(), idx.data_ptr(), batch, lk, losses.data_ptr() + 4 * k)
    net.sync()
    return losses.cpu().numpy()


def converged(r, tol=1e-4) -> bool:
    return r["result_name"] == "converged" and r["primal"] <= tol and r["dual"] <= tol


def solve_warm_with_fallback(solver, grids, net, X_dev, opts, precision="mixed", stream_ptr=None, base_rho=2e4,
                             use_lambda=True, use_pi=True, use_rho=False):
    """Warm-started solve of every scenario (rows of X_dev) on the prepared
    handle `solver` over `grids`; any instance that does not pass the
    solver's own convergence test is solved again from a cold start in a
    handle of its own, so the cold-start method stays the fallback.  Returns
    per-instance residual dicts, objectives and the indices that fell back."""
    import torch

    n = len(grids)
    if stream_ptr is not None:
        net.set_stream(stream_ptr)
    pred = torch.zeros((n, net.dims[-1]), device=X_dev.device)
    net.forward(X_dev.data_ptr(), n, pred.data_ptr())
    solver.set_warm_start_device(pred.data_ptr(), net.dims[-1], base_rho=base_rho, use_x=True, use_pi=use_pi,
                                 use_lambda=use_lambda, use_rho=use_rho)
    solver.sqp_solve_graph(opts, check_every=2)
    res = [solver.get_residuals(k) for k in range(n)]
    obj = [solver.get_solution(k)["obj"] for k in range(n)]
    failed = [k for k in range(n) if not converged(res[k])]
    if failed:
        c = binding.Solver([grids[k] for k in failed], precision=precision)
        if stream_ptr is not None:
            c.set_stream(stream_ptr)
        c.sqp_solve_graph(opts, check_every=2)
        for j, k in enumerate(failed):
            res[k] = c.get_residuals(j)
            obj[k] = c.get_solution(j)["obj"]
        c.close()
    return res, obj, failed
