"""Benchmark: ACOPF solves/s to 1e-4 KKT with the SQP-ADMM solver on one GB300.

One step = one complete SQP solve (Alg. 1, every QP solved by the fused ADMM
sweep of Alg. 2) of the synthetic 2,000-bus grid from a flat start, i.e. one
pass of the whole hot path.  Inputs live in HBM before the timed region; the
L2 cache is flushed (a 512 MB device write) between steps, outside the timed
events.  Multi-GPU runs are replicas (one independent instance per rank,
weak scaling, no collective on the data path).

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores (the reference arm of this project).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "ACOPF solves/s to 1e-4 KKT (batched vs plain); ADMM iter/s; HBM roofline %"


def _peaks():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def alg_bytes_per_iter(B, L, G, wbytes):
    """Algorithmic bytes one ADMM iteration of Alg. 2 must move with its
    state in memory, per the scope table's count: 8 words per coupling
    (component side: read z, lambda, write x; bus side: read x, lambda, old
    z, write z, lambda), 40 words of static QP data per branch, 8 per
    generator, 4 per bus, and a 4-byte CSR index per branch end and per
    generator.  Words in the sweep precision (wbytes)."""
    C = 8 * L + 2 * G
    return (8 * C + 40 * L + 8 * G + 4 * B) * wbytes + 4 * (2 * L + G)


def layout_bytes_per_iter(B, L, G, tbytes):
    """Bytes this implementation's layout moves per ADMM iteration: phase A
    reads the 56-value line record, z, lambda, the line-limit multipliers
    and rho and writes x and the multipliers; generators read 8 + 4 values
    and write 2; phase B reads x, lambda, old z and rho per branch end and
    writes z and lambda, and does the same for generators; buses read 4
    values and write 4; plus the 32-bit CSR/instance indices."""
    line_a = L * (56 + 8 + 8 + 4 + 1 + 8 + 4) * tbytes
    gen_a = G * (8 + 2 + 2 + 2) * tbytes
    ends_b = 2 * L * (4 + 4 + 4 + 1 + 4 + 4) * tbytes
    gens_b = G * (2 + 2 + 2 + 4 + 2 + 2) * tbytes
    bus_b = B * (4 + 2 + 2) * tbytes
    idx = 4 * (2 * L + 2 * (B + 1) + B + L + G)
    return line_a + gen_a + ends_b + gens_b + bus_b + idx


def roofline(B, L, G, wbytes, iters_per_launch, avg_launch_ms, traffic, kernel):
    """Roofline of the sweep from CUDA-event launch times: algorithmic bytes
    per launch / launch time against the measured HBM copy bandwidth; the
    layout's own bytes are reported beside it."""
    hbm, which = _peaks()
    alg = alg_bytes_per_iter(B, L, G, wbytes)
    lay = layout_bytes_per_iter(B, L, G, wbytes)
    t = avg_launch_ms / 1e3
    achieved = alg * iters_per_launch / t / 1e9 if t > 0 else 0.0
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "traffic_unit": "bytes per launch", "peak_source": which, "kernel": kernel,
            "bytes_per_iter": alg, "bytes_model": "algorithmic (8 words/coupling, 40/branch, 8/gen, 4/bus, "
                                                  "4 B index per branch end and generator)",
            "layout_bytes_per_iter": lay,
            "layout_frac": (lay * iters_per_launch / t / 1e9) / hbm if t > 0 else 0.0,
            "iters_per_launch": iters_per_launch, "avg_launch_ms": avg_launch_ms}


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile(prefix="clk", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
            sm = [float(r[1]) for r in rows]
            mx = float(rows[0][2])
            reasons = set()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for r in rows:
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                    "samples": len(rows)}
        except Exception as e:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": str(e)}


MAX_SQP = 20  # the paper's runs need at most 18 SQP iterations (Sec. V); instances that converge here need <= 16


def solver_options(binding, precision, soc=0, restore=0):
    """SQP tolerance 1e-4, at most MAX_SQP iterations; ADMM with the paper's
    large-case settings (rho 2e4, 1,000 iterations, eps 1e-3; Table II); the
    FP32 sweep's dual residual is tested against 5e-3 (its floor is rho times
    the FP32 resolution of z).  soc, restore: second-order correction and
    feasibility restoration (off for the paper's plain method)."""
    return binding.default_sqp(tol=1e-4, max_sqp=MAX_SQP, soc=soc, restore=restore,
                               admm=dict(rho=2e4, max_iter=1000, eps=1e-3,
                                         eps_dual=5e-3 if precision == "mixed" else 0.0))


def headline_config(grid, precision, world):
    """The workload of the headline line; the reference arm reports the same."""
    return {"workload": f"synthetic 2000-bus grid ({grid.nbranch} branches, {grid.ngen} generators, voltage band "
                        f"[0.9, 1.1]), one full SQP-ADMM solve per step from a flat start to 1e-4 primal and dual "
                        f"infeasibility; "
                        + ("FP32 ADMM sweep, FP64 build, residual norms, acceptance and iterate"
                           if precision == "mixed" else "FP64 throughout"),
            "global_batch": world, "parallelism": f"replicas x{world}",
            "l2": "flushed between steps (512 MB device write, outside the timed events)",
            "admm": {"rho": 2e4, "max_iter": 1000, "eps": 1e-3, "eps_dual": 5e-3 if precision == "mixed" else 1e-3},
            "sqp_tol": 1e-4, "max_sqp": MAX_SQP}


def measure(args, grid, precision, steps, warmup, local_rank, world, dev, with_e2e, with_clocks):
    import numpy as np
    import torch

    from paper_2310_13143_gb300 import binding

    stream = torch.cuda.Stream(device=dev)
    s = binding.Solver(grid, precision=precision, device=local_rank)
    s.set_stream(stream.cuda_stream)
    opts = solver_options(binding, precision)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    # launch shape of the sweep from the autotuner (cached per device, precision and size class)
    shape, tune_us = s.autotune(os.path.join(tempfile.gettempdir(), "acopf_tune_cache.json"), iters=200)

    for _ in range(warmup):
        s.sqp_solve(opts)
    torch.cuda.synchronize()
    l0 = s.launch_count()
    s.profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    conv = 0
    admm_iters = 0
    last = None
    clk = Clocks(local_rank) if with_clocks else None
    if clk:
        clk.__enter__()
    try:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 255)
            ev[k][0].record(stream)
            s.sqp_solve(opts)
            ev[k][1].record(stream)
            last = s.get_residuals(0)
            conv += int(last["result_name"] == "converged" and last["primal"] <= 1e-4 and last["dual"] <= 1e-4)
            admm_iters += last["admm_iter"]
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    finally:
        if clk:
            clk.__exit__()
    total_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    prof = s.get_profile()
    launches = s.launch_count() - l0
    s.profile(False)
    sol = s.get_solution(0)
    out = dict(total_s=total_s, conv=conv, admm_iters=admm_iters, prof=prof, launches=launches, last=last,
               obj=sol["obj"], clocks=clk.summary() if clk else None,
               launch_shape={"block_threads": shape[0], "ctas_per_sm": shape[1], "stages": shape[2],
                             "tuned_us_per_iter": tune_us})
    if with_e2e:
        # end to end through the C ABI with host buffers: new loads in from
        # pinned host memory, solve, solution out
        pd = torch.from_numpy(grid.pd.copy()).pin_memory()
        qd = torch.from_numpy(grid.qd.copy()).pin_memory()
        e2e_conv = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            s.set_loads(0, pd.numpy(), qd.numpy())
            s.sqp_solve(opts)
            s.get_solution(0)
            r = s.get_residuals(0)
            e2e_conv += int(r["result_name"] == "converged" and r["primal"] <= 1e-4 and r["dual"] <= 1e-4)
        out["e2e_s"] = time.perf_counter() - t0
        out["e2e_conv"] = e2e_conv
    s.close()
    return out


def replica_grid(rank, world):
    """The instance a rank solves: the 2,000-bus grid on one GPU; with N ranks,
    replicas of it under N correlated load scenarios, one per rank (weak
    scaling, no data-path collective)."""
    from paper_2310_13143_gb300 import gridgen

    grid = gridgen.grid_2000bus()
    if world > 1:
        grid = gridgen.scenarios_rff(grid, world, seed=4000)[rank]
    return grid


def combine_ranks(total_s, conv, admm_iters, world, dev):
    """Job totals over ranks: the slowest rank's time, the sum of converged
    solves and of ADMM iterations."""
    import torch

    t = torch.tensor([total_s, conv, admm_iters], dtype=torch.float64)
    if world > 1:
        tt = t.to(dev)
        torch.distributed.all_reduce(tt[0:1], op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(tt[1:3], op=torch.distributed.ReduceOp.SUM)
        t = tt.cpu()
    return float(t[0]), int(t[1]), int(t[2])


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_2310_13143_gb300.build import build

    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    grid = replica_grid(rank, world)

    m = measure(args, grid, args.precision, args.steps, args.warmup, local_rank, world, dev,
                with_e2e=not args.no_e2e, with_clocks=True)
    plain = None
    if args.precision == "mixed" and not args.no_plain:
        plain = measure(args, grid, "fp64", max(2, args.steps // 2), args.warmup, local_rank, world, dev,
                        with_e2e=False, with_clocks=False)

    total_s, conv_all, iters_all = combine_ranks(m["total_s"], m["conv"], m["admm_iters"], world, dev)
    if rank != 0:
        return None
    wb = 4 if args.precision == "mixed" else 8
    prof = m["prof"]
    avg_ms = prof["sweep_ms"] / max(prof["sweeps"], 1)
    iters_per_launch = prof["admm_iters"] / max(prof["sweeps"], 1)
    kernel = sweep_kernel(args.precision, m["launch_shape"]["stages"])
    traffic = measured_traffic("syn2000", iters_per_launch, kernel) if args.precision == "mixed" and world == 1 else None
    last = m["last"]
    out = {
        "metric": METRIC,
        "value": conv_all / total_s if total_s > 0 else 0.0,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": headline_config(grid, args.precision, world),
        "admm_iter_per_s": iters_all / total_s if total_s > 0 else 0.0,
        "converged_steps": conv_all,
        "admm_iters_per_solve": iters_all / max(args.steps * world, 1),
        "sqp_iters_last": last["sqp_iter"],
        "objective_last": m["obj"],
        "primal_last": last["primal"],
        "dual_last": last["dual"],
        "roofline": roofline(grid.nbus, grid.nbranch, grid.ngen, wb, iters_per_launch, avg_ms, traffic, kernel),
        "gpu_launches": m["launches"],
        "clocks": m["clocks"],
        "launch_shape": m["launch_shape"],
        # the paper's timings for grids of similar size (Table II): other grids, hardware and tolerance,
        # so context only, not a ratio
        "paper_context": {"cases": "case2383wp, case2736sp, case2737sop, case2746wop (2,383-2,746 buses)",
                          "seconds_per_solve": [11.79, 11.07, 10.62, 10.58], "sqp_iters": 2, "tolerance": 1e-3,
                          "hardware": "Quadro GV100 (Volta), ExaAdmm.jl", "source": "Table II"},
    }
    if "e2e_s" in m:
        out["e2e"] = {"value": m["e2e_conv"] / m["e2e_s"] if m["e2e_s"] > 0 else 0.0, "unit": "solves/s",
                      "h2d_bytes_per_step": 2 * 8 * grid.nbus,
                      "d2h_bytes_per_step": 8 * (2 * grid.ngen + 2 * grid.nbus + 2 * grid.nbranch + 1) + 88}
    summary = {}
    if plain is not None:
        ps = plain["total_s"]
        nst = max(2, args.steps // 2)
        out["plain_fp64"] = {"value": plain["conv"] / ps if ps > 0 else 0.0, "unit": "solves/s",
                             "ms_per_step": 1e3 * ps / nst, "admm_iter_per_s": plain["admm_iters"] / ps,
                             "objective": plain["obj"], "objective_rel_diff_vs_mixed": abs(plain["obj"] - m["obj"]) / abs(plain["obj"]),
                             "avg_sweep_launch_ms": plain["prof"]["sweep_ms"] / max(plain["prof"]["sweeps"], 1)}
        summary["plain_fp64_solves_s"] = round(out["plain_fp64"]["value"], 3)
    if world == 1 and not args.no_small:
        sm = small_30bus()
        out["small_30bus"] = sm
        summary["small_30bus"] = {"solves_s": round(sm["value"], 2), "oracle_solves_s": round(sm["oracle"]["value"], 2),
                                  "mixed_solves_s": round(sm["mixed"]["value"], 2),
                                  "batched_1024_solves_s": round(sm["batched_1024"]["value"], 1)}
    if world == 1 and not args.no_rho_sweep:
        out["rho_sweep"] = rho_sweep(grid, args.precision)
        summary["rho_sweep_solves_s"] = {f"{r['rho']:g}": round(r["solves_per_s"], 2) for r in out["rho_sweep"]}
    if world == 1 and not args.no_learned:
        lw = learned_warm_start(args)
        out["learned_warm_start"] = lw
        summary["learned"] = {"cold_s": round(lw["cold"]["seconds"], 3), "warm_s": round(lw["warm"]["seconds"], 3),
                              "speedup": round(lw["speedup_wall"], 2), "admm_ratio": round(lw["admm_iter_ratio"], 3),
                              "warm_conv": lw["warm"]["converged"], "of": lw["held_out"],
                              "gemm_frac": round(lw["tensor_gemm"]["frac"], 3)}
        if "rho_effect" in lw:
            summary["learned"]["rho_effect"] = lw["rho_effect"]
    if world == 1 and not args.no_batched:
        bgrids = workload_grids("batched")
        bs = sweep_only(bgrids, args.precision, 50, 3, 1, workload="batched")
        bs["workload"] = ("256 correlated load scenarios of the 2,000-bus grid + 64 grids of 118-10,000 buses "
                          "(log-uniform), one persistent launch, ADMM sweep only")
        out["batched_sweep"] = bs
        bsol = batched_solve(bgrids)
        out["batched_solve"] = bsol
        summary["batched_sweep"] = {"us_iter": round(bs["us_per_iter"], 1), "frac": round(bs["roofline"]["frac"], 3),
                                    "layout_frac": round(bs["roofline"]["layout_frac"], 3)}
        summary["batched_solve"] = {"solves_s": round(bsol["value"], 1), "conv": bsol["converged"],
                                    "of": bsol["instances"], "uneven": bsol["outcomes"]["uneven"],
                                    "s": round(bsol["seconds"], 3),
                                    "plain_est_s": round(bsol["plain_fp64_sample"]["estimated_seconds_all"], 1),
                                    "vs_plain": round(bsol["batched_vs_plain"], 1),
                                    "MB": round(bsol["device_bytes"] / 2 ** 20)}
        if world == 1 and not args.no_cpu_baseline:
            cb3 = cpu_batched_leg(bgrids)
            out["cpu_batched"] = cb3
            summary["cpu_batched"] = {"solves_s": round(cb3["value"], 3), "cores": cb3["cores"]}
    if world == 1 and not args.no_large:
        big = workload_grids("syn70k_x16")
        lg = sweep_only(big, "mixed", 30, 2, 1)
        lg["workload"] = ("16 correlated load scenarios of a 70,000-bus grid (90,000 branches, 10,000 generators) "
                          "in one persistent launch, ADMM sweep only")
        out["large_70k_x16"] = lg
        summary["large_70k_x16"] = {"us_iter": round(lg["us_per_iter"], 1), "frac": round(lg["roofline"]["frac"], 3),
                                    "MB": round(lg["device_bytes"] / 2 ** 20)}
        if not args.no_large_solve:
            ls = large_solve(big)
            out["large_70k_solve"] = ls
            summary["large_70k_solve"] = ls.get("summary", {})
        if not args.no_cpu_baseline:
            cl = cpu_large_leg(big[0])
            out["cpu_large"] = cl
            summary["cpu_large_iter_s"] = round(cl["admm_iter_per_s"], 2)
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(grid)
    # the figures above that the end of the line must carry (it is what a
    # truncated record keeps): compact, last
    out["summary"] = summary
    return out


def small_30bus(reps=20):
    """The synthetic 30-bus grid (the first workload): plain FP64 solves on the
    GPU, one handle, from the flat start to 1e-4 with the solver's default
    ADMM settings (rho 2e4, eps 1e-4), against the oracle's single-thread
    solves of the same grid and settings; beside them the mixed-precision
    path on the same grid and 1,024 load scenarios of it in one FP64 handle."""
    import torch

    import oracle
    from paper_2310_13143_gb300 import binding, gridgen

    g = gridgen.grid_30bus()
    opts = binding.default_sqp(tol=1e-4, max_sqp=30)
    stream = torch.cuda.Stream()
    cache = os.path.join(tempfile.gettempdir(), "acopf_tune_cache.json")
    s = binding.Solver(g, precision="fp64")
    s.set_stream(stream.cuda_stream)
    shape, _ = s.autotune(cache, iters=30)
    s.sqp_solve(opts)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    conv = 0
    a.record(stream)
    for _ in range(reps):
        s.sqp_solve(opts)
        r = s.get_residuals(0)
        conv += int(r["result_name"] == "converged" and r["primal"] <= 1e-4 and r["dual"] <= 1e-4)
    b.record(stream)
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / 1e3
    obj = s.get_solution(0)["obj"]
    s.close()
    # the same grid on the mixed-precision path (FP32 sweep, its dual residual
    # tested against 5e-3: rho times the FP32 resolution of z bounds it below)
    mopts = binding.default_sqp(tol=1e-4, max_sqp=30, admm=dict(eps_dual=5e-3))
    sm = binding.Solver(g, precision="mixed")
    sm.set_stream(stream.cuda_stream)
    mshape, _ = sm.autotune(cache, iters=30)
    sm.sqp_solve(mopts)
    mconv = 0
    a.record(stream)
    for _ in range(reps):
        sm.sqp_solve(mopts)
        mconv += int(_converged(sm.get_residuals(0)))
    b.record(stream)
    torch.cuda.synchronize()
    tm = a.elapsed_time(b) / 1e3
    mres = sm.get_residuals(0)
    mobj = sm.get_solution(0)["obj"]
    sm.close()
    # the same grid under 1,024 correlated load scenarios, one handle, FP64
    scen = gridgen.scenarios_cholesky(g, 1024, seed=1007)
    sb = binding.Solver(scen, precision="fp64")
    sb.set_stream(stream.cuda_stream)
    bshape, _ = sb.autotune(cache, iters=30)
    sb.sqp_solve_graph(opts, check_every=2)
    a.record(stream)
    sb.sqp_solve_graph(opts, check_every=2)
    b.record(stream)
    torch.cuda.synchronize()
    tb = a.elapsed_time(b) / 1e3
    bconv = sum(int(_converged(sb.get_residuals(k))) for k in range(len(scen)))
    sb.close()
    oracle.build()
    m = oracle.Model(g)
    t0 = time.perf_counter()
    n = oconv = 0
    while n < 3 or time.perf_counter() - t0 < 2.0:
        ro = m.sqp(oracle.SqpOptions(tol=1e-4, max_sqp=30))
        oconv += int(_oracle_converged(ro))
        n += 1
    to = time.perf_counter() - t0
    return {"workload": "synthetic 30-bus grid (41 branches, 6 generators), FP64, default ADMM settings",
            "value": conv / t, "unit": "solves/s", "ms_per_solve": 1e3 * t / reps, "converged": conv, "of": reps,
            "sqp_iters": r["sqp_iter"], "admm_iters": r["admm_iter"], "objective": obj,
            "objective_rel_diff_vs_oracle": abs(obj - ro["obj"]) / abs(ro["obj"]),
            "launch_shape": list(shape),
            "mixed": {"value": mconv / tm, "unit": "solves/s", "ms_per_solve": 1e3 * tm / reps, "converged": mconv,
                      "of": reps, "sqp_iters": mres["sqp_iter"], "admm_iters": mres["admm_iter"],
                      "objective_rel_diff_vs_oracle": abs(mobj - ro["obj"]) / abs(ro["obj"]),
                      "launch_shape": list(mshape), "eps_dual": 5e-3},
            "batched_1024": {"value": bconv / tb, "unit": "solves/s", "converged": bconv, "of": len(scen),
                             "seconds": tb, "launch_shape": list(bshape),
                             "workload": "1,024 correlated load scenarios of the 30-bus grid in one handle, FP64"},
            "oracle": {"value": oconv / to, "unit": "solves/s", "cores": 1, "solves": n}}


def rho_sweep(grid, precision, rhos=(2e3, 5e3, 1e4, 2e4, 5e4), reps=3):
    """The same solve under other ADMM penalties (the paper tunes rho per case,
    Tables I-II): solves/s, iterations and the objective for each; the
    headline keeps the paper's large-case 2e4."""
    import torch

    from paper_2310_13143_gb300 import binding

    stream = torch.cuda.Stream()
    rows = []
    for rho in rhos:
        opts = binding.default_sqp(tol=1e-4, max_sqp=MAX_SQP, admm=dict(rho=rho, max_iter=1000, eps=1e-3,
                                                                   eps_dual=5e-3 if precision == "mixed" else 0.0))
        s = binding.Solver(grid, precision=precision)
        s.set_stream(stream.cuda_stream)
        s.autotune(os.path.join(tempfile.gettempdir(), "acopf_tune_cache.json"), iters=30)
        s.sqp_solve(opts)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        conv = 0
        a.record(stream)
        for _ in range(reps):
            s.sqp_solve(opts)
            r = s.get_residuals(0)
            conv += int(r["result_name"] == "converged" and r["primal"] <= 1e-4 and r["dual"] <= 1e-4)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 1e3
        rows.append({"rho": rho, "solves_per_s": conv / t, "converged": conv, "of": reps, "ms_per_solve": 1e3 * t / reps,
                     "sqp_iters": r["sqp_iter"], "admm_iters": r["admm_iter"], "objective": s.get_solution(0)["obj"]})
        s.close()
    return rows


def batched_solve(grids, nscen=256, stride=10):
    """The uneven 320-instance batch solved to the end: every instance in one
    handle (launch shape from the autotuner, SQP loop replayed from a CUDA
    graph), against the plain path -- one instance at a time, cold, FP64 --
    on every stride-th instance of the same batch (scenarios and uneven grids
    alike).  The plain time of the whole batch is estimated from that sample
    per kind (count x mean time); the comparison is reported as an estimate."""
    import torch

    from paper_2310_13143_gb300 import binding

    # second-order correction and feasibility restoration on: stalled instances
    # end early, certified locally infeasible
    opts = solver_options(binding, "mixed", soc=1, restore=1)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    s = binding.Solver(grids, precision="mixed")
    s.set_stream(stream.cuda_stream)
    torch.cuda.synchronize()
    footprint = free0 - torch.cuda.mem_get_info()[0]
    cache = os.path.join(tempfile.gettempdir(), "acopf_tune_cache.json")
    shape, tune_us = s.autotune(cache, iters=30)
    s.sqp_solve_graph(opts, check_every=2)  # warm-up (captures the graph)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.sqp_solve_graph(opts, check_every=2)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    rs = [s.get_residuals(k) for k in range(len(grids))]
    ok = [r["result_name"] == "converged" and r["primal"] <= 1e-4 and r["dual"] <= 1e-4 for r in rs]
    outcomes = {}
    for part, sl in (("scenarios", slice(0, nscen)), ("uneven", slice(nscen, None))):
        names = [r["result_name"] for r in rs[sl]]
        outcomes[part] = {n: names.count(n) for n in sorted(set(names))}
    s.close()
    # plain: one handle per sampled instance, cold, FP64, the same SQP options
    idx = list(range(0, len(grids), stride))
    popts = solver_options(binding, "fp64", soc=1, restore=1)
    times = {"scenario": [], "uneven": []}
    pconv = 0
    for i in idx:
        p = binding.Solver([grids[i]], precision="fp64")
        p.set_stream(stream.cuda_stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        p.sqp_solve(popts)
        b.record(stream)
        torch.cuda.synchronize()
        times["scenario" if i < nscen else "uneven"].append(a.elapsed_time(b) / 1e3)
        r = p.get_residuals(0)
        pconv += int(r["result_name"] == "converged" and r["primal"] <= 1e-4 and r["dual"] <= 1e-4)
        p.close()
    counts = {"scenario": nscen, "uneven": len(grids) - nscen}
    est = sum(counts[k] * (sum(v) / len(v)) for k, v in times.items() if v)
    pt = sum(sum(v) for v in times.values())
    return {"instances": len(grids), "converged": int(sum(ok)), "seconds": t,
            "value": sum(ok) / t, "unit": "solves/s",
            "instances_per_s": len(grids) / t,
            "sqp_iters_max": max(r["sqp_iter"] for r in rs),
            "admm_iters_mean": float(sum(r["admm_iter"] for r in rs) / len(rs)),
            "converged_scenarios": int(sum(ok[:nscen])), "converged_uneven": int(sum(ok[nscen:])),
            "outcomes": outcomes,
            "launch_shape": {"block_threads": shape[0], "ctas_per_sm": shape[1], "stages": shape[2],
                             "tuned_us_per_iter": tune_us},
            "device_bytes": int(footprint),
            "plain_fp64_sample": {"instances": len(idx), "stride": stride, "converged": pconv, "seconds": pt,
                                  "mean_seconds": {k: (sum(v) / len(v) if v else None) for k, v in times.items()},
                                  "value": pconv / pt if pt > 0 else 0.0, "unit": "solves/s",
                                  "estimated_seconds_all": est,
                                  "estimate": "per kind: instances in the batch x mean sampled plain time"},
            "batched_vs_plain": est / t if t > 0 else None,
            "workload": "256 correlated load scenarios of the 2,000-bus grid + 64 grids of 118-10,000 buses, "
                        f"one handle, SQP to 1e-4 (max {MAX_SQP} SQP iterations, 1,000 ADMM iterations per QP), "
                        "second-order correction and feasibility restoration on"}


def learned_warm_start(args, ntrain=4096, ntest=512, steps=6000, batch=256, lr=3e-3, rho_steps=1500, rho_lr=1e-3):
    """The learned warm start: the network trained on cold solves of sampled
    loads of the 2,000-bus grid and judged on held-out scenarios against
    cold starts of the same scenarios."""
    import numpy as np
    import torch

    from paper_2310_13143_gb300 import binding, gridgen, warmstart as ws

    base = gridgen.grid_2000bus()
    scen = gridgen.scenarios_cholesky(base, ntrain + ntest, seed=1004)
    opts = solver_options(binding, "mixed")
    t0 = time.perf_counter()
    T, conv, iters, objs = ws.solve_targets(scen, opts, precision="mixed", chunk=512)
    t_data = time.perf_counter() - t0
    X = ws.loads_matrix(scen)
    dims = ws.dims_for(base)
    net = binding.Mlp(dims, max_batch=batch)
    net.set_params(gridgen.mlp_init(dims, seed=1004))
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    net.fit_standardiser(Xd.data_ptr(), Td.data_ptr(), ntrain)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = ws.train(net, Xd, Td, ntrain, steps=steps, batch=batch, lr=lr, seed=1004, schedule="cos")
    t_train = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    # per-component penalties (form 4): targets from solves started at the
    # network's own predictions under candidate factors, then fine-tuning
    t0 = time.perf_counter()
    pick, cand = ws.rho_targets(scen[:ntrain], net, Xd, T, opts, stream_ptr=stream.cuda_stream)
    t_rho_data = time.perf_counter() - t0
    Td = torch.from_numpy(T).cuda()
    net.fit_standardiser(Xd.data_ptr(), Td.data_ptr(), ntrain)
    t0 = time.perf_counter()
    ws.train(net, Xd, Td, ntrain, steps=rho_steps, batch=batch, lr=rho_lr, seed=1005, schedule="cos")
    t_rho_train = time.perf_counter() - t0
    test = scen[ntrain:]
    res = {}
    # cold: one handle, every held-out scenario from a flat start
    s = binding.Solver(test, precision="mixed")
    s.set_stream(stream.cuda_stream)
    s.sqp_solve_graph(opts, check_every=2)  # warm-up of the handle (graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.sqp_solve_graph(opts, check_every=2)
    torch.cuda.synchronize()
    t_cold = time.perf_counter() - t0
    rs = [s.get_residuals(k) for k in range(ntest)]
    res["cold"] = {"seconds": t_cold, "rs": rs, "obj": np.array([s.get_solution(k)["obj"] for k in range(ntest)]),
                   "fallback": 0}
    s.close()
    # warm: the network's prediction, then cold solves of any instance that
    # fails the convergence test (inference, the scatter, the solve and the
    # fallback inside the timed region, on a handle prepared like the cold one)
    s = binding.Solver(test, precision="mixed")
    s.set_stream(stream.cuda_stream)
    s.sqp_solve_graph(opts, check_every=2)  # warm-up of the handle (graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rs, ob, failed = ws.solve_warm_with_fallback(s, test, net, Xd[ntrain:], opts, stream_ptr=stream.cuda_stream)
    torch.cuda.synchronize()
    t_warm = time.perf_counter() - t0
    s.close()
    res["warm"] = {"seconds": t_warm, "rs": rs, "obj": np.array(ob), "fallback": len(failed)}
    # the same with the predicted per-component penalties applied
    s = binding.Solver(test, precision="mixed")
    s.set_stream(stream.cuda_stream)
    s.sqp_solve_graph(opts, check_every=2)  # warm-up of the handle (graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rs, ob, failed = ws.solve_warm_with_fallback(s, test, net, Xd[ntrain:], opts, stream_ptr=stream.cuda_stream,
                                                 use_rho=True)
    torch.cuda.synchronize()
    t_warm_rho = time.perf_counter() - t0
    s.close()
    res["warm_rho"] = {"seconds": t_warm_rho, "rs": rs, "obj": np.array(ob), "fallback": len(failed)}
    # the paper's linear feasibility projection (eq. linfeas) of the predicted
    # starts before the solve: its cost and its effect on the iterations
    s = binding.Solver(test, precision="mixed")
    s.set_stream(stream.cuda_stream)
    pred = torch.zeros((ntest, dims[-1]), device="cuda")
    net.forward(Xd[ntrain:].data_ptr(), ntest, pred.data_ptr())
    s.set_warm_start_device(pred.data_ptr(), dims[-1], base_rho=2e4, use_rho=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p_it, p_r, p_s = s.project_linear(rho=0.5, eps=1e-4, max_iter=20000)
    torch.cuda.synchronize()
    t_proj = time.perf_counter() - t0
    s.sqp_solve_graph(opts, check_every=2)
    rsp = [s.get_residuals(k) for k in range(ntest)]
    s.close()
    projected = {"projection_seconds": t_proj, "projection_iters": p_it, "projection_r": p_r, "projection_s": p_s,
                 "converged": int(sum(ws.converged(r) for r in rsp)),
                 "sqp_iters_mean": float(np.mean([r["sqp_iter"] for r in rsp])),
                 "admm_iters_mean": float(np.mean([r["admm_iter"] for r in rsp])),
                 "note": "FP64 component ADMM, rho 0.5, eps 1e-4, all held-out predictions in one handle"}
    for m in res:
        rsm = res[m].pop("rs")
        ok = [ws.converged(r) for r in rsm]
        res[m].update({"converged": int(sum(ok)), "admm_iters_mean": float(np.mean([r["admm_iter"] for r in rsm])),
                       "sqp_iters_mean": float(np.mean([r["sqp_iter"] for r in rsm]))})
    net.close()
    okc = res["cold"]["obj"]
    rel = np.abs(res["warm"]["obj"] - okc) / np.abs(okc)
    rel_rho = np.abs(res["warm_rho"]["obj"] - okc) / np.abs(okc)
    for m in res:
        res[m].pop("obj")
        res[m]["solves_per_s"] = res[m]["converged"] / res[m]["seconds"]
    chosen = np.bincount(pick, minlength=len(ws.RHO_CHOICES))
    rho_effect = {"admm_ratio": round(res["warm_rho"]["admm_iters_mean"] / res["warm"]["admm_iters_mean"], 3),
                  "sqp": [round(res["warm"]["sqp_iters_mean"], 2), round(res["warm_rho"]["sqp_iters_mean"], 2)],
                  "wall_ratio": round(res["warm_rho"]["seconds"] / res["warm"]["seconds"], 3),
                  "conv": res["warm_rho"]["converged"]}
    res["cold"]["timing"] = "host wall clock of sqp_solve_graph on a prepared handle"
    res["warm"]["timing"] = ("host wall clock of inference, scatter and sqp_solve_graph on a prepared handle, plus "
                             "the cold fallback (new handle) of instances that failed the convergence test")
    return {"train_scenarios": ntrain, "held_out": ntest, "net": dims, "train_steps": steps, "batch": batch,
            "lr": f"{lr} with cosine decay to 0 (Adam)",
            "data_seconds": t_data, "train_seconds": t_train, "data_converged": int(conv.sum()),
            "loss_first": float(losses[:10].mean()), "loss_last": float(losses[-10:].mean()),
            "cold": res["cold"], "warm": res["warm"], "warm_rho": res["warm_rho"], "warm_projected_first": projected,
            "penalty_targets": {"choices_branch_gen": [list(c) for c in ws.RHO_CHOICES],
                                "chosen": chosen.tolist(), "data_seconds": t_rho_data,
                                "train_seconds": t_rho_train, "train_steps": rho_steps,
                                "rule": "per scenario, the candidate (branch, generator) penalty factors whose solve from "
                                        "the network's predicted start converges in the fewest ADMM iterations"},
            "rho_effect": rho_effect,
            "objective_rel_diff_max_with_rho": float(rel_rho.max()),
            "speedup_wall": res["cold"]["seconds"] / res["warm"]["seconds"],
            "speedup_wall_with_rho": res["cold"]["seconds"] / res["warm_rho"]["seconds"],
            "admm_iter_ratio": res["warm"]["admm_iters_mean"] / res["cold"]["admm_iters_mean"],
            "objective_rel_diff_max": float(rel.max()), "objective_rel_diff_median": float(np.median(rel)),
            "tensor_gemm": gemm_roofline()}


def gemm_roofline(M=8192, N=8192, K=8192, reps=5):
    """The tensor-core product alone on a large square problem: achieved
    dense BF16 TFLOP/s against the measured cuBLAS peak."""
    import torch

    from paper_2310_13143_gb300 import binding

    A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda").to(torch.bfloat16)
    C = torch.empty(M, N, device="cuda", dtype=torch.float32)
    st = torch.cuda.current_stream().cuda_stream
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        binding.gemm_bf16(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, 1, st)
    times = []
    for k in range(reps):
        flush.fill_(k & 255)  # operands leave L2 between repetitions
        times.append(binding.gemm_bf16(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, 1, st) / 1e3)
    t = sum(times) / len(times)
    tf = 2.0 * M * N * K / t / 1e12
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            peak, src = float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        peak, src = 1900.0, "fallback"
    return {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
            "traffic": None, "peak_source": src, "kernel": "k_gemm_tc", "shape": [M, N, K],
            "timing": "CUDA events around the kernel on its stream, mean of the repetitions, L2 flushed between them"}


def mlp_train_steps(steps, warmup, batch=256, dims=(4000, 512, 512, 512, 46504), n=1024):
    """Training steps of the warm-start network at the 2,000-bus sizes on
    seeded random data (the solver is not involved): device time per step and
    the step's matrix-product FLOP rate."""
    import torch

    from paper_2310_13143_gb300 import binding, gridgen

    dims = list(dims)
    gen = torch.Generator(device="cuda").manual_seed(7)
    X = torch.randn(n, dims[0], device="cuda", generator=gen)
    T = torch.randn(n, dims[-1], device="cuda", generator=gen)
    net = binding.Mlp(dims, max_batch=batch)
    stream = torch.cuda.Stream()
    net.set_stream(stream.cuda_stream)
    net.set_params(gridgen.mlp_init(dims, seed=7))
    net.fit_standardiser(X.data_ptr(), T.data_ptr(), n)
    idx = torch.arange(batch, dtype=torch.int32, device="cuda")
    for _ in range(warmup):
        net.train_step(X.data_ptr(), T.data_ptr(), idx.data_ptr(), batch, 1e-3, None)
    net.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        net.train_step(X.data_ptr(), T.data_ptr(), idx.data_ptr(), batch, 1e-3, None)
    b.record(stream)
    net.sync()
    ms = a.elapsed_time(b) / steps
    # forward 2 M sum(in out); backward twice that (weight and input gradients; none for layer 0's input)
    fwd = 2.0 * batch * sum(dims[i] * dims[i + 1] for i in range(len(dims) - 1))
    bwd = 2.0 * fwd - 2.0 * batch * dims[0] * dims[1]
    net.close()
    return {"metric": "warm-start network training step", "value": ms, "unit": "ms/step", "steps": steps,
            "warmup": warmup, "batch": batch, "net": dims, "gemm_tflops_per_step": (fwd + bwd) / 1e12,
            "effective_tflop_s": (fwd + bwd) / (ms * 1e-3) / 1e12}


def large_solve(grids, tol=1e-3, max_iter=1000):
    """The 70,000-bus workload solved by SQP on the mixed-precision path, all
    scenarios in one handle (graph loop), to the tolerance the paper uses on
    its large cases (1e-3, Sec. V-A, Table II), cold start."""
    import torch

    from paper_2310_13143_gb300 import binding

    stream = torch.cuda.Stream()
    s = binding.Solver(grids, precision="mixed")
    s.set_stream(stream.cuda_stream)
    s.autotune(os.path.join(tempfile.gettempdir(), "acopf_tune_cache.json"), iters=30)
    opts = binding.default_sqp(tol=tol, max_sqp=MAX_SQP, soc=1, restore=1,
                               admm=dict(rho=2e4, max_iter=max_iter, eps=1e-3, eps_dual=5e-3))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.sqp_solve_graph(opts, check_every=2)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    rs = [s.get_residuals(k) for k in range(len(grids))]
    s.close()
    ok = [r["result_name"] == "converged" and r["primal"] <= tol and r["dual"] <= tol for r in rs]
    primal = sorted(r["primal"] for r in rs)
    out = {"instances": len(grids), "tolerance": tol, "converged": int(sum(ok)), "seconds": t,
           "sqp_iters": [r["sqp_iter"] for r in rs], "admm_iters_mean": float(sum(r["admm_iter"] for r in rs) / len(rs)),
           "primal_median": primal[len(primal) // 2], "primal_max": primal[-1],
           "dual_max": max(r["dual"] for r in rs), "results": sorted({r["result_name"] for r in rs}),
           "settings": f"rho 2e4, {max_iter} ADMM iterations per QP, eps 1e-3 (dual 5e-3), at most {MAX_SQP} SQP, "
                       "second-order correction and feasibility restoration on"}
    names = [r["result_name"] for r in rs]
    out["outcomes"] = {n: names.count(n) for n in sorted(set(names))}
    out["summary"] = {"conv": out["converged"], "of": len(grids), "tol": tol, "s": round(t, 2),
                      "primal_med": float(f"{out['primal_median']:.2e}"), "outcomes": out["outcomes"]}
    return out


def workload_grids(name):
    from paper_2310_13143_gb300 import gridgen

    if name == "syn2000":
        return [gridgen.grid_2000bus()]
    if name == "batched":  # 256 correlated load scenarios of the 2,000-bus grid + 64 uneven grids
        return gridgen.batched_uneven()
    if name == "syn70k":
        return [gridgen.grid_70k()]
    if name == "syn70k_x16":
        return gridgen.scenarios_rff(gridgen.grid_70k(), 16, seed=1005)
    raise ValueError(name)


def sweep_kernel(precision, stages):
    """Name of the sweep kernel a launch shape runs (sweep_stages 4: one
    thread-block cluster per instance)."""
    t = "float" if precision == "mixed" else "double"
    return f"k_sweep_cluster<{t}>" if stages == 4 else f"k_sweep<{t}>"


def measured_traffic(workload, iters_per_launch, kernel=None):
    """DRAM bytes per launch of the FP32 sweep on a workload, from the ncu
    record in profiles/k_sweep_traffic.json, scaled by iterations per launch;
    None when no record exists or the sweep's sources changed since."""
    import hashlib

    try:
        with open(os.path.join(HERE, "profiles", "k_sweep_traffic.json")) as f:
            rec = json.load(f)["records"][workload]
        if kernel is not None and rec["kernel"] != kernel:
            return None
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(HERE, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != rec["sha256"]:
            return None
        return rec["dram_bytes_per_iter"] * iters_per_launch
    except Exception:
        return None


def sweep_only(grids, precision, iters, launches, warmup, workload=None):
    """ADMM sweep alone (fixed iteration count) on the QP at the flat start:
    ADMM iterations/s, the sweep's HBM roofline and the handle's device
    memory footprint on a given workload."""
    import torch

    from paper_2310_13143_gb300 import binding

    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    s = binding.Solver(grids, precision=precision)
    stream = torch.cuda.Stream()
    s.set_stream(stream.cuda_stream)
    shape, _ = s.autotune(os.path.join(tempfile.gettempdir(), "acopf_tune_cache.json"), iters=30)
    s.build_qp(1.0, 2e4, True)
    torch.cuda.synchronize()
    footprint = free0 - torch.cuda.mem_get_info()[0]
    opts = binding.default_admm()
    for _ in range(warmup):
        s.admm_iterate(iters, opts)
    s.profile(True)
    for _ in range(launches):
        s.admm_iterate(iters, opts)
    p = s.get_profile()
    s.close()
    B = sum(g.nbus for g in grids)
    L = sum(g.nbranch for g in grids)
    G = sum(g.ngen for g in grids)
    us = 1e3 * p["sweep_ms"] / (iters * launches)
    kernel = sweep_kernel(precision, shape[2])
    traffic = measured_traffic(workload, iters, kernel) if precision == "mixed" and workload else None
    rl = roofline(B, L, G, 4 if precision == "mixed" else 8, iters, us * iters / 1e3, traffic, kernel)
    return {"instances": len(grids), "buses": B, "branches": L, "generators": G, "precision": precision,
            "us_per_iter": us, "admm_iter_per_s": 1e6 / us, "instance_iters_per_s": len(grids) * 1e6 / us,
            "launch_shape": {"block_threads": shape[0], "ctas_per_sm": shape[1], "stages": shape[2]},
            "device_bytes": int(footprint), "roofline": rl}


def oracle_options():
    """The oracle's settings for the benchmark's solve (as solver_options for
    the FP64 path: rho 2e4, 1,000 ADMM iterations of eps 1e-3 per QP, SQP
    tolerance 1e-4, at most MAX_SQP iterations)."""
    import oracle

    return oracle.SqpOptions(tol=1e-4, max_sqp=MAX_SQP, rho=2e4, eps=1e-3, max_iter=1000)


def _oracle_converged(r):
    return r["status"] == 0 and r["primal"] <= 1e-4 and r["dual"] <= 1e-4


def _converged(r, tol=1e-4):
    """A GPU solve that ended converged with primal and dual infeasibility within tol."""
    return r["result_name"] == "converged" and r["primal"] <= tol and r["dual"] <= tol


def cpu_baseline(grid, min_seconds=10.0):
    """The oracle as it stands, one thread: full solves of the same grid from
    the flat start, as many as fit in about min_seconds (at least one)."""
    import oracle

    oracle.build()
    m = oracle.Model(grid)
    o = oracle_options()
    n = conv = admm = 0
    t = 0.0
    while n == 0 or t < min_seconds:
        t0 = time.perf_counter()
        r = m.sqp(o)
        t += time.perf_counter() - t0
        n += 1
        conv += int(_oracle_converged(r))
        admm += r["admm_total"]
    return {"value": conv / t, "unit": "solves/s", "cores": 1, "kind": "oracle", "nproc": os.cpu_count(),
            "sample": f"{n} full single-thread oracle solves of the same 2000-bus grid from the flat start "
                      f"({t:.1f} s, {conv} converged, {r['iters']} SQP iterations each)",
            "seconds_per_solve": t / n, "admm_iter_per_s": admm / t}


def _oracle_solve(job):
    """One oracle solve in a worker process: (status, primal, dual, seconds)."""
    import oracle

    grid, kw = job
    t0 = time.perf_counter()
    r = oracle.Model(grid).sqp(oracle.SqpOptions(**kw))
    return r["status"], r["primal"], r["dual"], time.perf_counter() - t0


def cpu_batched_leg(grids, max_bus=4000, nscen=256):
    """The oracle on the batched workload, one instance per host core over
    all cores (spawned worker processes): a bounded sample of nproc instances
    taken with an even stride through the batch, uneven grids above max_bus
    buses skipped (their oracle solves run for minutes)."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    n = os.cpu_count() or 1
    eligible = [i for i in range(len(grids)) if grids[i].nbus <= max_bus]
    pick = eligible[::max(1, len(eligible) // n)][:n]
    o = oracle_options()
    kw = dict(tol=o.tol, max_sqp=o.max_sqp, rho=o.rho, eps=o.eps, max_iter=o.max_iter)
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(pick)) as pool:
        t0 = time.perf_counter()
        res = pool.map(_oracle_solve, [(grids[k], kw) for k in pick], chunksize=1)
        wall = time.perf_counter() - t0
    conv = sum(int(st == 0 and p <= 1e-4 and d <= 1e-4) for st, p, d, _ in res)
    return {"value": conv / wall, "unit": "solves/s", "instances_per_s": len(pick) / wall, "cores": len(pick),
            "kind": "oracle", "nproc": n, "converged": conv, "wall_seconds": wall,
            "sample": f"{len(pick)} instances of the batch ({sum(k < nscen for k in pick)} load scenarios, "
                      f"{sum(k >= nscen for k in pick)} uneven grids of <= {max_bus} buses), one per process, "
                      f"solved concurrently on {len(pick)} host cores"}


def cpu_large_leg(grid, iters=50):
    """The oracle on one instance of the 70,000-bus workload: ADMM iterations
    of its first QP (flat start), one thread."""
    import oracle

    oracle.build()
    m = oracle.Model(grid)
    x = m.flat_start()
    t0 = time.perf_counter()
    qp = m.build(x, None, 1.0, 1)
    t_build = time.perf_counter() - t0
    st = m.new_state(2e4)
    t0 = time.perf_counter()
    m.admm(qp, st, rho=2e4, eps=0.0, max_iter=iters)
    t = time.perf_counter() - t0
    return {"admm_iter_per_s": iters / t, "unit": "ADMM iterations/s of one 70,000-bus instance", "cores": 1,
            "kind": "oracle", "sample": f"{iters} ADMM iterations of the first QP ({t:.1f} s; QP build {t_build:.1f} s)"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores (rank 0 only).
    Every step is one full single-thread solve of the benchmark's grid from
    the flat start, with the benchmark's settings."""
    import oracle

    from paper_2310_13143_gb300 import gridgen

    oracle.build()
    grid = gridgen.grid_2000bus()
    m = oracle.Model(grid)
    o = oracle_options()
    for _ in range(args.warmup):
        m.sqp(o)
    t = 0.0
    conv = 0
    last = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        last = m.sqp(o)
        t += time.perf_counter() - t0
        conv += int(_oracle_converged(last))
    val = conv / t if t > 0 else 0.0
    return {
        "metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": headline_config(grid, "fp64", args.gpus),
        "cpu_baseline": {"value": val, "unit": "solves/s", "cores": 1, "kind": "oracle", "nproc": os.cpu_count(),
                         "sample": f"{args.steps} full single-thread oracle solves (FP64), one per step, "
                                   f"after {args.warmup} untimed ones"},
        "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "converged_steps": conv, "sqp_iters_last": last["iters"] if last else None,
        "objective_last": last["obj"] if last else None,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-rho-sweep", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-large-solve", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--workload", default="syn2000",
                    choices=["syn2000", "batched", "syn70k", "syn70k_x16", "gemm", "mlp_train"])
    ap.add_argument("--gemm-shape", default="8192,8192,8192")
    ap.add_argument("--sweep-iters", type=int, default=0)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch

        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.workload == "mlp_train":  # the warm-start network's training step alone
        from paper_2310_13143_gb300.build import build

        build()
        if rank == 0:
            print(json.dumps(mlp_train_steps(args.steps, args.warmup)), flush=True)
        return
    if args.workload == "gemm":  # the tensor-core product alone (profiling and roofline studies)
        from paper_2310_13143_gb300.build import build

        build()
        M, N, K = (int(v) for v in args.gemm_shape.split(","))
        r = gemm_roofline(M, N, K, reps=max(args.steps, 1))
        r.update({"metric": "BF16 tensor-core GEMM TFLOP/s", "value": r["achieved"], "unit": "TFLOP/s"})
        if rank == 0:
            print(json.dumps(r), flush=True)
        return
    if args.sweep_iters > 0:  # ADMM sweep alone on a workload (profiling and roofline studies)
        from paper_2310_13143_gb300.build import build

        build()
        import torch

        torch.cuda.set_device(local_rank)
        r = sweep_only(workload_grids(args.workload), args.precision, args.sweep_iters, args.steps, args.warmup,
                       workload=args.workload)
        r.update({"metric": "ADMM iter/s (sweep only)", "value": r["admm_iter_per_s"], "unit": "iter/s",
                  "workload": args.workload, "steps": args.steps, "warmup": args.warmup})
        if rank == 0:
            print(json.dumps(r), flush=True)
        return
    out = run_gpu(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
