#!/usr/bin/env python
"""Benchmark of the online RBWS hot path on one GB300 (or N, one process per GPU).

Workload (the batched RB warm-start configuration): -div(kappa grad u) = 1 on the
unit cube, zero Dirichlet data, 7-point finite differences on a 64^3 interior
grid (262,144 DoFs), kappa = mu_q on 2x2x1 blocks (p = 4), mu log-uniform in
[0.1, 10]^4.  Offline: greedy RB with N <= 20 over 256 training mu (not timed,
reported as t_off).  One step = one rbws_solve_batch over 256 test mu: reduced
Galerkin solves, lift u0 = W c, and Jacobi-PCG to ||r||/||f|| < 1e-10 (verified
on the FP64 residual).  The headline arm runs the PCG in FP32 inside FP64
iterative refinement; the FP64 arm and the zero-start arms are reported beside
it.  Inputs are resident in HBM when the timed region starts; the working set
(about 1.3 GB of solver vectors) is larger than L2, so no L2 flush is used.

`--impl reference` times the CPU FP64 oracle instead (the reference of this
build), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
import types

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged solves/s at rel-res 1e-10, warm vs zero start; stencil % of HBM BW"
UNIT = "solves/s"
WORKLOAD = ("64^3 interior grid (262,144 DoFs), 2x2x1 blocks (p=4), mu log-uniform in [0.1,10]^4, "
            "RB N<=20 by greedy over 256 training mu, 256 test mu per step, PCG to rel-res 1e-10 "
            "(preconditioner in 'precond': MG V-cycle, or Jacobi as in the Jacobi-PCG arms)")
FALLBACK_HBM = 6800.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_per_dof(kernel_tag):
    """DRAM bytes per active DoF of a kernel from a committed ncu summary, or None.

    A tag "file#kernel" reads the line "traffic_bytes_per_dof[kernel]:" of a summary that
    covers several kernels; a plain tag reads "traffic_bytes_per_dof:"."""
    name, _, sub = kernel_tag.partition("#")
    key = "traffic_bytes_per_dof[%s]:" % sub if sub else "traffic_bytes_per_dof:"
    path = os.path.join(ROOT, "profiles", name + ".md")
    try:
        for line in open(path):
            if line.strip().startswith(key):
                return float(line.split(":", 1)[1].split()[0])
    except OSError:
        pass
    return None


_MG_STATE = {}


def _mg_worker_init(grid, blocks):
    """Oracle operator and multigrid hierarchy, once per worker process."""
    import oracle as O
    from oracle import mg
    op = O.assemble(grid, blocks)
    _MG_STATE["op"], _MG_STATE["hier"] = op, mg.Hierarchy(op)


def _mg_worker_solve(task):
    """One oracle MGCG solve (Algorithm 1 with Algorithm 2 as preconditioner) from u0."""
    from oracle import mg
    mu, u0, tol = task
    r = mg.mgcg(_MG_STATE["op"], mu, u0=u0, tol=tol, hier=_MG_STATE["hier"])
    return r.iters, r.status


def cpu_baseline(w, n_solves, threads, tol, n_train_sample, reference_steps=None, precond="jacobi"):
    """Times the CPU FP64 oracle (unchanged) on a bounded sample of the workload: the Galerkin RB
    start, then Jacobi-PCG (the oracle's C solver, OpenMP across instances) or MGCG (the oracle's
    scipy multigrid, one spawned process per core)."""
    import oracle as O
    from paper_2311_13862_gb300 import inputs
    op = O.assemble(w.grid, w.blocks)
    t0 = time.perf_counter()
    basis = O.greedy(op, inputs.train_mu(w)[:n_train_sample], w.n_max)
    t_off = time.perf_counter() - t0
    mus = inputs.test_mu(w)[:n_solves]
    res = []
    times = []
    if precond == "mg":
        import multiprocessing as mp
        u0 = [basis.W.T @ O.rb_solve(basis.ANq, basis.fN, m) for m in mus]
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ.update({"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1"})
        try:
            with mp.get_context("spawn").Pool(threads, initializer=_mg_worker_init,
                                              initargs=(w.grid, w.blocks)) as pool:
                pool.map(_mg_worker_solve, [(mus[0], u0[0], 1e-2)] * threads)  # workers up and warm
                for _ in range(reference_steps or 1):
                    t0 = time.perf_counter()
                    out = pool.map(_mg_worker_solve, [(m, u, tol) for m, u in zip(mus, u0)])
                    times.append(time.perf_counter() - t0)
                    res.append(types.SimpleNamespace(iters=np.array([o[0] for o in out])))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        return basis, res, times, t_off
    for _ in range(reference_steps or 1):
        t0 = time.perf_counter()
        r = O.solve_batch(op, mus, warm=O.WARM_GALERKIN, basis=basis, tol=tol, n_threads=threads)
        times.append(time.perf_counter() - t0)
        res.append(r)
    return basis, res, times, t_off


def reference_arm(args):
    """The CPU oracle as the reference arm (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2311_13862_gb300 import inputs
    import oracle as O
    w = inputs.WORKLOADS["c2"]
    threads = O.default_threads()
    n_solves = max(threads, 16)
    basis, res, times, t_off = cpu_baseline(w, n_solves, threads, w.tol, 32,
                                            reference_steps=args.warmup + args.steps, precond=args.precond)
    timed = times[args.warmup:]
    total = sum(timed)
    value = n_solves * len(timed) / total
    its = np.concatenate([r.iters for r in res])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "batch": n_solves, "warm": "galerkin",
                                            "precision": "fp64", "precond": args.precond, "sample": True},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "%d of the 256 test mu per step, Galerkin warm start from an oracle "
                                       "greedy over the first 32 training mu (N=%d), then %s to 1e-10" %
                                       (n_solves, basis.N, "MGCG" if args.precond == "mg" else "Jacobi-PCG")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "iters_mean": float(its.mean()), "t_off_s": t_off}
    print(json.dumps(line), flush=True)


def bench_gaussian(args):
    """The second workload (non-affine source): the 64^3, 2x2x1-block operator with, per parameter,
    a Gaussian source of its own centre.  Greedy with a source per training parameter (N <= 40),
    then 256 test (mu, source) pairs per step: MG-preconditioned FP32 PCG inside FP64 refinement to
    1e-10 from the Galerkin RB start (value) and from zero (arm)."""
    import torch
    from paper_2311_13862_gb300 import build, inputs, rbws
    build.build()
    torch.cuda.set_device(0)
    w = inputs.WORKLOADS["c2g"]
    P = rbws.Problem(w.grid, w.blocks)
    ft = torch.empty((w.n_train, P.n), dtype=torch.float64, device="cuda")
    rbws.rbws_gaussian_source(P.h, inputs.train_sources(w), ft)
    t0 = time.perf_counter()
    N, sel, eta = rbws.rbws_offline_greedy_rhs(P.h, inputs.train_mu(w), ft, w.n_max, 0.0, 1e-12)
    torch.cuda.synchronize()
    t_off = time.perf_counter() - t0
    del ft
    B = args.batch or w.n_test
    mus = inputs.test_mu(w, B)
    f = torch.empty((B, P.n), dtype=torch.float64, device="cuda")
    rbws.rbws_gaussian_source(P.h, inputs.test_sources(w, B), f)
    u = torch.empty_like(f)
    opt = rbws.rbws_options_default(precond=rbws.PREC_MG, precision=rbws.FP32_IR)
    arms = {}
    for name, warm in (("mgcg_galerkin_fp32ir", rbws.WARM_GALERKIN), ("mgcg_zero_fp32ir", rbws.WARM_ZERO)):
        for _ in range(args.warmup):
            rbws.rbws_solve_batch_rhs(P.h, mus, f, w.tol, warm, u, opt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            e0.record()
            for _ in range(args.steps):
                rc, it, rel, st = rbws.rbws_solve_batch_rhs(P.h, mus, f, w.tol, warm, u, opt)
            e1.record()
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        arms[name] = {"solves_per_s": B / (ms / 1e3), "ms_per_step": ms, "iters_mean": float(np.mean(it)),
                      "iters_max": int(np.max(it)), "relres_max": float(np.max(rel)),
                      "all_converged": bool(np.all(st == 0)), "clocks": clk.summary()}
    # error of every solution against the oracle: its own Gaussian sources, its FP64 MGCG
    # solutions from zero to 1e-13, and the relative L2 error and true residual of each GPU
    # solution (the Galerkin arm's, which u holds after the zero arm: re-solved once here)
    oracle_error = None
    if not args.no_oracle_check:
        from oracle import batch as O_batch
        from oracle import rhs as O_rhs
        f_or = O_rhs.gaussian_source(w.grid, inputs.test_sources(w, B))
        U_ref, _, r_rel, r_st, r_s, r_p = O_batch.reference_solutions(w.grid, mus, blocks=w.blocks, f=f_or,
                                                                      tol=1e-13)
        errs = {}
        for name, warm in (("mgcg_zero_fp32ir", rbws.WARM_ZERO), ("mgcg_galerkin_fp32ir", rbws.WARM_GALERKIN)):
            rbws.rbws_solve_batch_rhs(P.h, mus, f, w.tol, warm, u, opt)
            es = O_batch.error_summary(w.grid, mus, u.cpu().numpy(), U_ref, blocks=w.blocks, f=f_or)
            errs[name] = {k: v for k, v in es.items() if k not in ("relL2", "true_relres")}
        oracle_error = {"arms": errs, "reference": {"solver": "oracle MGCG (FP64) from zero, oracle Gaussian "
                                                              "sources", "tol": 1e-13, "relres_max": float(r_rel.max()),
                                                    "all_converged": bool(np.all(r_st == 0)), "processes": r_p,
                                                    "seconds": r_s}}
    head = arms["mgcg_galerkin_fp32ir"]
    line = {"metric": METRIC, "value": head["solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer", "data": "synthetic",
            "config": {"workload": "64^3 interior grid, 2x2x1 blocks, mu log-uniform in [0.1,10]^4, and per "
                       "parameter a Gaussian source exp(-|x-c|^2/(2 0.1^2)) with c uniform in [0.25,0.75]^3; "
                       "RB N<=40 by greedy over 256 training (mu, source) pairs; %d test pairs per step; "
                       "MG-PCG in FP32 inside FP64 refinement to rel-res 1e-10" % B,
                       "batch_per_gpu": B, "N": int(N), "warm": "galerkin", "precision": "fp32ir", "precond": "mg",
                       "tol": w.tol, "l2": "no flush: solver working set > 129 MB L2"},
            "clocks": head["clocks"], "arms": arms, "t_off_s": t_off, "greedy_eta_last": float(eta[-1]),
            "iters_mean": head["iters_mean"], "relres_max": head["relres_max"],
            "oracle_error": oracle_error}
    print(json.dumps(line))
    P.close()


def bench_requests(args):
    """96 requests (32 each on 96^3, 128^3, 256^3 grids, 3x3x3 blocks, mu in [0.1,10]^27) per step,
    interleaved in a fixed order, in one rbws_solve_requests call: learned start with one reduced
    correction, MG-preconditioned FP32 PCG inside FP64 refinement to 1e-10; per-request latency
    p50/p99; every request's error against the oracle's FP64 solution."""
    import torch
    from paper_2311_13862_gb300 import build, inputs, rbws
    build.build()
    torch.cuda.set_device(0)
    names = ["c5-96", "c5-128", "c5-256"]
    order = [k % 3 for k in range(96)]  # 96^3, 128^3, 256^3, 96^3, ...
    per = [order.count(k) for k in range(3)]
    # the oracle's FP64 solutions of every request, before any GPU work (MGCG from zero to 1e-12 on
    # A(mu) assembled per request; 8 worker processes for the 256^3 grid, about 7 GB each)
    refs = {}
    if not args.no_oracle_check:
        from oracle import batch as O_batch
        for k, nm in enumerate(names):
            w = inputs.WORKLOADS[nm]
            procs = 8 if w.grid[0] >= 256 else None
            U, _, r_rel, r_st, r_s, r_p = O_batch.reference_solutions(w.grid, inputs.test_mu(w)[:per[k]],
                                                                      blocks=w.blocks, tol=1e-12, processes=procs)
            refs[nm] = (U, {"relres_max": float(r_rel.max()), "all_converged": bool(np.all(r_st == 0)),
                            "seconds": r_s, "processes": r_p})
    probs, offline = [], {}
    for nm in names:
        w = inputs.WORKLOADS[nm]
        P = rbws.Problem(w.grid, w.blocks)
        t0 = time.perf_counter()
        N, sel, eta = rbws.rbws_offline_greedy(P.h, inputs.train_mu(w, args.c5_train), w.n_max, 0.0, 1e-12)
        t1 = time.perf_counter()
        loss = rbws.rbws_train_surrogate(P.h, inputs.surrogate_mu(w, 2048), hidden=256, epochs=args.mlp_epochs // 2,
                                         batch=256, lr=1e-3, mu_lo=w.mu_lo, mu_hi=w.mu_hi, seed=3005)
        t2 = time.perf_counter()
        tile = rbws.rbws_autotune(P.h, 32)
        offline[nm] = {"N": N, "greedy_s": t1 - t0, "train_s": t2 - t1, "train_loss": loss,
                       "eta_last": float(eta[-1]), "tile": tile[:3], "schedule": tile[4], "tile_pair_ms": tile[3]}
        probs.append((w, P))
    mus = [None] * 96
    count = [0, 0, 0]
    for r, k in enumerate(order):
        mus[r] = inputs.test_mu(probs[k][0])[count[k]]
        count[k] += 1
    handles = [probs[k][1].h for k in order]
    outs = [torch.empty(probs[k][1].n, dtype=torch.float64, device="cuda") for k in order]
    opt = rbws.rbws_options_default(precision=rbws.FP32_IR, precond=rbws.PREC_MG)
    for _ in range(args.warmup):
        rbws.rbws_solve_requests(handles, mus, outs, 1e-10, rbws.WARM_LEARNED_CORRECTED, opt)
    torch.cuda.synchronize()
    lats, its, times = [], [], []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            rc, it, rel, st, lat = rbws.rbws_solve_requests(handles, mus, outs, 1e-10,
                                                            rbws.WARM_LEARNED_CORRECTED, opt)
            times.append(time.perf_counter() - t0)
            assert np.all(st == 0), st
            lats.append(lat)
            its.append(it)
    lat = np.concatenate(lats)
    it = np.concatenate(its)
    ms = 1e3 * float(np.mean(times))
    per_grid = {}
    for k, nm in enumerate(names):
        sel_k = np.array([order[r] == k for r in range(96)] * args.steps)
        per_grid[nm] = {"iters_mean": float(it[sel_k].mean()), "iters_max": int(it[sel_k].max()),
                        "latency_ms_p50": float(np.percentile(lat[sel_k], 50)),
                        "latency_ms_p99": float(np.percentile(lat[sel_k], 99))}
        if nm in refs:
            w = probs[k][0]
            rows = [r for r in range(96) if order[r] == k]
            U = np.stack([outs[r].cpu().numpy() for r in rows])
            es = O_batch.error_summary(w.grid, np.stack([mus[r] for r in rows]), U, refs[nm][0], blocks=w.blocks)
            per_grid[nm]["oracle_error"] = {kk: v for kk, v in es.items() if kk not in ("relL2", "true_relres")}
            per_grid[nm]["oracle_error"]["reference"] = dict(refs[nm][1], solver="oracle MGCG (FP64) from zero",
                                                             tol=1e-12)
    line = {"metric": METRIC, "value": 96 / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 inner / f64 outer", "data": "synthetic",
            "config": {"workload": "96 requests per step: 32 each on 96^3, 128^3, 256^3 interior grids, 3x3x3 "
                                   "blocks (p=27), mu log-uniform in [0.1,10]^27, RB N<=60 per grid, learned "
                                   "start + one reduced correction, MG-preconditioned FP32 PCG in FP64 "
                                   "refinement to 1e-10",
                       "timing": "host wall clock around each rbws_solve_requests call (synchronous)"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "per_grid": per_grid, "offline": offline, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    for w, P in probs:
        P.close()


def bench_c3(args):
    """The mixed-precision workload: 128^3 interior grid (2,097,152 DoFs), 2x2x2 octants, mu
    log-uniform in [0.01,100]^8 (contrast up to 1e4), RB N<=40 by greedy over 256 training mu,
    64 test mu per step.  Headline: Galerkin RB start, MG-preconditioned FP32 PCG inside FP64
    refinement to 1e-10.  Arms: zero start, FP64, and the learned start (8 -> 256 -> 256 -> 256
    -> N network trained on the GPU on the Galerkin coefficients of 4096 parameters), with and
    without one reduced correction.  Every solution of every arm is measured against the
    oracle's FP64 solution."""
    import torch
    from paper_2311_13862_gb300 import build, inputs, rbws
    w = inputs.WORKLOADS["c3"]
    B = args.batch or w.n_test
    mus = inputs.test_mu(w, B)
    U_ref, ref_info = None, None
    if not args.no_oracle_check:
        from oracle import batch as O_batch
        U_ref, _, r_rel, r_st, r_s, r_p = O_batch.reference_solutions(w.grid, mus, blocks=w.blocks, tol=1e-12)
        ref_info = {"solver": "oracle MGCG (FP64) from zero", "tol": 1e-12, "relres_max": float(r_rel.max()),
                    "all_converged": bool(np.all(r_st == 0)), "processes": r_p, "seconds": r_s}
    build.build()
    torch.cuda.set_device(0)
    P = rbws.Problem(w.grid, w.blocks)
    t0 = time.perf_counter()
    N, sel, eta = rbws.rbws_offline_greedy(P.h, inputs.train_mu(w), w.n_max, 0.0, 1e-12)
    torch.cuda.synchronize()
    t_off = time.perf_counter() - t0
    tile = rbws.rbws_autotune(P.h, B)
    t0 = time.perf_counter()
    loss = rbws.rbws_train_surrogate(P.h, inputs.surrogate_mu(w, 4096), hidden=256, epochs=args.mlp_epochs,
                                     batch=256, lr=1e-3, mu_lo=w.mu_lo, mu_hi=w.mu_hi, seed=3003)
    torch.cuda.synchronize()
    learned = {"train_s": time.perf_counter() - t0, "final_loss": loss, "samples": 4096,
               "epochs": args.mlp_epochs, "hidden": 256, "layers": "%d -> 256 -> 256 -> 256 -> %d" % (w.Q, N)}
    u = torch.empty((B, P.n), dtype=torch.float64, device="cuda")
    M, FP32, FP64 = rbws.PREC_MG, rbws.FP32_IR, rbws.FP64
    arm_list = [("mgcg_galerkin_fp32ir", rbws.WARM_GALERKIN, FP32), ("mgcg_zero_fp32ir", rbws.WARM_ZERO, FP32),
                ("mgcg_learned_fp32ir", rbws.WARM_LEARNED, FP32),
                ("mgcg_learned_corrected_fp32ir", rbws.WARM_LEARNED_CORRECTED, FP32),
                ("mgcg_galerkin_fp64", rbws.WARM_GALERKIN, FP64), ("mgcg_zero_fp64", rbws.WARM_ZERO, FP64)]
    arms, head_err, clocks = {}, None, None
    for name, warm, pr in arm_list:
        steps = args.steps if name == "mgcg_galerkin_fp32ir" else max(1, args.arm_steps)
        opt = rbws.rbws_options_default(precision=pr, precond=M)
        for _ in range(args.warmup if name == "mgcg_galerkin_fp32ir" else 1):
            rbws.rbws_solve_batch(P.h, mus, w.tol, warm, u, opt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            e0.record()
            for _ in range(steps):
                rc, it, rel, st = rbws.rbws_solve_batch(P.h, mus, w.tol, warm, u, opt)
            e1.record()
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        arms[name] = {"solves_per_s": B / (ms / 1e3), "ms_per_step": ms, "iters_mean": float(np.mean(it)),
                      "iters_max": int(np.max(it)), "relres_max": float(np.max(rel)),
                      "all_converged": bool(np.all(st == 0))}
        if name == "mgcg_galerkin_fp32ir":
            clocks = clk.summary()
        if U_ref is not None:
            uh = u.cpu().numpy()
            if name == "mgcg_galerkin_fp32ir":
                es = O_batch.error_summary(w.grid, mus, uh, U_ref, blocks=w.blocks)
                head_err = {k: v for k, v in es.items() if k not in ("relL2", "true_relres")}
                head_err["reference"] = ref_info
                arms[name]["oracle_relL2_max"], arms[name]["oracle_relL2_mean"] = es["relL2_max"], es["relL2_mean"]
            else:
                e = O_batch.relL2(uh, U_ref)
                arms[name]["oracle_relL2_max"], arms[name]["oracle_relL2_mean"] = float(e.max()), float(e.mean())
    head = arms["mgcg_galerkin_fp32ir"]
    line = {"metric": METRIC, "value": head["solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer", "data": "synthetic",
            "config": {"workload": "128^3 interior grid (2,097,152 DoFs), 2x2x2 octants (p=8), mu log-uniform in "
                                   "[0.01,100]^8, RB N<=40 by greedy over 256 training mu, %d test mu per step, "
                                   "MG-PCG in FP32 inside FP64 refinement to rel-res 1e-10" % B,
                       "batch_per_gpu": B, "N": int(N), "warm": "galerkin", "precision": "fp32ir",
                       "precond": "mg", "tol": w.tol, "l2": "no flush: solver working set > 129 MB L2"},
            "clocks": clocks, "arms": arms, "t_off_s": t_off, "greedy_eta_last": float(eta[-1]),
            "autotune": {"tile": list(tile[:3]), "schedule": tile[4]}, "learned_training": learned,
            "iters_mean": head["iters_mean"], "relres_max": head["relres_max"], "oracle_error": head_err}
    if "mgcg_zero_fp64" in arms:
        line["speedup_vs_mgcg_zero_fp64"] = head["solves_per_s"] / arms["mgcg_zero_fp64"]["solves_per_s"]
    print(json.dumps(line), flush=True)
    P.close()


def bench_ex1(args):
    """The paper's Example 1 (Sec. 4) on a 64^3 interior grid (262,144 DoFs): kappa = 1 +
    mu_1 g(x) given at the cell faces (two affine terms), Dirichlet data (1 - mu_2) G1 + mu_2 G2
    eliminated into the right-hand side, source 3 pi^2 sin sin sin, mu uniform on [0,2] x [0,1].
    Offline: greedy over 70 training mu (the paper's training-set size), each with its own
    right-hand side, N <= 20.  Each step forms the 256 right-hand sides on the device
    (rbws_affine_sources: source + lifts) and solves them to rel-res 1e-10.  Headline: Galerkin
    start with the FP64 MG-PCG.  The solution depends smoothly on mu_1 and affinely on mu_2, so
    the reduced space alone meets the tolerance for almost every instance; the mixed-precision
    start (an FP32 lift) is accurate only to FP32 rounding and needs a few V-cycles more, and
    with per-node coefficient tables the FP32 iteration saves little traffic.  Arms: FP32
    refinement from the Galerkin start, zero starts in both precisions.  Every solution is
    measured against the oracle's FP64 solution."""
    import torch
    from paper_2311_13862_gb300 import build, inputs, rbws
    grid, n_max, n_train, tol = (64, 64, 64), 20, 70, 1e-10
    B = args.batch or 256
    mu = inputs.example1_mu(2007, B)
    mu_t = inputs.example1_mu(1007, n_train)
    m1, m2 = mu[:, 0], mu[:, 1]
    th_f = np.column_stack([np.ones(B), 1.0 - m2, m1 * (1.0 - m2), m2, m1 * m2])
    th = np.column_stack([np.ones(B), m1])
    tt1, tt2 = mu_t[:, 0], mu_t[:, 1]
    th_ft = np.column_stack([np.ones(n_train), 1.0 - tt2, tt1 * (1.0 - tt2), tt2, tt1 * tt2])
    th_t = np.column_stack([np.ones(n_train), tt1])
    faces = inputs.example1_faces(grid)
    G1, G2 = inputs.example1_boundary(grid)
    U_ref, ref_info, F_ref = None, None, None
    if not args.no_oracle_check:
        import oracle as O
        from oracle import batch as O_batch
        from oracle import rhs as O_rhs
        L1, L2 = (O.dirichlet_lift(grid, *faces, G) for G in (G1, G2))
        F_ref = O_rhs.example1_rhs(inputs.example1_source(grid), L1, L2, mu)
        U_ref, _, r_rel, r_st, r_s, r_p = O_batch.reference_solutions(grid, th, f=F_ref, tol=1e-12, fields=faces)
        ref_info = {"solver": "oracle MGCG (FP64) from zero", "tol": 1e-12, "relres_max": float(r_rel.max()),
                    "all_converged": bool(np.all(r_st == 0)), "processes": r_p, "seconds": r_s}
    build.build()
    torch.cuda.set_device(0)
    P = rbws.Problem.field(grid, *faces)
    L = torch.empty((2, 2, P.n), dtype=torch.float64, device="cuda")
    rbws.rbws_dirichlet_lift(P.h, G1, L[0])
    rbws.rbws_dirichlet_lift(P.h, G2, L[1])
    Fd = torch.from_numpy(inputs.example1_source(grid)).cuda()
    Fk = torch.stack([Fd, L[0, 0], L[0, 1], L[1, 0], L[1, 1]]).contiguous()
    t0 = time.perf_counter()
    ft = torch.empty((n_train, P.n), dtype=torch.float64, device="cuda")
    rbws.rbws_affine_sources(P.h, Fk, th_ft, ft)
    N, sel, eta = rbws.rbws_offline_greedy_rhs(P.h, th_t, ft, n_max, 0.0, 1e-12)
    torch.cuda.synchronize()
    t_off = time.perf_counter() - t0
    del ft
    f = torch.empty((B, P.n), dtype=torch.float64, device="cuda")
    u = torch.empty_like(f)
    M, FP32, FP64 = rbws.PREC_MG, rbws.FP32_IR, rbws.FP64
    HEAD = "mgcg_galerkin_fp64"
    arm_list = [(HEAD, rbws.WARM_GALERKIN, FP64), ("mgcg_galerkin_fp32ir", rbws.WARM_GALERKIN, FP32),
                ("mgcg_zero_fp32ir", rbws.WARM_ZERO, FP32), ("mgcg_zero_fp64", rbws.WARM_ZERO, FP64)]
    if args.arm_steps == 0:
        arm_list = arm_list[:1]
    arms, head_err, clocks = {}, None, None

    def step(warm, opt):
        rbws.rbws_affine_sources(P.h, Fk, th_f, f)
        return rbws.rbws_solve_batch_rhs(P.h, th, f, tol, warm, u, opt)

    for name, warm, pr in arm_list:
        head = name == HEAD
        steps = args.steps if head else max(1, args.arm_steps)
        opt = rbws.rbws_options_default(precision=pr, precond=M)
        for _ in range(args.warmup if head else 1):
            step(warm, opt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            e0.record()
            for _ in range(steps):
                rc, it, rel, st = step(warm, opt)
            e1.record()
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        arms[name] = {"solves_per_s": B / (ms / 1e3), "ms_per_step": ms, "iters_mean": float(np.mean(it)),
                      "iters_max": int(np.max(it)), "relres_max": float(np.max(rel)),
                      "all_converged": bool(np.all(st == 0))}
        if head:
            clocks = clk.summary()
        if U_ref is not None:
            uh = u.cpu().numpy()
            if head:
                es = O_batch.error_summary(grid, th, uh, U_ref, f=F_ref, fields=faces)
                head_err = {k: v for k, v in es.items() if k not in ("relL2", "true_relres")}
                head_err["reference"] = ref_info
                arms[name]["oracle_relL2_max"], arms[name]["oracle_relL2_mean"] = es["relL2_max"], es["relL2_mean"]
            else:
                e = O_batch.relL2(uh, U_ref)
                arms[name]["oracle_relL2_max"], arms[name]["oracle_relL2_mean"] = float(e.max()), float(e.mean())
    head = arms[HEAD]
    line = {"metric": METRIC, "value": head["solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "the paper's Example 1 (Sec. 4) on a 64^3 interior grid (262,144 DoFs): kappa = "
                                   "1 + mu_1 sin^2(20 pi r(x)) at the cell faces, affine Dirichlet data, mu uniform "
                                   "on [0,2]x[0,1], RB N<=20 by greedy over 70 training mu, %d test mu per step; "
                                   "each step forms the right-hand sides on the device and solves them from the "
                                   "Galerkin start with FP64 MG-PCG to rel-res 1e-10" % B,
                       "batch_per_gpu": B, "N": int(N), "warm": "galerkin", "precision": "fp64",
                       "precond": "mg", "tol": tol, "l2": "no flush: solver working set > 129 MB L2"},
            "clocks": clocks, "arms": arms, "t_off_s": t_off, "greedy_eta_last": float(eta[-1]),
            "iters_mean": head["iters_mean"], "relres_max": head["relres_max"], "oracle_error": head_err}
    if "mgcg_zero_fp64" in arms:
        line["speedup_vs_mgcg_zero_fp64"] = head["solves_per_s"] / arms["mgcg_zero_fp64"]["solves_per_s"]
    print(json.dumps(line), flush=True)
    P.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32ir", choices=["fp32ir", "fp64"])
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="FP32_IR reliable-update factor (0: the library default)")
    ap.add_argument("--precond", default="mg", choices=["mg", "jacobi"],
                    help="preconditioner of the headline arm: multigrid V-cycle (MGCG) or Jacobi")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the oracle's reference solutions (per-instance errors of every result)")
    ap.add_argument("--arm-steps", type=int, default=2, help="timed steps of each side arm (0: skip arms)")
    ap.add_argument("--batch", type=int, default=0, help="parameters per GPU and step (0: the workload's 256)")
    ap.add_argument("--mlp-epochs", type=int, default=2000,
                    help="epochs of the learned warm start's training (0: skip the learned arms)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c5", "c2g", "ex1"],
                    help="c2: the 64^3 batched workload (default line); c3: 128^3 octants, contrast 1e4, 64 mu; "
                         "c5: 96 requests on 96^3/128^3/256^3; c2g: the 64^3 operator with a Gaussian source "
                         "per parameter; ex1: the paper's Example 1 on 64^3")
    ap.add_argument("--c5-train", type=int, default=256, help="greedy training parameters per grid (c5)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the built-in FP32 tile/schedule instead of the autotuned one")
    ap.add_argument("--schedule", type=int, default=-1,
                    help="force an FP32 schedule (0..3) with the built-in tile instead of autotuning")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "c5":
        return bench_requests(args)
    if args.workload == "ex1":
        return bench_ex1(args)
    if args.workload == "c2g":
        return bench_gaussian(args)
    if args.workload == "c3":
        return bench_c3(args)

    import torch
    import torch.distributed as dist
    from paper_2311_13862_gb300 import build, inputs, ranks, rbws

    ri = ranks.rank_info()
    world, rank, local = ri.world, ri.rank, ri.local
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    build.build()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    w = inputs.WORKLOADS["c2"]
    B = args.batch or w.n_test
    # each rank solves its own batch of B parameters (weak scaling, no collective on the data path)
    mus = ranks.shard(inputs.test_mu(w, B * world), B, rank, world)
    # the oracle's FP64 solutions of this rank's parameters (MGCG from zero to 1e-13, spawned
    # worker processes, before any timed region): every solution of every arm is measured
    # against them below
    from oracle import batch as O_batch
    U_ref, oracle_ref = None, None
    if rank == 0 and not args.no_oracle_check:
        U_ref, r_it, r_rel, r_st, r_s, r_p = O_batch.reference_solutions(w.grid, mus, blocks=w.blocks, tol=1e-13)
        oracle_ref = {"solver": "oracle MGCG (FP64, scipy CSR) from zero", "tol": 1e-13, "instances": int(B),
                      "relres_max": float(r_rel.max()), "all_converged": bool(np.all(r_st == 0)),
                      "processes": r_p, "seconds": r_s}
    P = rbws.Problem(w.grid, w.blocks, device=local)
    t0 = time.perf_counter()
    N, sel, eta = rbws.rbws_offline_greedy(P.h, inputs.train_mu(w), w.n_max, 0.0, 1e-12)
    torch.cuda.synchronize()
    t_off = time.perf_counter() - t0
    # r_N: the largest (and mean) relative residual of the Galerkin RB solutions over the test set
    # with the first n basis vectors, n = 1..N (outside every timed region)
    r_curve = []
    for n in range(1, int(N) + 1):
        rr = rbws.rbws_rb_residuals(P.h, mus, n)
        r_curve.append([float(rr.max()), float(rr.mean())])
    # the residual manifold after k iterations of the RB-initialised Jacobi-PCG (FP64): relative
    # singular values of the B residual snapshots (a POD), as in the paper's n-width discussion
    residual_pod = {}
    if rank == 0:
        try:
            for k in (0, 10, 50, 150):
                uk = torch.empty((B, P.n), dtype=torch.float64, device="cuda")
                rbws.rbws_solve_batch(P.h, mus, 1e-15, rbws.WARM_GALERKIN, uk,
                                      rbws.rbws_options_default(max_iters=k, precond=rbws.PREC_JACOBI))
                au = torch.empty_like(uk)
                rbws.rbws_apply_operator(P.h, mus, uk, au)
                R = 1.0 - au  # residual snapshots (analysis only: the Gram matrix by torch)
                G = (R @ R.T).cpu().numpy()
                sv = np.sqrt(np.maximum(np.linalg.eigvalsh(G)[::-1], 0.0))
                residual_pod[str(k)] = [float(x) for x in sv[:21] / sv[0]]
                del uk, au, R
        except Exception as ex:  # an analysis field: never fails the bench
            residual_pod = {"error": str(ex)[:200]}

    tuned = None
    if args.schedule >= 0:
        # a one-line tuning cache forces the schedule (tile 16x16, z-chunks of 16)
        path = os.path.join(tempfile.mkdtemp(), "tiles.txt")
        with open(path, "w") as f:
            f.write("%dx%dx%d/B%d/fp32 16 16 16 1.0 %d\n" % (w.grid + (B, args.schedule)))
        tx, ty, zc, pair_ms, sched = rbws.rbws_autotune(P.h, B, path)
        tuned = {"tile": [tx, ty, zc], "schedule": sched, "forced": True}
    elif not args.no_autotune:
        t0 = time.perf_counter()
        tx, ty, zc, pair_ms, sched = rbws.rbws_autotune(P.h, B)
        tuned = {"tile": [tx, ty, zc], "schedule": sched, "pair_ms": pair_ms, "tune_s": time.perf_counter() - t0}
    stream = torch.cuda.Stream()
    u = torch.empty((B, P.n), dtype=torch.float64, device="cuda")
    prec = {"fp32ir": rbws.FP32_IR, "fp64": rbws.FP64}

    def run(warm, precision, steps, warmup, profile=False, precond=rbws.PREC_JACOBI, persistent=0):
        prof = rbws.rbws_profile()
        o = rbws.rbws_options_default(precision=precision, stream=stream.cuda_stream, precond=precond,
                                      persistent=persistent)
        if args.inner_tol > 0:
            o.inner_tol = args.inner_tol
        out = None
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                rbws.rbws_solve_batch(P.h, mus, w.tol, warm, u, o)
            if profile:
                import ctypes
                o.profile = ctypes.pointer(prof)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            acc = {"launches": 0, "samples": 0, "stencil_ms": 0.0, "update_ms": 0.0, "active_dofs": 0.0,
                   "precond_ms": 0.0, "mg_prolong_ms": 0.0}
            acc_fine = [0.0] * 4
            acc_schedule = None
            torch.cuda.nvtx.range_push("timed")
            e0.record(stream)
            for _ in range(steps):
                out = rbws.rbws_solve_batch(P.h, mus, w.tol, warm, u, o)
                if profile:
                    for k in acc:
                        acc[k] += getattr(prof, k)  # every key of acc is a field of rbws_profile
                    for k in range(4):
                        acc_fine[k] += prof.mg_fine_ms[k]
                    acc_schedule = prof.schedule
            e1.record(stream)
            torch.cuda.nvtx.range_pop()
            barrier()
        ms = ranks.max_over_ranks(e0.elapsed_time(e1) / steps, "cuda")
        rc, it, rel, st = out
        acc["elem_bytes"] = prof.elem_bytes
        acc["schedule"] = acc_schedule
        acc["mg_fine_ms"] = acc_fine
        return ms, it, rel, st, acc

    headline = prec[args.precision]
    head_pc = rbws.PREC_MG if args.precond == "mg" else rbws.PREC_JACOBI
    head_name = ("mgcg_galerkin_" if args.precond == "mg" else "galerkin_") + args.precision
    # ---- timed region of the headline arm, clocks sampled meanwhile ----
    with ClockSampler(local) as clk:
        ms, it, rel, st, acc = run(rbws.WARM_GALERKIN, headline, args.steps, args.warmup, profile=True,
                                   precond=head_pc)
    clocks = clk.summary()
    value = ranks.job_rate(B, world, ms)

    # ---- end to end: host parameters in, solution and counts back to pinned host memory.  As a
    # serving loop would, the solution of one step goes back on a copy stream while the next step
    # solves (two device and two pinned host buffers); every step's copy is inside the timed
    # region, and a buffer is reused only after its copy has left the device ----
    u_dev = [u, torch.empty_like(u)]
    u_hosts = [torch.empty((B, P.n), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    copied = [None, None]
    mu_pinned = torch.from_numpy(mus.copy()).pin_memory()
    o = rbws.rbws_options_default(precision=headline, stream=stream.cuda_stream, precond=head_pc)
    if args.inner_tol > 0:
        o.inner_tol = args.inner_tol
    e2e_steps = max(4, args.steps)  # the last copy is the only one not overlapped
    with torch.cuda.stream(stream):
        barrier()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            slot = k % 2
            if copied[slot] is not None:
                stream.wait_event(copied[slot])
            rbws.rbws_solve_batch(P.h, mu_pinned.numpy(), w.tol, rbws.WARM_GALERKIN, u_dev[slot], o)
            solved = torch.cuda.Event()
            solved.record(stream)
            copy_stream.wait_event(solved)
            with torch.cuda.stream(copy_stream):
                u_hosts[slot].copy_(u_dev[slot], non_blocking=True)
            copied[slot] = torch.cuda.Event()
            copied[slot].record(copy_stream)
        stream.synchronize()
        copy_stream.synchronize()
        barrier()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    u_host = u_hosts[(e2e_steps - 1) % 2]
    e2e_ms = ranks.max_over_ranks(e2e_ms, "cuda")

    # ---- side arms: zero start, the other precision, the learned starts, MSRB, L1ROC ----
    arms = {}
    J, M, PJ, PG = rbws.PREC_JACOBI, rbws.PREC_MG, rbws.FP32_IR, rbws.FP64
    arm_list = [] if args.arm_steps <= 0 else [
        ("galerkin_fp32ir", rbws.WARM_GALERKIN, PJ, J), ("zero_fp64", rbws.WARM_ZERO, PG, J),
        ("galerkin_fp64", rbws.WARM_GALERKIN, PG, J), ("zero_fp32ir", rbws.WARM_ZERO, PJ, J),
        # the same FP64 Jacobi-PCG as one persistent cooperative launch per solve
        ("galerkin_fp64_persistent", rbws.WARM_GALERKIN, PG, J), ("zero_fp64_persistent", rbws.WARM_ZERO, PG, J)]
    learned = None
    if args.arm_steps > 0 and args.mlp_epochs > 0:
        # learned warm start (same 64^3 problem): p -> 256 -> 256 -> 256 -> N network trained on
        # the GPU on the reduced Galerkin coefficients of 4096 seeded parameters; its arms run with
        # the headline's preconditioner and precision
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = rbws.rbws_train_surrogate(P.h, inputs.surrogate_mu(inputs.WORKLOADS["c4"], 4096), hidden=256,
                                         epochs=args.mlp_epochs, batch=256, lr=1e-3, mu_lo=w.mu_lo,
                                         mu_hi=w.mu_hi, seed=3004)
        learned = {"train_s": time.perf_counter() - t0, "final_loss": loss, "samples": 4096,
                   "epochs": args.mlp_epochs, "hidden": 256}
        pre = "mgcg_" if args.precond == "mg" else ""
        arm_list += [(pre + "learned_" + args.precision, rbws.WARM_LEARNED, headline, head_pc),
                     (pre + "learned_corrected_" + args.precision, rbws.WARM_LEARNED_CORRECTED, headline, head_pc)]
    if args.arm_steps > 0:
        # the RB-preconditioned start: Galerkin start, then PCG with the MSRB preconditioner
        # (Algorithm 3, FP64 only)
        arm_list.append(("msrb_fp64", rbws.WARM_GALERKIN, PG, rbws.PREC_MSRB))
        # MGCG (Algorithm 2 as the preconditioner), from zero and from the RB initial value
        arm_list += [("mgcg_zero_fp64", rbws.WARM_ZERO, PG, M), ("mgcg_galerkin_fp64", rbws.WARM_GALERKIN, PG, M),
                     ("mgcg_zero_fp32ir", rbws.WARM_ZERO, PJ, M), ("mgcg_galerkin_fp32ir", rbws.WARM_GALERKIN, PJ, M)]
        # the paper's own RBWS start: L1ROC (DEIM points, over-collocation), then MGCG; its offline
        # greedy replaces the Galerkin basis, so this arm runs last
        arm_list.append(("l1roc_mgcg_fp32ir", rbws.WARM_L1ROC, PJ, M))
    l1roc_off = None
    for name, warm, pr, pc in arm_list:
        if name == "l1roc_mgcg_fp32ir":
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            N1, _, eta1 = rbws.rbws_offline_l1roc(P.h, inputs.train_mu(w), w.n_max, 1e-12)
            torch.cuda.synchronize()
            l1roc_off = {"t_off_s": time.perf_counter() - t0, "N": int(N1),
                         "collocation_points": int(len(rbws.rbws_l1roc_info(P.h)[0]))}
        if name == head_name:
            a_ms, a_it, a_rel, a_st = ms, it, rel, st
            a_err = None
        else:
            a_ms, a_it, a_rel, a_st, _ = run(warm, pr, args.arm_steps, 1, precond=pc,
                                             persistent=int(name.endswith("_persistent")))
            # error of this arm's solutions against the oracle's FP64 solutions (every instance)
            a_err = None if U_ref is None else O_batch.relL2(u.cpu().numpy(), U_ref)
        arms[name] = {"solves_per_s": ranks.job_rate(B, world, a_ms), "ms_per_step": a_ms,
                      "iters_mean": float(np.mean(a_it)), "iters_max": int(np.max(a_it)),
                      "relres_max": float(np.max(a_rel)), "all_converged": bool(np.all(a_st == 0))}
        if a_err is not None:
            arms[name]["oracle_relL2_max"] = float(a_err.max())
            arms[name]["oracle_relL2_mean"] = float(a_err.mean())

    # ---- roofline of the dominant kernel, with the stencil phase beside it ----
    peak, peak_kind = peaks()
    eb = acc["elem_bytes"] or 8
    sched = acc.get("schedule")
    f32 = eb == 4
    # kernels of each schedule: (stencil-phase name, bytes/DoF, profile tag), (update-phase ...)
    kernels = {
        -1: (("k_cg_a<float> (one node per thread)", 16, None), ("k_cg_b<float>", 28, None)),
        0: (("k_cg_a_v4 (register prefetch: p = s + beta p, q = A p, p.q)", 16, None),
            ("k_cg_b_v4 (u += alpha p, r -= alpha q, s = D^-1 r, r.s, r.r)", 28, "cg_update_phase_f32_v4_64cube")),
        1: (("k_cg_a32_v4 (u += alpha' p_old, p = D^-1 r + beta p, p.A p)", 20, None),
            ("k_cg_b32_v4 (r -= alpha A p recomputed, r.s, r.r)", 12, None)),
        2: (("k_cg_a_tma (TMA-staged planes: p = s + beta p, q = A p, p.q)", 16, "cg_stencil_phase_f32_tma_64cube"),
            ("k_cg_b_v4 (u += alpha p, r -= alpha q, s = D^-1 r, r.s, r.r)", 28, "cg_update_phase_f32_v4_64cube")),
        3: (("k_cg_a_tma<1> (TMA-staged: u += alpha' p_old, p = s + beta p, p.A p)", 20,
             "cg_stencil_phase_f32_stma_64cube"),
            ("k_cg_b_s_tma (TMA-staged: s -= alpha D^-1 A p, r = D s, r.s, r.r)", 12, "cg_update_phase_f32_stma_64cube")),
    }
    if f32:
        (st_name, alg_stencil, st_tag), (up_name, alg_update, up_tag) = kernels[sched if sched in kernels else -1]
        if args.precond == "mg" and sched in (0, 2):
            # with the V-cycle as preconditioner the update phase stores no s
            up_name, alg_update, up_tag = ("k_cg_b_v4 (u += alpha p, r -= alpha q, r.r; s from the V-cycle)", 24,
                                           "cg_update_phase_f32_v4_mg_64cube")
            if sched == 2:
                st_tag = "cg_stencil_phase_f32_tma_mg_64cube"
    else:
        st_name, alg_stencil, st_tag = "k_cg_a<double> (FP64 stencil phase)", 32, None
        up_name, alg_update, up_tag = "k_cg_b<double> (FP64 update phase)", 56, None
    minimal = 6 * eb  # u, r, p read and written once per iteration
    res = {}
    if acc["samples"] > 0:
        launch_dofs = acc["active_dofs"] / acc["samples"]
        st_gbs = acc["active_dofs"] * alg_stencil / (acc["stencil_ms"] * 1e-3) / 1e9
        up_gbs = acc["active_dofs"] * alg_update / (acc["update_ms"] * 1e-3) / 1e9
        solver_gbs = acc["active_dofs"] * minimal / ((acc["stencil_ms"] + acc["update_ms"]) * 1e-3) / 1e9
        st_t = traffic_per_dof(st_tag) if st_tag else None
        up_t = traffic_per_dof(up_tag) if up_tag else None
        stencil = {"kernel": st_name, "achieved": round(st_gbs, 1), "frac": round(st_gbs / peak, 4),
                   "algorithmic_bytes_per_dof": alg_stencil, "ms_per_launch": acc["stencil_ms"] / acc["samples"],
                   "traffic": None if st_t is None else st_t * launch_dofs}
        update = {"kernel": up_name, "achieved": round(up_gbs, 1), "frac": round(up_gbs / peak, 4),
                  "algorithmic_bytes_per_dof": alg_update, "ms_per_launch": acc["update_ms"] / acc["samples"],
                  "traffic": None if up_t is None else up_t * launch_dofs}
        dom = update if acc["update_ms"] >= acc["stencil_ms"] else stencil
        if not f32:
            # FP64 kernels are bound by GB300's FP64 issue rate, not HBM: report them against the
            # FP64 FMA peak (1.25 TFLOP/s nominal; 1.196 measured on this machine's GB300 by a
            # dependent-free DFMA loop).  Flops per DoF: stencil phase 17 (p update 2, stencil
            # 13, p.q 2), update phase 9 (u 2, r 2, s 1, r.s 2, r.r 2).
            fp64_peak = 1196.0
            st_gf = acc["active_dofs"] * 17 / (acc["stencil_ms"] * 1e-3) / 1e9
            up_gf = acc["active_dofs"] * 9 / (acc["update_ms"] * 1e-3) / 1e9
            dom_gf = up_gf if dom is update else st_gf
            res = {"bound": "alu", "achieved": round(dom_gf, 1), "peak": fp64_peak, "unit": "GFLOP/s",
                   "frac": round(dom_gf / fp64_peak, 4), "traffic": dom["traffic"], "kernel": dom["kernel"],
                   "peak_kind": "FP64 FMA loop measured on GB300 (no MEASURED_PEAKS entry for FP64)",
                   "stencil_phase_gflops": round(st_gf, 1), "update_phase_gflops": round(up_gf, 1),
                   "hbm_stencil_phase": stencil, "hbm_update_phase": update, "sampled_launches": acc["samples"]}
            dom = None
    fine = []
    if acc["samples"] > 0 and dom is not None and args.precond == "mg" and sum(acc["mg_fine_ms"]) > 0:
        # the fused finest-level steps of each V-cycle: algorithmic bytes per DoF (FP32):
        # read r, write Y (8; the first step also reads omega/D, 4 B/DoF of traffic beyond the
        # algorithmic bytes); read Y, r, write the restricted residual at 1/8 of the nodes
        # (8.5); read and write Y, the coarse correction at 1/8 of the nodes, then read Y, r,
        # write X (8 + 0.5 + 12, two launches timed together); read X, r, write s (12)
        # (each a single kernel, timed by CUDA events around its own launch)
        fine_kernels = [("k_mg_smooth_od_tma (two damped Jacobi steps from zero, r and omega/D staged)", 8.0,
                         "mg_fine_smooth_od_f32_64cube"),
                        ("k_mg_fine_rr_tma (restricted residual P^T (r - A Y))", 8.5,
                         "mg_fine_residual_restrict_f32_64cube"),
                        ("k_mg_prolong_add4 (Y += P e)", 8.5, "mg_fine_prolong_smooth_f32_64cube#prolong"),
                        ("k_mg_smooth_tma<0,0> (damped Jacobi step)", 12.0, "mg_fine_prolong_smooth_f32_64cube#smooth"),
                        ("k_mg_smooth_tma<0,1> (damped Jacobi step + rho partials)", 12.0,
                         "mg_fine_smooth_rho_f32_64cube")]
        mf = acc["mg_fine_ms"]
        times = [mf[0], mf[1], acc["mg_prolong_ms"], mf[2] - acc["mg_prolong_ms"], mf[3]]
        for (name, alg, tag), t_ms in zip(fine_kernels, times):
            gbs = acc["active_dofs"] * alg / (t_ms * 1e-3) / 1e9
            tr = traffic_per_dof(tag) if tag else None
            fine.append({"kernel": name, "achieved": round(gbs, 1), "frac": round(gbs / peak, 4),
                         "algorithmic_bytes_per_dof": alg, "ms_per_launch": t_ms / acc["samples"],
                         "traffic": None if tr is None else tr * launch_dofs, "ms_total": t_ms})
        # the dominant kernel: the single kernel with the largest total time of the sampled ones
        phases = [dict(stencil, ms_total=acc["stencil_ms"]), dict(update, ms_total=acc["update_ms"])] + fine
        dom = max(phases, key=lambda k: k["ms_total"])
    if acc["samples"] > 0 and dom is not None:
        total_ms = acc["update_ms"] + acc["stencil_ms"] + acc["precond_ms"]
        res = {"bound": "hbm", "achieved": dom["achieved"], "peak": peak, "unit": "GB/s", "frac": dom["frac"],
               "traffic": dom["traffic"], "kernel": dom["kernel"], "peak_kind": peak_kind, "schedule": sched,
               "algorithmic_bytes_per_dof": dom["algorithmic_bytes_per_dof"],
               "dominant_share": round(dom.get("ms_total", max(acc["update_ms"], acc["stencil_ms"])) / total_ms, 3),
               "stencil_phase": stencil, "update_phase": update,
               "solver_frac_minimal_bytes": round(solver_gbs / peak, 4), "sampled_launches": acc["samples"]}
        if fine:
            res["mg_fine_steps"] = [dict({k: v for k, v in f.items() if k != "ms_total"},
                                         share=round(f["ms_total"] / total_ms, 3)) for f in fine]
            for ph in ("stencil_phase", "update_phase"):
                res[ph]["share"] = round(acc[ph.split("_")[0] + "_ms"] / total_ms, 3)
            res["vcycle_ms_per_iteration"] = acc["precond_ms"] / acc["samples"]
            res.pop("solver_frac_minimal_bytes")
            res["dominant_share_of"] = "the sampled iterations: phase A + phase B + V-cycle"

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 inner / f64 outer" if headline == rbws.FP32_IR else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch_per_gpu": B, "N": int(N), "warm": "galerkin",
                       "precision": args.precision, "precond": args.precond, "tol": w.tol,
                       "l2": "no flush: solver working set ~1.3 GB > 129 MB L2",
                       "parallelism": "independent batches per GPU (no collective)"},
            "roofline": res, "gpu_launches": int(acc["launches"]), "clocks": clocks,
            "e2e": {"value": ranks.job_rate(B, world, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": int(B * w.Q * 8),
                    "d2h_bytes_per_step": int(B * P.n * 8 + B * (4 + 8 + 4))},
            "arms": arms, "l1roc_offline": l1roc_off, "learned_training": learned, "autotune": tuned, "t_off_s": t_off, "greedy_eta_last": float(eta[-1]),
            "r_N_max_mean": r_curve, "residual_pod_sv": residual_pod,
            "iters_mean": float(np.mean(it)), "relres_max": float(np.max(rel))}
    if "zero_fp64" in arms:
        line["speedup_vs_zero_fp64"] = value / arms["zero_fp64"]["solves_per_s"]
        t_zero = 1.0 / (arms["zero_fp64"]["solves_per_s"] / world)
        t_warm = 1.0 / (value / world)
        line["bep_solves"] = t_off / (t_zero - t_warm) if t_zero > t_warm else None

    # ---- error of every headline solution against the oracle: relative L2 error against the
    # oracle's FP64 solution and the oracle's true relative residual (CSR operator) ----
    if U_ref is not None:
        es = O_batch.error_summary(w.grid, mus, u_host.numpy(), U_ref, blocks=w.blocks)
        line["oracle_error"] = {k: v for k, v in es.items() if k not in ("relL2", "true_relres")}
        line["oracle_error"]["reference"] = oracle_ref
        if head_name in arms:
            arms[head_name]["oracle_relL2_max"] = es["relL2_max"]
            arms[head_name]["oracle_relL2_mean"] = es["relL2_mean"]

    # ---- CPU baseline: the oracle on the host cores, bounded sample (rank 0, N = 1) ----
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        threads = O.default_threads()
        n_solves = max(threads, 16)
        basis, r, times, cpu_off = cpu_baseline(w, n_solves, threads, w.tol, 32, precond=args.precond)
        line["cpu_baseline"] = {"value": n_solves / times[0], "unit": UNIT,
                                "cores": getattr(r[0], "threads", threads), "kind": "oracle",
                                "sample": "%d of the 256 test mu, Galerkin warm start from an oracle greedy "
                                          "over the first 32 training mu (N=%d), %s FP64 to 1e-10; "
                                          "greedy took %.1f s (not in the rate)" %
                                          (n_solves, basis.N, "MGCG" if args.precond == "mg" else "Jacobi-PCG",
                                           cpu_off),
                                "iters_mean": float(r[0].iters.mean())}
    if rank == 0:
        print(json.dumps(line), flush=True)
    P.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
