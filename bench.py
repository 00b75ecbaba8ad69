#!/usr/bin/env python
"""Benchmark: restarted PDHG on the 6,049-bus / 700-unit / 48-period UC LP relaxation.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config ...]

One step = one solve of the whole hot path on the device-resident presolved LP:
reset to the cold start, PDHG iterations in CUDA-graph replays of 64, KKT /
restart evaluation every 64 iterations, until relative KKT <= 1e-4.  `value`
is PDHG iterations per second summed over ranks (weak scaling: every rank
solves its own copy; no collective on the data path).  Time-to-1e-4 per LP,
the algorithmic HBM bandwidth and the kernel roofline are reported beside it.
`e2e` repeats the step through the public C ABI from host arrays (LP build,
presolve with its power iteration on the device, upload, solve, download,
postsolve).  `--impl reference` times the CPU oracle (the same algorithm,
plain numpy) on a bounded sample.

Other configurations (`--config`): paper-fp32 (FP32 matrix values), tiny
(30 buses, with the dense simplex timed too), batch64 (64 uneven LPs in one
block-diagonal session against one-at-a-time solves), served (a Poisson
request stream through the continuous-batching server, 2 shared-matrix slots,
cold starts unless --warm-start), paper-lanes (load variants sharing one
stored matrix).  `--algorithm average [--adaptive-step]` selects PDLP
averaging, optionally with its adaptive step size.
"""
import os

# the CPU oracle legs use exactly one core; set before numpy is imported
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-4 KKT per UC LP; PDHG iters/s and HBM GB/s; p50/p99 served latency"
UNIT = "PDHG iter/s"
TOL = 1e-4
MAX_ITER = 100_000

# DRAM bytes per launch of the iteration kernels from one ncu capture with
# --cache-control none (steady-state L2), 6,049-bus LP, FP64 values, Halpern
# (profiles/pdhg_kernels_grid6049.md; mean read + mean written over three
# launches): valid only for the kernel source they were taken on (the hash of
# the row kernels' section of uc_device.cu, the device layout and the
# strided-slot builder) and the launch shape (threads per CTA, rows per thread).
NCU_TRAFFIC = {}
NCU_TRAFFIC_RPT2 = {
    ("paper", "halpern", "k_primal"): {"src": "2332a82d9f753da8", "launch": (128, 2), "bytes": 36162645 + 4488107},
    ("paper", "halpern", "k_dual"): {"src": "2332a82d9f753da8", "launch": (128, 2), "bytes": 16699563 + 2484651},
}


def _src_hash():
    """sha256 (16 hex digits) of the row kernels and their helpers in uc_device.cu,
    of the code that lays the LP out in device order and of the builder of the
    period-strided slot records."""
    with open(os.path.join(ROOT, "paper_2607_03627_gb300", "csrc", "uc_device.cu")) as f:
        src = f.read()
    a = src.index("// FP64 is scarce on this GPU")
    b = src.index("// staged iteration kernels (Halpern)")
    c = src.index("// Device view of an LP.")
    d = src.index("// same scaled matrix (structure, values as stored, equality rows)")
    e = src.index("// Slot records of the period-strided groups")
    f_ = src.index("// natural-order vector -> device order")
    return hashlib.sha256((src[a:b] + src[c:d] + src[e:f_]).encode()).hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max_sum(values, device):
    """Across ranks: (max of values[0], sum of values[1]) -- the job's wall time
    (slowest rank) and its total work.  Single process: returned as is."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(values[0]), float(values[1])
    t = torch.tensor([float(values[0]), float(values[1])], device=device, dtype=torch.float64)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return tmax[0].item(), tsum[1].item()


def bytes_per_iter(n, m, nnz, vs, algorithm="halpern"):
    """Algorithmic bytes of the primal (A^T y) and dual (A x-bar) kernels: the
    matrix and its row pointers once, every vector element touched once.
    Halpern: primal reads x, c, l, u, x0, gathers y, writes x-bar and x;
    dual gathers x-bar, reads y, q, y0, writes y.  Averaging: primal reads x,
    c, l, u, sum and writes x+, sum; dual gathers x+ and x, reads y, q, sum,
    writes y+, sum."""
    mat = nnz * (vs + 4)
    if algorithm == "halpern":
        return mat + 4 * (n + 1) + 8 * m + 56 * n, mat + 4 * (m + 1) + 8 * n + 32 * m
    # averaging, constant or adaptive step (the adaptive kernels add the previous
    # attempt's accepted point to the sums, so they touch the same vectors)
    return mat + 4 * (n + 1) + 8 * m + 56 * n, mat + 4 * (m + 1) + 16 * n + 40 * m


# FP64 instructions the device issues per row (FP64 FMA/add/mul each count 1;
# selections, clipping and FP32 widening run on the integer pipe; the
# accumulators start at -c / -q, so the step is one FMA).  Halpern per column:
# the row's FMAs, the step, the reflection, (1 - w) x0 and the combination;
# averaging: the row's FMAs (dual: two per entry), the step and the sum.
def fp64_inst_per_iter(n, m, nnz, algorithm="halpern"):
    if algorithm == "halpern":
        return nnz + 4 * n, nnz + 4 * m
    if algorithm == "average-adaptive":
        # primal per column: the step, clip bounds, dx, dx^2 and the sum (FP64 min / max
        # counted); dual per entry: x-bar, its FMA, dx and the A dx FMA; per row: the
        # step, projection, dy, dy^2, dy (A dx) and the sum
        return nnz + 6 * n, 4 * nnz + 6 * m
    return nnz + 2 * n, 2 * nnz + 2 * m


# GPU-wide FP64 pipe issue rate: 2 thread-instructions per SM per clock
# (sm__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained = 304 on 152 SMs)
FP64_INST_PER_CLK = 304


def make_workload(name, rank):
    import ucgen
    if name in ("paper", "paper-fp32"):
        P = ucgen.paper_scale(0)
        desc = dict(workload="UC LP relaxation, 6049 buses / 8000 lines / 700 units / 48 periods",
                    buses=P.B, lines=P.L, units=P.G, periods=P.T, seed=0)
    elif name == "tiny":
        P = ucgen.tiny(0)
        desc = dict(workload="UC LP relaxation, 30 buses / 41 lines / 6 units / 24 periods",
                    buses=P.B, lines=P.L, units=P.G, periods=P.T, seed=0)
    else:
        raise SystemExit(f"unknown config {name}")
    return P, desc, (32 if name == "paper-fp32" else 64)


def _gains(args):
    return None if not args.pw_gains else tuple(float(v) for v in args.pw_gains.split(","))


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300 import binding as B

    P, desc, vbits = make_workload(args.config, rank)
    t0 = time.perf_counter()
    lp = B.uc_build_lp(P)
    pw_dev = 0 if args.power_host else 1
    ps = B.uc_presolve(lp, value_bits=vbits, power_device=pw_dev, aggressive=int(args.aggressive),
                       eliminate_angles=int(args.angles))
    presolve_s = time.perf_counter() - t0
    n, m, m_eq, nnz = B.uc_presolved_dims(ps)
    vs = 4 if vbits == 32 else 8
    if args.rows_per_thread or args.cta_rows:
        rpt, cta = args.rows_per_thread or 1, args.cta_rows
    else:
        from paper_2607_03627_gb300.tune import Tuner
        cta, rpt = Tuner().choose_pair(ps, vbits)
    sess = B.Session([ps], tol=TOL, max_iter=args.max_iter, kernel_timing=True, spmv_kernel=args.spmv_kernel,
                     stages=args.stages,
                     rows_per_thread=[rpt], cta_rows=cta,
                     algorithm=args.algorithm, restart_metric=args.restart_metric, pdl=not args.no_pdl,
                     adaptive_step=args.adaptive_step, pw_gains=_gains(args), pw_guard=args.pw_guard,
                     reorder=not args.no_reorder)

    def solve_once():
        sess.reset(-1)
        sess.run()

    def read_stats():
        res, rc = sess.result(0)
        st = B.uc_get_stats(res)
        return res, st

    for _ in range(args.warmup):
        solve_once()
    _, st_w = read_stats()
    tp0, td0, nt0 = st_w["primal_kernel_ms"] * st_w["timed_launches"], st_w["dual_kernel_ms"] * st_w["timed_launches"], st_w["timed_launches"]
    launches0 = st_w["kernel_launches"]

    stream = torch.cuda.current_stream()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            solve_once()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    res, st = read_stats()
    # every timed solve starts cold from the same point and takes the same path
    iters = [st["iters"]] * args.steps
    ms_max, total_iters = reduce_max_sum([ms, float(sum(iters))], "cuda")
    value = total_iters / (ms_max / 1e3)
    n_timed = st["timed_launches"] - nt0
    tp = (st["primal_kernel_ms"] * st["timed_launches"] - tp0) / max(n_timed, 1)
    td = (st["dual_kernel_ms"] * st["timed_launches"] - td0) / max(n_timed, 1)
    alg_key = "average-adaptive" if args.adaptive_step else args.algorithm
    bp, bd = bytes_per_iter(n, m, nnz, vs, alg_key)
    fp, fd = fp64_inst_per_iter(n, m, nnz, alg_key)
    pname, dname = ("k_ad_primal", "k_ad_dual") if args.adaptive_step else ("k_primal", "k_dual")
    peak, peak_kind = _peaks()
    clk_sum = clk.summary()
    sm_mhz = clk_sum.get("sm_mhz") or 2070.0
    fp64_peak = FP64_INST_PER_CLK * sm_mhz * 1e6 / 1e9      # G FP64 instructions / s
    kern = {}
    for name, b_, f_, t_ in ((pname, bp, fp, tp), (dname, bd, fd, td)):
        if t_ <= 0:
            continue
        gbs = b_ / (t_ / 1e3) / 1e9
        gis = f_ / (t_ / 1e3) / 1e9
        kern[name] = {"mean_launch_us": t_ * 1e3, "algorithmic_bytes_per_launch": b_,
                      "fp64_inst_per_launch": f_,
                      "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak},
                      "alu_fp64": {"achieved": gis, "peak": fp64_peak, "unit": "G FP64 inst/s",
                                   "frac": gis / fp64_peak}}
    dom = max(kern, key=lambda k: kern[k]["mean_launch_us"]) if kern else pname
    dk = kern.get(dom, {"hbm": {"frac": 0, "achieved": 0, "peak": peak, "unit": "GB/s"},
                        "alu_fp64": {"frac": 0, "achieved": 0, "peak": fp64_peak, "unit": ""},
                        "mean_launch_us": 0, "algorithmic_bytes_per_launch": 0})
    bound = "alu" if dk["alu_fp64"]["frac"] >= dk["hbm"]["frac"] else "hbm"
    main = dk["alu_fp64"] if bound == "alu" else dk["hbm"]
    traffic = None
    rec = (NCU_TRAFFIC if rpt == 1 else NCU_TRAFFIC_RPT2).get((args.config, args.algorithm, dom))
    # the capture was taken on the default presolve's LP
    if (args.spmv_kernel != 2 and not args.angles and not args.aggressive and rec and rec["src"] == _src_hash()
            and tuple(rec["launch"]) == (cta or 128, rpt)):
        traffic = rec["bytes"]
    roofline = {"bound": bound, "kernel": dom, "achieved": main["achieved"], "peak": main["peak"],
                "unit": main["unit"], "frac": main["frac"], "traffic": traffic,
                "peak_kind": (peak_kind if bound == "hbm" else
                              "derived: 304 FP64 thread-instructions/clock x median SM clock"),
                "other_bound": ({"bound": "hbm", **dk["hbm"]} if bound == "alu"
                                else {"bound": "alu", **dk["alu_fp64"]}),
                "timed_launches": n_timed, "kernels": kern}
    per_iter_ms = ms_max / max(total_iters / world, 1)
    alg_gbs = (bp + bd) / (per_iter_ms / 1e3) / 1e9

    # end to end through the public API from host arrays
    e2e = None
    if args.e2e_steps > 0:
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        tot_it = 0
        h2d = d2h = 0
        for _ in range(args.e2e_steps):
            lp2 = B.uc_build_lp(P)
            ps2 = B.uc_presolve(lp2, value_bits=vbits, power_device=pw_dev, aggressive=int(args.aggressive),
                                eliminate_angles=int(args.angles))
            r2, rc2 = B.uc_solve(ps2, tol=TOL, max_iter=args.max_iter, algorithm=args.algorithm,
                                 adaptive_step=args.adaptive_step,
                                 restart_metric=args.restart_metric)
            sol = B.uc_get_solution(r2, P.T, P.B, P.L, P.G)
            tot_it += sol["stats"]["iters"]
            h2d += sol["stats"]["h2d_bytes"]
            d2h += sol["stats"]["d2h_bytes"]
        e2e_s = time.perf_counter() - t0
        e2e_s, tot_it = reduce_max_sum([e2e_s, float(tot_it)], "cuda")
        e2e = {"value": tot_it / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d // args.e2e_steps),
               "d2h_bytes_per_step": int(d2h // args.e2e_steps),
               "seconds_per_lp": e2e_s / args.e2e_steps,
               "includes": "uc_build_lp + uc_presolve (power iteration for ||A|| on the %s) + uc_solve "
                           "(upload, solve, download) + uc_get_solution" % ("host" if args.power_host else "device")}

    # primal feasibility polishing (outside the timed region): the paper's
    # absolute feasibility tolerance of 1e-5 (Sec. II-D) on the same solve
    polish = None
    if not args.no_polish and not args.adaptive_step and args.algorithm == "halpern":
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rp_, rcp = B.uc_solve(ps, tol=TOL, max_iter=args.max_iter, rows_per_thread=[rpt], cta_rows=cta,
                              pw_gains=_gains(args), pw_guard=args.pw_guard, polish=True, tol_abs_feas=1e-5)
        sp = B.uc_get_stats(rp_)
        polish = {"status": sp["status_name"], "main_iters": sp["iters"], "polish_iters": sp["polish_iters"],
                  "abs_primal_before": sp["abs_primal_unpolished"], "abs_primal_after": sp["abs_primal"],
                  "rel_kkt_after": max(sp["rel_primal"], sp["rel_dual"], sp["rel_gap"]),
                  "wall_s": time.perf_counter() - t0, "tol_abs_feas": 1e-5}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(P, args.cpu_iters, desc["workload"], simplex=args.config == "tiny")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if vbits == 64 else "f32-values/f64",
            "data": "synthetic (seeded generator standing in for the GO3 6,049-bus cases)",
            "config": dict(desc, n=n, m=m, nnz=nnz, matrix_values=f"fp{vbits}", vectors="fp64",
                           tol_rel_kkt=TOL, max_iter=args.max_iter, n_eval=64,
                           algorithm=args.algorithm, restart_metric=args.restart_metric,
                           presolve="+".join(k for k, on in (("aggressive", args.aggressive), ("angles", args.angles))
                                             if on) or "default",
                           adaptive_step=bool(args.adaptive_step),
                           rows_per_thread=rpt, cta_rows=cta or 128,
                           l2="inputs larger than L2 (working set %.0f MB > 126 MB)" % ((bp + bd) / 1e6),
                           parallelism=f"replicas x{world}"),
            "time_to_1e-4_ms": ms_max / args.steps,
            "iters_per_solve": st["iters"], "status": st["status_name"], "rejected_steps": st["rejected_steps"],
            "rel_kkt": max(st["rel_primal"], st["rel_dual"], st["rel_gap"]),
            "objective": st["objective"], "restarts": st["restarts"],
            "pdhg_iters_per_s_per_gpu": total_iters / world / (ms_max / 1e3),
            "algorithmic_GBps": alg_gbs, "bytes_per_iter": bp + bd,
            "presolve_s": presolve_s, "power_iteration": "host" if args.power_host else "device",
            "roofline": roofline,
            "clocks": clk_sum,
            "gpu_launches": st["kernel_launches"] - launches0,
            "e2e": e2e,
            "polish": polish,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def cpu_baseline(P, iters, workload, simplex=False):
    """The oracle PDHG as it stands, single core, on a bounded sample of the
    workload: `iters` iterations (evaluations every 64 included) on the same LP
    the oracle builds, presolves and scales itself (that set-up is not timed).
    With `simplex` (the 30-bus workload only) the oracle's dense simplex is
    timed on the presolved LP as well."""
    from oracle import lp as olp, pdhg, presolve as ops
    raw = olp.build_lp(P)
    ps = ops.presolve(raw)
    S = ops.scale(ps.lp)
    st = pdhg.halpern_initial_state(S)
    AT = S.A.T.tocsr()
    U = pdhg._unscaled_lp(S)
    t0 = time.perf_counter()
    for _ in range(iters):
        pdhg.halpern_step(S, st, AT)
        if st.k % pdhg.N_EVAL == 0:
            pdhg.halpern_evaluate(S, st, U, TOL)
    dt = time.perf_counter() - t0
    out = {"value": iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{iters} PDHG iterations (with {iters // 64} KKT/restart evaluations) of the oracle "
                     f"on the same LP ({workload}); oracle build/presolve/scaling not timed",
           "seconds": dt}
    if simplex:
        from oracle import simplex as osx
        t0 = time.perf_counter()
        r = osx.solve_lp(ps.lp)
        out["simplex"] = {"seconds": time.perf_counter() - t0, "status": r.status, "objective": r.obj,
                          "iterations": r.iters, "note": "oracle dense bounded simplex, one core"}
    return out


def run_reference(args):
    """The CPU oracle as the reference arm: each step is one 64-iteration
    block (PDHG steps + one KKT/restart evaluation) of the paper-scale LP."""
    world, rank, local = _dist()
    if rank != 0:
        return
    import ucgen  # noqa: F401
    from oracle import lp as olp, pdhg, presolve as ops
    P, desc, vbits = make_workload(args.config if args.config != "paper-fp32" else "paper", rank)
    raw = olp.build_lp(P)
    ps = ops.presolve(raw)
    S = ops.scale(ps.lp)
    st = pdhg.halpern_initial_state(S)
    AT = S.A.T.tocsr()
    U = pdhg._unscaled_lp(S)

    def block():
        for _ in range(pdhg.N_EVAL):
            pdhg.halpern_step(S, st, AT)
        pdhg.halpern_evaluate(S, st, U, TOL)

    for _ in range(args.warmup):
        block()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        block()
    dt = time.perf_counter() - t0
    value = args.steps * pdhg.N_EVAL / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator standing in for the GO3 6,049-bus cases)",
            "config": dict(desc, n=S.A.shape[1], m=S.A.shape[0], nnz=int(S.A.nnz),
                           step="64 oracle PDHG iterations + 1 KKT/restart evaluation"),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} x 64 iterations after {args.warmup} warm-up blocks"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """64 uneven UC LPs (buses log-uniform in [300, 6049], T in {24, 48}, seeds
    1-64) in one block-diagonal session with FP32 (or, --value-bits 64, FP64) matrix values and autotuned
    row splits, against one-at-a-time FP64 solves of the same LPs."""
    import numpy as np
    import torch
    import ucgen
    torch.cuda.set_device(0)
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300 import binding as B
    from paper_2607_03627_gb300.batch import presolve_all, solve_batch
    from paper_2607_03627_gb300.tune import Tuner
    probs = [ucgen.batch_member(s) for s in range(1, args.batch + 1)]
    vb = args.value_bits
    t0 = time.perf_counter()
    ps32 = presolve_all(probs, value_bits=vb, eliminate_angles=int(args.angles))
    presolve_s = time.perf_counter() - t0
    tuner = Tuner()
    kw = dict(restart_metric=args.restart_metric, pw_gains=_gains(args), pw_guard=args.pw_guard)
    solve_batch(ps32, tol=TOL, max_iter=args.max_iter, tuner=tuner, value_bits=vb, **kw)      # warm-up + tuning
    with ClockSampler(0) as clk:
        res32, info = solve_batch(ps32, tol=TOL, max_iter=args.max_iter, tuner=tuner, value_bits=vb, **kw)
    st32 = [B.uc_get_stats(r) for r, _ in res32]
    line = {"metric": METRIC, "value": args.batch / (info["solve_ms"] / 1e3), "unit": "UC LP/s",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": info["solve_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32-values/f64" if vb == 32 else "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.batch} UC LPs, buses log-uniform in [300, 6049], T 24/48, seeds 1-{args.batch}",
                       "total_nnz": int(sum(B.uc_presolved_dims(p)[3] for p in ps32)),
                       "matrix_values": f"fp{vb}", "vectors": "fp64", "tol_rel_kkt": TOL,
                       "max_iter": args.max_iter, "presolve": "angles" if args.angles else "default"},
            "rows_per_thread": info["rows_per_thread"], "all_optimal": all(s["status"] == 0 for s in st32),
            "per_lp": [{"buses": P.B, "T": P.T, "iters": s["iters"], "status": s["status_name"],
                        "rel_kkt": max(s["rel_primal"], s["rel_dual"], s["rel_gap"])} for P, s in zip(probs, st32)],
            "max_iters": max(s["iters"] for s in st32), "presolve_s": presolve_s,
            "device_bytes": info["device_bytes"], "clocks": clk.summary(), "impl": "ours"}
    if not args.no_sequential:
        ps64 = presolve_all(probs, value_bits=64, eliminate_angles=int(args.angles))
        tot_ms = 0.0
        errs = []
        seq_iters = []
        for p, (r32, _), s32 in zip(ps64, res32, st32):
            sess = B.Session([p], tol=TOL, max_iter=args.max_iter, **kw)
            sess.reset(-1); sess.run()                      # warm-up
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(); sess.reset(-1); sess.run(); e1.record(); torch.cuda.synchronize()
            tot_ms += e0.elapsed_time(e1)
            r64, _ = sess.result(0)
            s64 = B.uc_get_stats(r64)
            o64 = s64["objective"]
            seq_iters.append((s64["iters"], s64["status_name"]))
            errs.append(abs(s32["objective"] - o64) / max(1.0, abs(o64)))
            sess.close()
        line["sequential_fp64"] = {"ms": tot_ms, "lp_per_s": args.batch / (tot_ms / 1e3), "per_lp": seq_iters,
                                   "note": "one-at-a-time FP64 sessions, device-resident, summed device time"}
        line["speedup_vs_sequential_fp64"] = tot_ms / info["solve_ms"]
        line["objective_gap_vs_fp64"] = {"max": max(errs), "mean": float(np.mean(errs))}
    print(json.dumps(line), flush=True)


def run_lanes(args):
    """Shared-matrix session: `--lanes` (2 or 4) load variants of the 6,049-bus
    grid (served-request recipe, wave 0) presolved with the base scaling and
    solved together with the matrix stored once and the vectors interleaved,
    against the same LPs solved one at a time on the device (FP64)."""
    import torch
    import ucgen
    torch.cuda.set_device(0)
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300 import binding as B
    base = ucgen.paper_scale(0)
    base_ps = B.uc_presolve(B.uc_build_lp(base))
    pss = [B.uc_presolve_reuse(base_ps, B.uc_build_lp(ucgen.served_request(base, 0, r))) for r in range(args.lanes)]
    n, m, _, nnz = B.uc_presolved_dims(pss[0])
    sess = B.Session(pss, tol=TOL, max_iter=args.max_iter, lanes=True)
    for _ in range(args.warmup):
        sess.reset(-1); sess.run()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            sess.reset(-1); sess.run()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    st = [B.uc_get_stats(sess.result(i)[0]) for i in range(args.lanes)]
    sess.close()
    lp_iters = sum(s["iters"] for s in st)
    line = {"metric": METRIC, "value": lp_iters / (ms / 1e3), "unit": "LP-PDHG iter/s (summed over lanes)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.lanes} load variants (x0.80..) of the 6049-bus / 700-unit / 48-period LP, "
                                   "one shared-matrix session", "n": n, "m": m, "nnz": nnz, "lanes": args.lanes,
                       "tol_rel_kkt": TOL},
            "per_lp": [{"iters": s["iters"], "status": s["status_name"], "objective": s["objective"]} for s in st],
            "all_optimal": all(s["status"] == 0 for s in st), "clocks": clk.summary(), "impl": "ours"}
    if not args.no_sequential:
        tot = 0.0
        seq = []
        for p in pss:
            s1 = B.Session([p], tol=TOL, max_iter=args.max_iter)
            s1.reset(-1); s1.run()
            a = torch.cuda.Event(enable_timing=True); b_ = torch.cuda.Event(enable_timing=True)
            a.record(stream); s1.reset(-1); s1.run(); b_.record(stream); torch.cuda.synchronize()
            tot += a.elapsed_time(b_)
            seq.append(B.uc_get_stats(s1.result(0)[0])["iters"])
            s1.close()
        line["sequential_fp64"] = {"ms": tot, "iters": seq, "lp_iter_per_s": sum(seq) / (tot / 1e3)}
        line["speedup_vs_sequential"] = tot / ms
    print(json.dumps(line), flush=True)


def run_served(args):
    """Served stream: requests on the 6,049-bus grid with loads scaled by
    {0.80..1.20} and AR(1) noise, Poisson arrivals at 2 req/s, continuous
    batching (2 slots in a shared-matrix session; warm starts with
    --warm-start), against one-at-a-time cold FP64 solves."""
    import torch
    import ucgen
    torch.cuda.set_device(0)
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300.serve import Request, Server, sequential_baseline
    base = ucgen.paper_scale(0)
    reqs = []
    t = 0.0
    for w in range((args.requests + 44) // 45):
        n = min(45, args.requests - 45 * w)
        arr = ucgen.poisson_arrivals(100 + w, n, 2.0) + t
        if args.burst:               # the whole wave arrives at once, when its first request would
            arr[:] = arr[0]
        for r in range(n):
            reqs.append(Request(rid=45 * w + r, problem=ucgen.served_request(base, w, r), arrival=float(arr[r])))
        t = float(arr[-1]) if not args.burst else float(ucgen.poisson_arrivals(100 + w, n, 2.0)[-1] + t)
    srv = Server(base, slots=args.slots, hbm_budget_gb=args.hbm_budget_gb, tol=TOL, max_iter=args.max_iter,
                 warm_start=args.warm_start)
    with ClockSampler(0) as clk:
        m = srv.serve(reqs, realtime=True)
    srv.close()
    line = {"metric": METRIC, "value": m["p50_latency_s"], "unit": "s (p50 served latency)",
            "n_gpus": 1, "steps": len(reqs), "warmup": 0, "ms_per_step": m["makespan_s"] / len(reqs) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"{len(reqs)} requests on the 6049-bus / 700-unit / 48-period grid, "
                                            "load x{0.80..1.20} + AR(1) 5%, Poisson 2 req/s" +
                                            (", each wave in one burst" if args.burst else ""),
                                            "slots": m["slots"], "hbm_budget_gb": args.hbm_budget_gb,
                                            "tol_rel_kkt": TOL, "warm_start": args.warm_start},
            "served": m, "clocks": clk.summary(), "impl": "ours",
            "per_request": [{"rid": r.rid, "iters": r.iters, "status": r.status, "warm_from": r.warm_from,
                             "latency_s": r.latency, "omega": r.omega, "start_omega": r.start_omega}
                            for r in sorted(reqs, key=lambda r: r.rid)]}
    if not args.no_sequential:
        line["sequential_fp64_cold"] = sequential_baseline(reqs, base, tol=TOL, max_iter=args.max_iter)
    print(json.dumps(line), flush=True)


def run_served_mixed(args):
    """Served stream of requests on grids of different sizes (the batch
    members' grids: 300 to 6,049 buses, T 24/48), Poisson arrivals at
    `--rate` req/s, continuous batching with one session per admitted request
    on its own stream (MixedServer, `--slots` at most, HBM budget
    `--hbm-budget-gb`), against one-at-a-time cold FP64 solves of the same
    requests replayed on a simulated clock."""
    import numpy as np
    import torch
    import ucgen
    torch.cuda.set_device(0)
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300 import binding as B
    from paper_2607_03627_gb300.serve import MixedServer, Request
    arr = ucgen.poisson_arrivals(200, args.requests, args.rate)
    probs = [ucgen.batch_member(1 + (r % 64)) for r in range(args.requests)]
    reqs = [Request(rid=r, problem=probs[r], arrival=float(arr[r])) for r in range(args.requests)]
    srv = MixedServer(max_active=args.slots, hbm_budget_gb=args.hbm_budget_gb, tol=TOL, max_iter=args.max_iter)
    with ClockSampler(0) as clk:
        m = srv.serve(reqs)
    srv.close()
    line = {"metric": METRIC, "value": m["p50_latency_s"], "unit": "s (p50 served latency)",
            "n_gpus": 1, "steps": len(reqs), "warmup": 0, "ms_per_step": m["makespan_s"] / len(reqs) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{len(reqs)} requests on grids of 300-6049 buses (batch members 1-64, cycled), "
                                   f"Poisson {args.rate} req/s", "max_active": args.slots,
                       "hbm_budget_gb": args.hbm_budget_gb, "tol_rel_kkt": TOL},
            "served": m, "clocks": clk.summary(), "impl": "ours",
            "per_request": [{"rid": r.rid, "buses": r.problem.B, "iters": r.iters, "status": r.status,
                             "latency_s": r.latency} for r in reqs]}
    if not args.no_sequential:
        t = 0.0
        lat = []
        for r in reqs:
            ps = B.uc_presolve(B.uc_build_lp(r.problem))
            sess = B.Session([ps], tol=TOL, max_iter=args.max_iter)
            g0 = time.perf_counter()
            sess.reset(-1)
            sess.run()
            sess.result(0)
            g = time.perf_counter() - g0
            sess.close()
            t = max(t, r.arrival) + g
            lat.append(t - r.arrival)
        lat = np.array(lat)
        line["sequential_fp64_cold"] = {
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "throughput_req_per_s": len(reqs) / (t - reqs[0].arrival),
            "note": "device-resident cold solves one at a time, replayed on a simulated clock; presolve and "
                    "upload not counted"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="paper",
                    choices=["paper", "paper-fp32", "tiny", "batch64", "served", "served-mixed", "paper-lanes"])
    ap.add_argument("--lanes", type=int, default=4, help="paper-lanes: LPs in the shared-matrix session (2 or 4)")
    ap.add_argument("--batch", type=int, default=64, help="batch64: number of LPs")
    ap.add_argument("--value-bits", type=int, default=32, choices=[32, 64],
                    help="batch64: matrix values of the batched session (the one-at-a-time baseline is FP64)")
    ap.add_argument("--requests", type=int, default=45, help="served: requests (45 per wave)")
    ap.add_argument("--slots", type=int, default=2, help="served: session slots (served-mixed: sessions at once)")
    ap.add_argument("--hbm-budget-gb", type=float, default=150.0, help="served: HBM budget for admission")
    ap.add_argument("--burst", action="store_true", help="served: every wave arrives at once")
    ap.add_argument("--rate", type=float, default=2.0, help="served-mixed: Poisson arrival rate (req/s)")
    ap.add_argument("--warm-start", action="store_true",
                    help="served: warm-start requests from the nearest solved one (duals + primal weight)")
    ap.add_argument("--no-sequential", action="store_true", help="batch64/served: skip the one-at-a-time baseline")
    ap.add_argument("--max-iter", type=int, default=MAX_ITER)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--power-host", action="store_true",
                    help="presolve's power iteration for ||A|| on host threads instead of the device")
    ap.add_argument("--cpu-iters", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--spmv-kernel", type=int, default=0,
                    help="0 default (thread per row), 1 thread per row, 2 staged")
    ap.add_argument("--stages", type=int, default=0, help="staged kernels: chunks in flight per CTA (0: 2)")
    ap.add_argument("--algorithm", default="halpern", choices=["halpern", "average"])
    ap.add_argument("--adaptive-step", action="store_true",
                    help="PDLP adaptive step size (needs --algorithm average)")
    ap.add_argument("--no-pdl", action="store_true", help="no programmatic dependent launch")
    ap.add_argument("--no-reorder", action="store_true", help="keep the natural row/column order on the device")
    ap.add_argument("--cta-rows", type=int, default=0, help="threads per CTA of the iteration kernels (0: 128)")
    ap.add_argument("--rows-per-thread", type=int, default=0,
                    help="row split of the iteration kernels (0: autotuned, else 1, 2 or 4)")
    ap.add_argument("--restart-metric", default="kkt", choices=["kkt", "fpr", "fprp"])
    ap.add_argument("--aggressive", action="store_true",
                    help="paper configs: aggressive presolve (doubleton equations substituted)")
    ap.add_argument("--angles", action="store_true",
                    help="paper and batch configs: bus angles substituted out along a spanning tree")
    ap.add_argument("--no-polish", action="store_true",
                    help="skip the untimed feasibility-polishing solve reported beside the line")
    ap.add_argument("--pw-gains", default=None,
                    help="primal-weight controller gains kp,ki,kd (default: the library's)")
    ap.add_argument("--pw-guard", type=float, default=None,
                    help="residual-balance guard kappa on the primal-weight update (0: off; default: the library's)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batch64":
        run_batch(args)
    elif args.config == "paper-lanes":
        run_lanes(args)
    elif args.config == "served":
        run_served(args)
    elif args.config == "served-mixed":
        run_served_mixed(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
