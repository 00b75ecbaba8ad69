"""Continuous-batching server for unit-commitment LP requests on one GPU.

Requests share a grid and unit fleet and differ in load (day-ahead re-solves),
so every request's scaled matrix is the base LP's.  The server keeps one
device-resident session whose slots hold the base matrix; admitting a
request replaces a free slot's right-hand side and bounds (uc_session_update_lp,
no matrix upload), warm-starts it from the solved request with the nearest
net-load vector, and resets just that slot while the other slots keep
iterating.  A warm-started request that ends without meeting the tolerance
is solved again from the cold start in its slot.  Finished slots are harvested between short runs of CUDA-graph
replays and refilled from the queue (continuous batching).  The number of
slots is capped by an HBM budget.  Host presolve (uc_presolve_reuse: the
base LP's scaling is reused) runs on a thread pool as requests arrive.

Because every slot's arithmetic is independent and deterministic, a request
returns the same iterates and solution alone or in the mix (tested).  With 2
or 4 slots the session is a shared-matrix ("lanes") session: the base matrix
is stored once, the slots' vectors are interleaved, and every matrix row is
read once for all slots.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import math
import threading
import time

import numpy as np

from . import binding as B


@dataclasses.dataclass
class Request:
    rid: int
    problem: object          # ucgen.UCProblem-like
    arrival: float           # seconds after the stream starts
    admitted: float = math.nan
    finished: float = math.nan
    status: int = 1
    iters: int = 0
    objective: float = math.nan
    rel_kkt: float = math.nan
    warm_from: int = -1
    slot: int = -1
    start_x: np.ndarray | None = None    # warm start actually used (scaled presolved)
    start_y: np.ndarray | None = None
    start_omega: float = 0.0
    omega: float = math.nan              # final primal weight
    x: np.ndarray | None = None          # returned point (scaled presolved)
    y: np.ndarray | None = None
    retried_cold: bool = False           # the warm start failed and the request was solved cold
    warm_iters: int = 0                  # iterations spent on the failed warm start

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Server:
    def __init__(self, base_problem, slots: int = 8, hbm_budget_gb: float = 150.0, tol: float = 1e-4,
                 max_iter: int = 100_000, value_bits: int = 64, warm_start: bool = True,
                 replays_per_step: int = 4, presolve_workers: int = 8, keep_solutions: bool = False,
                 warm_policy: str = "dual", lanes: bool | None = None):
        if warm_policy not in ("dual", "full"):
            raise ValueError("warm_policy must be 'dual' or 'full'")
        self.warm_policy = warm_policy
        self.tol = tol
        self.warm_start = warm_start
        self.replays = replays_per_step
        self.keep = keep_solutions
        self.base_lp = B.uc_build_lp(base_problem)
        self.base_ps = B.uc_presolve(self.base_lp, value_bits=value_bits)
        self.n, self.m, _, _ = B.uc_presolved_dims(self.base_ps)
        # slots the HBM budget allows (bytes of a one-slot session, scaled)
        probe = B.Session([self.base_ps], tol=tol, max_iter=max_iter)
        per_slot = probe.device_bytes()
        probe.close()
        fit = max(1, int(hbm_budget_gb * 1e9 // per_slot))
        self.slots = max(1, min(slots, fit))
        self.bytes_per_slot = per_slot
        # 2 or 4 slots share one stored matrix and interleave their vectors
        # (a lanes session) unless told otherwise
        self.lanes = (self.slots in (2, 4)) if lanes is None else (bool(lanes) and self.slots in (2, 4))
        self.sess = B.Session([self.base_ps] * self.slots, tol=tol, max_iter=max_iter, lanes=self.lanes)
        self.pool = cf.ThreadPoolExecutor(max_workers=presolve_workers)
        self.library: list[tuple] = []   # (load, x, y, rid, omega) of solved requests

    def close(self):
        self.sess.close()
        self.pool.shutdown(wait=False)

    def _presolve(self, req: Request):
        lp = B.uc_build_lp(req.problem)
        return B.uc_presolve_reuse(self.base_ps, lp)

    def _nearest(self, load: np.ndarray):
        if not self.library:
            return None
        d = [float(np.linalg.norm(load - entry[0])) for entry in self.library]
        j = int(np.argmin(d))
        return self.library[j]

    def serve(self, requests: list[Request], realtime: bool = True) -> dict:
        """Serve the requests (arrival times relative to now); returns metrics."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        futures: dict[int, cf.Future] = {}
        queue: list[Request] = []            # arrived, waiting for presolve / a slot
        running: dict[int, Request] = {}     # slot -> request
        free = list(range(self.slots))
        done = 0
        nxt = 0
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else None
        sim_t = 0.0
        gpu_busy = 0.0
        while done < len(reqs):
            now = clock() if realtime else sim_t
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                r = reqs[nxt]
                futures[r.rid] = self.pool.submit(self._presolve, r)
                queue.append(r)
                nxt += 1
            # admit in arrival order while slots are free and presolve is ready
            while free and queue and futures[queue[0].rid].done():
                r = queue.pop(0)
                ps = futures.pop(r.rid).result()
                slot = free.pop(0)
                self.sess.update_lp(slot, ps)
                load = np.ascontiguousarray(r.problem.load, dtype=np.float64).ravel()
                near = self._nearest(load) if self.warm_start else None
                if near is not None:
                    # warm start from the neighbour's dual and primal weight (the
                    # "dual" policy): on the 6,049-bus grid its primal point slowed
                    # the solves down, its duals and weight saved a few percent
                    if self.warm_policy == "full":
                        self.sess.set_start(slot, near[1], near[2], near[4])
                    else:
                        self.sess.set_start(slot, None, near[2], near[4])
                    r.warm_from = near[3]
                    r.start_omega = near[4]
                    if self.keep:
                        r.start_x = near[1].copy() if self.warm_policy == "full" else None
                        r.start_y = near[2].copy()
                self.sess.reset(slot)
                r.slot = slot
                r.admitted = clock() if realtime else sim_t
                r._ps = ps
                r._load = load
                running[slot] = r
            if running:
                g0 = time.perf_counter()
                self.sess.run(self.replays)
                g = time.perf_counter() - g0
                gpu_busy += g
                if not realtime:
                    sim_t += g
                for slot in list(running):
                    st = self.sess.status(slot)
                    if st == 2:
                        continue
                    r = running[slot]
                    res, rc = self.sess.result(slot)
                    stats = B.uc_get_stats(res)
                    if rc != B.UC_OK and r.warm_from >= 0 and not r.retried_cold:
                        # a warm start can stall the method (the neighbour's primal
                        # weight can be far from this request's): solve it again from
                        # the cold start in the same slot, which holds its LP already
                        r.retried_cold = True
                        r.warm_iters = stats["iters"]
                        r.start_x = r.start_y = None     # the start the result comes from
                        r.start_omega = 0.0
                        self.sess.set_start(slot, None, None, 0.0)
                        self.sess.reset(slot)
                        continue
                    running.pop(slot)
                    r.finished = clock() if realtime else sim_t
                    r.status = rc
                    r.iters = stats["iters"]
                    r.objective = stats["objective"]
                    r.rel_kkt = max(stats["rel_primal"], stats["rel_dual"], stats["rel_gap"])
                    r.omega = stats["omega"]
                    x, y = B.uc_get_iterate(res, 2, self.n, self.m)
                    if self.keep:
                        r.x, r.y = x, y
                    if rc == B.UC_OK:
                        self.library.append((r._load, x, y, r.rid, r.omega))
                    del r._ps, r._load
                    free.append(slot)
                    done += 1
            else:
                # idle: wait for the next arrival or a presolve to finish
                if realtime:
                    waits = [reqs[nxt].arrival - now] if nxt < len(reqs) else []
                    time.sleep(min([0.002] + [w for w in waits if w > 0]))
                else:
                    if queue:
                        futures[queue[0].rid].result()
                    elif nxt < len(reqs):
                        sim_t = max(sim_t, reqs[nxt].arrival)
        lat = np.array([r.latency for r in reqs])
        span = max(r.finished for r in reqs) - min(r.arrival for r in reqs)
        return {"requests": len(reqs), "slots": self.slots, "lanes": self.lanes, "bytes_per_slot": self.bytes_per_slot,
                "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                "mean_latency_s": float(lat.mean()), "throughput_req_per_s": len(reqs) / span,
                "makespan_s": span, "gpu_busy_s": gpu_busy,
                "mean_iters": float(np.mean([r.iters for r in reqs])),
                "warm_started": int(sum(r.warm_from >= 0 for r in reqs)),
                "retried_cold": int(sum(r.retried_cold for r in reqs)),
                "all_optimal": bool(all(r.status == B.UC_OK for r in reqs))}


def sequential_baseline(requests: list[Request], base_problem, tol: float = 1e-4, max_iter: int = 100_000,
                        value_bits: int = 64) -> dict:
    """Plain one-at-a-time cold FP64 solves of the same requests in arrival
    order (each starts when it has arrived and the previous one finished)."""
    base_ps = B.uc_presolve(B.uc_build_lp(base_problem), value_bits=value_bits)
    sess = B.Session([base_ps], tol=tol, max_iter=max_iter)
    t = 0.0
    lat = []
    iters = []
    reqs = sorted(requests, key=lambda r: r.arrival)
    for r in reqs:
        ps = B.uc_presolve_reuse(base_ps, B.uc_build_lp(r.problem))
        g0 = time.perf_counter()
        sess.update_lp(0, ps)
        sess.reset(0)
        sess.run()
        res, rc = sess.result(0)
        g = time.perf_counter() - g0
        iters.append(B.uc_get_stats(res)["iters"])
        t = max(t, r.arrival) + g
        lat.append(t - r.arrival)
    sess.close()
    lat = np.array(lat)
    return {"p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "throughput_req_per_s": len(reqs) / (t - reqs[0].arrival), "mean_iters": float(np.mean(iters)),
            "note": "device time of cold solves replayed on a simulated clock; presolve not counted"}


def session_bytes_estimate(ps, value_bits: int = 64, max_iter: int = 100_000) -> int:
    """Device bytes of a one-LP session of `ps`, estimated from its sizes: the
    matrix and its transpose (int32 indices, FP64 or FP32 values, row pointers),
    the period-strided slot records, eight constant and start vectors and ten
    state vectors per column or row, and the Halpern weight tables."""
    n, m, _, nnz = B.uc_presolved_dims(ps)
    vs = 4 if value_bits == 32 else 8
    slot = 8 if value_bits == 32 else 16
    per_col = 4 + 8 * 8 + 5 * 8 + slot
    per_row = 4 + 4 * 8 + 5 * 8 + slot
    tables = 2 * 8 * min(max_iter + 1, 1 << 22)
    return int(1.05 * (2 * nnz * (4 + vs) + n * per_col + m * per_row + tables) + (1 << 20))


class MixedServer:
    """Continuous batching of UC requests on grids of any size.

    A shared-matrix session needs one scaled matrix for all its slots, so
    requests on different grids cannot share one.  Here every admitted request
    gets a session of its own, with its own CUDA stream, driven by a worker
    thread: requests that arrive while others are on the GPU are admitted in
    arrival order as soon as a worker is free and the HBM budget holds their
    session (estimated from their sizes, then measured for each grid seen), and
    the kernels of the running sessions overlap on the device.  Presolve runs on
    a thread pool as requests arrive; a request on a grid already seen reuses
    that grid's scaling (uc_presolve_reuse).  Each session's arithmetic is its
    own, so a request's iterates and solution are those of a solve alone, bit
    for bit (tested).
    """

    def __init__(self, max_active: int = 4, hbm_budget_gb: float = 150.0, tol: float = 1e-4,
                 max_iter: int = 100_000, value_bits: int = 64, presolve_workers: int = 8,
                 keep_solutions: bool = False):
        self.max_active = max(1, int(max_active))
        self.budget = float(hbm_budget_gb) * 1e9
        self.tol = tol
        self.max_iter = max_iter
        self.value_bits = value_bits
        self.keep = keep_solutions
        self.pool = cf.ThreadPoolExecutor(max_workers=presolve_workers)
        self.workers = cf.ThreadPoolExecutor(max_workers=self.max_active)
        self.bases: list = []          # presolved base LP of every grid seen
        self.grid_bytes: dict = {}     # measured session bytes by LP sizes
        self.lock = threading.Lock()

    def close(self):
        self.pool.shutdown(wait=True)
        self.workers.shutdown(wait=True)

    def _presolve(self, req: Request):
        lp = B.uc_build_lp(req.problem)
        with self.lock:
            bases = list(self.bases)
        for base in bases:
            try:
                return B.uc_presolve_reuse(base, lp)
            except B.UCError:
                continue
        ps = B.uc_presolve(lp, value_bits=self.value_bits)
        with self.lock:
            self.bases.append(ps)
        return ps

    def _need(self, ps) -> int:
        key = B.uc_presolved_dims(ps)
        return self.grid_bytes.get(key, session_bytes_estimate(ps, self.value_bits, self.max_iter))

    def _solve(self, r: Request, ps, t0: float):
        import torch
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            sess = B.Session([ps], tol=self.tol, max_iter=self.max_iter)
            nbytes = sess.device_bytes()
            sess.reset(-1)
            sess.run()
            res, rc = sess.result(0)
            stats = B.uc_get_stats(res)
            n, m, _, _ = B.uc_presolved_dims(ps)
            x, y = B.uc_get_iterate(res, 2, n, m)
            sess.close()
        r.finished = time.perf_counter() - t0
        r.status = rc
        r.iters = stats["iters"]
        r.objective = stats["objective"]
        r.rel_kkt = max(stats["rel_primal"], stats["rel_dual"], stats["rel_gap"])
        r.omega = stats["omega"]
        if self.keep:
            r.x, r.y = x, y
        return nbytes

    def serve(self, requests: list[Request]) -> dict:
        """Serve the requests (arrival times in seconds from now); returns metrics."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        futures = {}
        queue: list[Request] = []
        running = {}                   # future -> (request, reserved bytes, size key)
        used = 0
        peak_active = 0
        nxt = 0
        done = 0
        while done < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                r = reqs[nxt]
                futures[r.rid] = self.pool.submit(self._presolve, r)
                queue.append(r)
                nxt += 1
            while queue and futures[queue[0].rid].done() and len(running) < self.max_active:
                ps = futures[queue[0].rid].result()
                need = self._need(ps)
                if running and used + need > self.budget:
                    break                   # wait for memory (one request always runs)
                r = queue.pop(0)
                del futures[r.rid]
                r.admitted = time.perf_counter() - t0
                r.slot = len(running)
                f = self.workers.submit(self._solve, r, ps, t0)
                running[f] = (r, need, B.uc_presolved_dims(ps))
                used += need
                peak_active = max(peak_active, len(running))
            finished = [f for f in running if f.done()]
            for f in finished:
                r, need, key = running.pop(f)
                nbytes = f.result()
                self.grid_bytes[key] = nbytes
                used -= need
                done += 1
            if not finished:
                waits = [reqs[nxt].arrival - now] if nxt < len(reqs) else []
                time.sleep(min([0.002] + [w for w in waits if w > 0]))
        lat = np.array([r.latency for r in reqs])
        span = max(r.finished for r in reqs) - min(r.arrival for r in reqs)
        return {"requests": len(reqs), "max_active": self.max_active, "peak_active": peak_active,
                "hbm_budget_gb": self.budget / 1e9,
                "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                "mean_latency_s": float(lat.mean()), "throughput_req_per_s": len(reqs) / span,
                "makespan_s": span, "mean_iters": float(np.mean([r.iters for r in reqs])),
                "all_optimal": bool(all(r.status == B.UC_OK for r in reqs))}
