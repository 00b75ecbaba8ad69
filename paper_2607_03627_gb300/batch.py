"""Batched solves: many UC LPs of uneven size in one block-diagonal session.

All LPs are packed block-diagonally into one session, so every PDHG iteration
is one primal and one dual launch for the whole batch (captured in a CUDA
graph); each LP keeps its own step sizes, restarts and stopping test, and the
session drops finished LPs from its launch tables as the batch shrinks.  The
row split of each LP comes from the autotuner, per size bucket.
"""
from __future__ import annotations

import concurrent.futures as cf
import time

from . import binding as B
from .tune import Tuner, bucket_of


def presolve_all(problems, value_bits: int = 64, workers: int = 8, **kw):
    """uc_build_lp + uc_presolve (options ``kw``) for every problem, on host threads."""
    def one(P):
        return B.uc_presolve(B.uc_build_lp(P), value_bits=value_bits, **kw)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(one, problems))


def solve_batch(pss, tol: float = 1e-4, max_iter: int = 100_000, tuner: Tuner | None = None,
                value_bits: int = 64, **kw):
    """Solve presolved LPs together.  Returns (results, info): results[i] is
    (ResultHandle, status) of LP i; info has the wall time, the row split of
    every LP and the session's device bytes."""
    rpts = None
    if tuner is not None:
        rep = {}
        for p in pss:
            b = bucket_of(B.uc_presolved_dims(p)[3])
            rep.setdefault(b, p)
        chosen = {b: tuner.choose(p, value_bits) for b, p in rep.items()}
        rpts = [chosen[bucket_of(B.uc_presolved_dims(p)[3])] for p in pss]
    import torch
    t0 = time.perf_counter()
    sess = B.Session(pss, tol=tol, max_iter=max_iter, rows_per_thread=rpts, **kw)
    t1 = time.perf_counter()
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    sess.reset(-1)
    sess.run()
    e1.record(s)
    torch.cuda.synchronize()
    results = [sess.result(i) for i in range(len(pss))]
    info = {"solve_ms": e0.elapsed_time(e1), "setup_ms": (t1 - t0) * 1e3, "rows_per_thread": rpts,
            "device_bytes": sess.device_bytes()}
    sess.close()
    return results, info
