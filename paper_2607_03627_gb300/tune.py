"""Autotuner for the row split of the iteration kernels.

The iteration kernels give each thread `rows_per_thread` rows (1, 2 or 4) of
one LP; the results do not depend on the choice, the speed does (more rows
per thread means more independent loads in flight per thread but fewer
CTAs).  The tuner times a few CUDA-graph replays of one representative LP of
each size bucket (by nonzeros) for every choice and keeps the fastest, cached
in a JSON file keyed by GPU name, bucket and value precision.
"""
from __future__ import annotations

import json
import os
import threading

from . import binding as B

CHOICES = (1, 2, 4)
CTA_CHOICES = (128, 256)
# nonzero-count buckets: [lo, hi)
BUCKETS = ((0, 1 << 17), (1 << 17, 1 << 19), (1 << 19, 1 << 21), (1 << 21, 1 << 62))
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")


def bucket_of(nnz: int) -> int:
    for i, (lo, hi) in enumerate(BUCKETS):
        if lo <= nnz < hi:
            return i
    return len(BUCKETS) - 1


class Tuner:
    def __init__(self, cache_path: str | None = DEFAULT_CACHE, trial_replays: int = 16):
        self.cache_path = cache_path
        self.trial_replays = trial_replays
        self._lock = threading.Lock()
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            try:
                with open(cache_path) as f:
                    self.cache = json.load(f)
            except (OSError, ValueError):
                self.cache = {}

    @staticmethod
    def _gpu_name() -> str:
        import torch
        return torch.cuda.get_device_name()

    def key(self, nnz: int, value_bits: int) -> str:
        return f"{self._gpu_name()}|bucket{bucket_of(nnz)}|fp{value_bits}"

    def time_choice(self, ps, rpt: int, cta: int = 0) -> float:
        """Milliseconds per PDHG iteration of `ps` with `rpt` rows per thread
        and `cta` threads per CTA (0: the library default): `trial_replays`
        graph replays of 64 iterations after a warm-up solve, timed on the
        device."""
        import torch
        n_eval = 64
        replays = max(2, self.trial_replays)
        sess = B.Session([ps], tol=0.0, max_iter=n_eval * replays, rows_per_thread=[rpt], cta_rows=cta)
        sess.reset(-1)
        sess.run()                       # warm-up (graph already captured)
        s = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sess.reset(-1)
        sess.run(1)                      # the reset's start-point evaluation and one replay
        e0.record(s)
        sess.run()                       # the remaining replays, steady state
        e1.record(s)
        torch.cuda.synchronize()
        sess.close()
        return e0.elapsed_time(e1) / (n_eval * (replays - 1))

    def choose(self, ps, value_bits: int) -> int:
        nnz = B.uc_presolved_dims(ps)[3]
        k = self.key(nnz, value_bits)
        with self._lock:
            if k in self.cache:
                return int(self.cache[k]["rows_per_thread"])
        times = {r: self.time_choice(ps, r) for r in CHOICES}
        best = min(times, key=times.get)
        with self._lock:
            self.cache[k] = {"rows_per_thread": best, "ms_per_iter": times, "nnz_sample": nnz}
            if self.cache_path:
                tmp = self.cache_path + f".tmp{os.getpid()}"
                with open(tmp, "w") as f:
                    json.dump(self.cache, f, indent=1)
                os.replace(tmp, self.cache_path)
        return best

    def choose_pair(self, ps, value_bits: int) -> tuple[int, int]:
        """(threads per CTA, rows per thread) for a session holding `ps` alone."""
        nnz = B.uc_presolved_dims(ps)[3]
        k = "pair|" + self.key(nnz, value_bits)
        with self._lock:
            if k in self.cache:
                e = self.cache[k]
                return int(e["cta_rows"]), int(e["rows_per_thread"])
        # two rounds, interleaved, best of both: the choices differ by a few
        # percent, so each trial times 15 steady-state replays
        pairs = [(c, r) for c in CTA_CHOICES for r in CHOICES if r <= 2]
        times = {p: float("inf") for p in pairs}
        for _ in range(2):
            for c, r in pairs:
                times[(c, r)] = min(times[(c, r)], self.time_choice(ps, r, c))
        best = min(times, key=times.get)
        with self._lock:
            self.cache[k] = {"cta_rows": best[0], "rows_per_thread": best[1],
                             "ms_per_iter": {f"{c}x{r}": t for (c, r), t in times.items()}, "nnz_sample": nnz}
            if self.cache_path:
                tmp = self.cache_path + f".tmp{os.getpid()}"
                with open(tmp, "w") as f:
                    json.dump(self.cache, f, indent=1)
                os.replace(tmp, self.cache_path)
        return best
