"""Write the stored expected values under tests/golden/ from the oracle alone.

    python tests/golden/make_golden.py

Calls only ``oracle`` (and ``ucgen`` for the seeded inputs); nothing here
touches the CUDA path.  Outputs:

* tiny_lp.json -- the 30-bus / 6-unit / 24-period LP relaxation (seed 0):
  raw and presolved sizes and the exact LP optimum from the dense simplex,
  plus the optima of seeds 1-3 (``objective_by_seed``).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import ucgen  # noqa: E402
from oracle import kkt, lp as olp, presolve as ops, simplex  # noqa: E402


def tiny_lp():
    out = {"config": "30 buses, 41 lines, 6 units, 24 periods, load 0.4-0.8 of capacity, VOLL 1e4",
           "seed": 0, "objective_by_seed": {}}
    for seed in range(4):
        P = ucgen.tiny(seed)
        raw = olp.build_lp(P)
        ps = ops.presolve(raw)
        t = time.time()
        r = simplex.solve_lp(ps.lp)
        assert r.status == "optimal", r.status
        rel = kkt.relative_kkt(ps.lp, r.x, r.y)
        assert max(rel) <= 1e-9, rel
        out["objective_by_seed"][str(seed)] = r.obj
        if seed == 0:
            out.update(raw_n=raw.n, raw_m=raw.m, raw_m_eq=raw.m_eq, raw_nnz=int(raw.A.nnz),
                       n=ps.lp.n, m=ps.lp.m, m_eq=ps.lp.m_eq, nnz=int(ps.lp.A.nnz),
                       objective=r.obj, simplex_iters=r.iters, max_rel_kkt=max(rel))
        print(f"seed {seed}: obj {r.obj:.10g} ({r.iters} pivots, {time.time() - t:.1f} s)")
    with open(os.path.join(HERE, "tiny_lp.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    tiny_lp()
