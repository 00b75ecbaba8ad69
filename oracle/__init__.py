"""CPU oracle for the unit-commitment LP relaxation solved by restarted PDHG.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package; only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline / reference arm of ``bench.py`` use it.  It shares no code
with the CUDA path: the only common input is the seeded data generator in
``ucgen`` (problem data, no solver arithmetic).

Contents (each function cites the passage it follows; the paper defers its UC
model to the GO Challenge 3 specification (Sec. II-A) and names PDHG without
stating it (Sec. II-C, Sec. III-C), so the model follows the DC relaxation the
benchmark configurations define and the PDHG follows the published PDLP method
(Applegate et al., NeurIPS 2021) with constant steps, or with PDLP's adaptive
step size as an option of the averaging variant):

* ``lp``        -- O-builder: raw DC-UC LP from problem data (Sec. II-A/II-B,
                   Alg. 1 "same relaxed problem").
* ``presolve``  -- fixed columns, singleton rows to bounds, empty rows/columns,
                   Ruiz + Pock-Chambolle scaling, power iteration for ||A||_2,
                   postsolve (Sec. II-D presolve, reduced form).
* ``kkt``       -- relative KKT residuals of the presolved LP (stopping test,
                   convergence tolerance 1e-4, Sec. II-D).
* ``pdhg``      -- O1: plain FP64 restarted PDHG (Sec. II-C solver 1).
* ``simplex``   -- O2: dense bounded-variable primal simplex (plain C).
* ``brute``     -- O3: vertex and commitment enumeration on micro instances.
* ``closed``    -- O4: one-bus merit order, two-bus congestion, PTDF flows.

Parity status: every function is pinned by tests under ``tests/`` against
brute force, closed forms or invariants (the absolute feasibility figure
``kkt.abs_primal_inf``, reported only, against element-by-element loops and
the simplex optimum).
"""
