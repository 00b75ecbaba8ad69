"""ctypes binding of libucpdhg.so: the C ABI of include/uc_pdhg.h with the same
names.  It only marshals arguments; every step of the solve runs in the
library (host presolve in C++, PDHG in the sm_103a kernels).  There is no
fallback: if the library is missing or cannot load, import fails loudly.

Device memory for uc_solve comes from PyTorch's caching allocator and the
solve runs on PyTorch's current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libucpdhg.so")

UC_OK, UC_EINVAL, UC_ENOMEM, UC_EINFEASIBLE, UC_EUNBOUNDED = 0, -1, -2, -3, -4
UC_EITERLIMIT, UC_ETIMEOUT, UC_ENUMERIC, UC_ECANCELLED, UC_ECUDA = -5, -6, -7, -8, -9
STATUS_NAMES = {0: "optimal", -1: "invalid", -2: "out_of_memory", -3: "infeasible",
                -4: "unbounded", -5: "iteration_limit", -6: "timeout", -7: "numeric",
                -8: "cancelled", -9: "cuda_error"}

_P = C.POINTER
_d = _P(C.c_double)
_i = _P(C.c_int32)


class uc_problem(C.Structure):
    _fields_ = [("B", C.c_int), ("L", C.c_int), ("G", C.c_int), ("T", C.c_int), ("ref_bus", C.c_int),
                ("line_from", _i), ("line_to", _i), ("x_pu", _d), ("fmax", _d),
                ("gen_bus", _i), ("pmax", _d), ("pmin", _d), ("ramp", _d), ("c_lin", _d),
                ("c_nl", _d), ("c_su", _d), ("u0", _d), ("load", _d), ("voll", C.c_double)]


class uc_presolve_opts(C.Structure):
    _fields_ = [("ruiz_iters", C.c_int), ("pock_chambolle", C.c_int), ("power_max_iter", C.c_int),
                ("power_tol", C.c_double), ("value_bits", C.c_int), ("threads", C.c_int),
                ("aggressive", C.c_int), ("power_device", C.c_int), ("eliminate_angles", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class uc_solve_opts(C.Structure):
    _fields_ = [("tol_rel_kkt", C.c_double), ("tol_abs_feas", C.c_double), ("max_iter", C.c_int),
                ("n_eval", C.c_int), ("use_graph", C.c_int), ("kernel_timing", C.c_int),
                ("timeout_ms", C.c_double), ("warm_x", _d), ("warm_y", _d), ("warm_omega", C.c_double),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
                ("spmv_kernel", C.c_int), ("cta_rows", C.c_int), ("rows_per_thread", _P(C.c_int)),
                ("no_reorder", C.c_int), ("no_pdl", C.c_int), ("algorithm", C.c_int),
                ("restart_metric", C.c_int),
                ("cancel", _P(C.c_int)), ("stages", C.c_int), ("lanes", C.c_int),
                ("adaptive_step", C.c_int), ("pw_kp", C.c_double), ("pw_ki", C.c_double),
                ("pw_kd", C.c_double), ("polish", C.c_int), ("polish_max_iter", C.c_int),
                ("pw_guard", C.c_double)]


class uc_device_lp(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("m_eq", C.c_int),
                ("A_rowptr", C.c_void_p), ("A_colidx", C.c_void_p), ("A_val", C.c_void_p),
                ("AT_rowptr", C.c_void_p), ("AT_colidx", C.c_void_p), ("AT_val", C.c_void_p),
                ("c", C.c_void_p), ("l", C.c_void_p), ("u", C.c_void_p), ("Dc", C.c_void_p),
                ("q", C.c_void_p), ("Dr", C.c_void_p), ("q_inf", C.c_double), ("c_inf", C.c_double)]


class uc_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("restarts", C.c_int), ("evals", C.c_int),
                ("returned_average", C.c_int), ("rel_primal", C.c_double), ("rel_dual", C.c_double),
                ("rel_gap", C.c_double), ("abs_primal", C.c_double), ("objective", C.c_double),
                ("dual_objective", C.c_double), ("omega", C.c_double), ("solve_ms", C.c_double),
                ("upload_ms", C.c_double), ("primal_kernel_ms", C.c_double),
                ("dual_kernel_ms", C.c_double), ("timed_launches", C.c_int),
                ("kernel_launches", C.c_int), ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64),
                ("rejected_steps", C.c_int), ("polish_iters", C.c_int), ("superbasic", C.c_int),
                ("abs_primal_unpolished", C.c_double)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


_SIGS = {
    "uc_default_presolve_opts": (None, [_P(uc_presolve_opts)]),
    "uc_default_solve_opts": (None, [_P(uc_solve_opts)]),
    "uc_build_lp": (C.c_int, [_P(uc_problem), _P(C.c_void_p)]),
    "uc_lp_dims": (C.c_int, [C.c_void_p, _P(C.c_int), _P(C.c_int), _P(C.c_int), _P(C.c_int64)]),
    "uc_lp_export": (C.c_int, [C.c_void_p, _i, _i, _d, _d, _d, _d, _d]),
    "uc_presolve": (C.c_int, [C.c_void_p, _P(uc_presolve_opts), _P(C.c_void_p)]),
    "uc_presolve_reuse": (C.c_int, [C.c_void_p, C.c_void_p, _P(C.c_void_p)]),
    "uc_presolved_dims": (C.c_int, [C.c_void_p, _P(C.c_int), _P(C.c_int), _P(C.c_int), _P(C.c_int64)]),
    "uc_presolved_export": (C.c_int, [C.c_void_p, _i, _i, _d, _d, _d, _d, _d, _d, _d, _i, _i, _d]),
    "uc_solve": (C.c_int, [C.c_void_p, _P(uc_solve_opts), C.c_void_p, _P(C.c_void_p)]),
    "uc_solve_batch": (C.c_int, [_P(C.c_void_p), C.c_int, _P(uc_solve_opts), C.c_void_p, _P(C.c_void_p)]),
    "uc_get_solution": (C.c_int, [C.c_void_p, _d, _d, _d, _d, _d, _d, _d, _P(uc_stats)]),
    "uc_get_raw_solution": (C.c_int, [C.c_void_p, _d, _d]),
    "uc_crossover": (C.c_int, [C.c_void_p, C.c_int64, _P(C.c_void_p)]),
    "uc_result_from_point": (C.c_int, [C.c_void_p, _d, _d, _P(C.c_void_p)]),
    "uc_simplex_solve": (C.c_int, [C.c_void_p, C.c_int64, _P(C.c_int), _P(C.c_void_p)]),
    "uc_solve_concurrent": (C.c_int, [C.c_void_p, _P(uc_solve_opts), C.c_void_p, _P(C.c_void_p), _P(C.c_int)]),
    "uc_get_iterate": (C.c_int, [C.c_void_p, C.c_int, _d, _d]),
    "uc_presolved_device_order": (C.c_int, [C.c_void_p, C.c_int, _P(C.c_int32), _P(C.c_int32)]),
    "uc_presolved_strided_groups": (C.c_int, [C.c_void_p, C.c_int, _P(C.c_int64), _P(C.c_int32),
                                              _P(C.c_int32), _P(C.c_int32), _d]),
    "uc_session_create": (C.c_int, [_P(C.c_void_p), C.c_int, _P(uc_solve_opts), C.c_void_p, _P(C.c_void_p)]),
    "uc_session_reset": (C.c_int, [C.c_void_p, C.c_int]),
    "uc_session_run": (C.c_int, [C.c_void_p, C.c_int, _P(C.c_int)]),
    "uc_session_status": (C.c_int, [C.c_void_p, C.c_int]),
    "uc_session_result": (C.c_int, [C.c_void_p, C.c_int, _P(C.c_void_p)]),
    "uc_session_set_start": (C.c_int, [C.c_void_p, C.c_int, _d, _d, C.c_double]),
    "uc_session_update_lp": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "uc_session_device_bytes": (C.c_size_t, [C.c_void_p]),
    "uc_session_free": (None, [C.c_void_p]),
    "uc_kkt_noalloc": (C.c_int, [_P(uc_device_lp), C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                 C.c_void_p]),
    "uc_free_lp": (None, [C.c_void_p]),
    "uc_free_presolved": (None, [C.c_void_p]),
    "uc_free_result": (None, [C.c_void_p]),
    "uc_last_error": (C.c_char_p, []),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2607_03627_gb300._build.build() "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


class UCError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib.uc_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} ({code}): {msg}")
        self.code = code


def _check(code: int, where: str):
    if code != UC_OK:
        raise UCError(code, where)


def _ptr(a, ct):
    return a.ctypes.data_as(_P(ct)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class _Handle:
    _free = None

    def __init__(self, ptr: int, keep=None):
        self.ptr = C.c_void_p(ptr)
        self._keep = keep

    def __del__(self):
        if self.ptr and self._free is not None and lib is not None:
            getattr(lib, self._free)(self.ptr)
            self.ptr = C.c_void_p(0)


class LpHandle(_Handle):
    _free = "uc_free_lp"


class PresolvedHandle(_Handle):
    _free = "uc_free_presolved"


class ResultHandle(_Handle):
    _free = "uc_free_result"


def uc_build_lp(P) -> LpHandle:
    """P: any object with the fields of ``uc_problem`` (e.g. ``ucgen.UCProblem``)."""
    arrs = dict(line_from=_i32(P.line_from), line_to=_i32(P.line_to), x_pu=_f64(P.x_pu),
                fmax=_f64(P.fmax), gen_bus=_i32(P.gen_bus), pmax=_f64(P.pmax), pmin=_f64(P.pmin),
                ramp=_f64(P.ramp), c_lin=_f64(P.c_lin), c_nl=_f64(P.c_nl), c_su=_f64(P.c_su),
                u0=_f64(P.u0), load=_f64(P.load).reshape(-1))
    prob = uc_problem(B=P.B, L=P.L, G=P.G, T=P.T, ref_bus=P.ref_bus, voll=float(P.voll))
    for k, a in arrs.items():
        setattr(prob, k, _ptr(a, C.c_int32 if a.dtype == np.int32 else C.c_double))
    out = C.c_void_p()
    _check(lib.uc_build_lp(C.byref(prob), C.byref(out)), "uc_build_lp")
    return LpHandle(out.value)


def uc_lp_dims(lp):
    n, m, me, z = C.c_int(), C.c_int(), C.c_int(), C.c_int64()
    _check(lib.uc_lp_dims(lp.ptr, C.byref(n), C.byref(m), C.byref(me), C.byref(z)), "uc_lp_dims")
    return n.value, m.value, me.value, z.value


def uc_lp_export(lp) -> dict:
    n, m, m_eq, nnz = uc_lp_dims(lp)
    d = dict(rowptr=np.zeros(m + 1, np.int32), colidx=np.zeros(nnz, np.int32), val=np.zeros(nnz),
             q=np.zeros(m), c=np.zeros(n), l=np.zeros(n), u=np.zeros(n))
    _check(lib.uc_lp_export(lp.ptr, _ptr(d["rowptr"], C.c_int32), _ptr(d["colidx"], C.c_int32),
                            _ptr(d["val"], C.c_double), _ptr(d["q"], C.c_double), _ptr(d["c"], C.c_double),
                            _ptr(d["l"], C.c_double), _ptr(d["u"], C.c_double)), "uc_lp_export")
    d.update(n=n, m=m, m_eq=m_eq)
    return d


def default_presolve_opts(**kw) -> uc_presolve_opts:
    o = uc_presolve_opts()
    lib.uc_default_presolve_opts(C.byref(o))
    fields = {f[0] for f in uc_presolve_opts._fields_}
    for k, v in kw.items():
        if k not in fields:
            raise TypeError(f"unknown presolve option {k!r}")
        setattr(o, k, v)
    return o


def uc_presolve(lp, value_bits: int = 64, **kw) -> PresolvedHandle:
    o = default_presolve_opts(value_bits=value_bits, **kw)
    out = C.c_void_p()
    _check(lib.uc_presolve(lp.ptr, C.byref(o), C.byref(out)), "uc_presolve")
    return PresolvedHandle(out.value, keep=lp)


def uc_presolve_reuse(base, lp) -> PresolvedHandle:
    out = C.c_void_p()
    _check(lib.uc_presolve_reuse(base.ptr, lp.ptr, C.byref(out)), "uc_presolve_reuse")
    return PresolvedHandle(out.value, keep=lp)


def uc_presolved_dims(ps):
    n, m, me, z = C.c_int(), C.c_int(), C.c_int(), C.c_int64()
    _check(lib.uc_presolved_dims(ps.ptr, C.byref(n), C.byref(m), C.byref(me), C.byref(z)),
           "uc_presolved_dims")
    return n.value, m.value, me.value, z.value


def uc_presolved_export(ps) -> dict:
    n, m, m_eq, nnz = uc_presolved_dims(ps)
    d = dict(rowptr=np.zeros(m + 1, np.int32), colidx=np.zeros(nnz, np.int32), val=np.zeros(nnz),
             q=np.zeros(m), c=np.zeros(n), l=np.zeros(n), u=np.zeros(n), Dr=np.zeros(m),
             Dc=np.zeros(n), col_map=np.zeros(n, np.int32), row_map=np.zeros(m, np.int32),
             scalars=np.zeros(7))
    _check(lib.uc_presolved_export(
        ps.ptr, _ptr(d["rowptr"], C.c_int32), _ptr(d["colidx"], C.c_int32), _ptr(d["val"], C.c_double),
        _ptr(d["q"], C.c_double), _ptr(d["c"], C.c_double), _ptr(d["l"], C.c_double),
        _ptr(d["u"], C.c_double), _ptr(d["Dr"], C.c_double), _ptr(d["Dc"], C.c_double),
        _ptr(d["col_map"], C.c_int32), _ptr(d["row_map"], C.c_int32), _ptr(d["scalars"], C.c_double)),
        "uc_presolved_export")
    s = d.pop("scalars")
    d.update(n=n, m=m, m_eq=m_eq, eta=s[0], omega0=s[1], norm_A=s[2], obj_const=s[3],
             q_inf=s[4], c_inf=s[5], norm_bound=s[6])
    return d


def uc_presolved_device_order(ps, reorder: bool = True):
    """(prow, pcol): the presolved row / column at each device position."""
    n, m, _, _ = uc_presolved_dims(ps)
    prow = np.zeros(m, np.int32)
    pcol = np.zeros(n, np.int32)
    _check(lib.uc_presolved_device_order(ps.ptr, int(bool(reorder)), _ptr(prow, C.c_int32), _ptr(pcol, C.c_int32)),
           "uc_presolved_device_order")
    return prow, pcol


def uc_presolved_strided_groups(ps, transpose: bool = False) -> dict:
    """Period-strided 16-row groups of the device layout of A (or A^T): counts
    and the descriptors (k per group, slot offsets, slot columns and values)."""
    counts = np.zeros(5, np.int64)
    _check(lib.uc_presolved_strided_groups(ps.ptr, int(bool(transpose)), _ptr(counts, C.c_int64),
                                           None, None, None, None), "uc_presolved_strided_groups")
    ng, slots = int(counts[0]), int(counts[4])
    d = dict(k=np.zeros(ng, np.int32), off=np.zeros(ng + 1, np.int32), col=np.zeros(slots, np.int32),
             val=np.zeros(slots))
    _check(lib.uc_presolved_strided_groups(ps.ptr, int(bool(transpose)), _ptr(counts, C.c_int64),
                                           _ptr(d["k"], C.c_int32), _ptr(d["off"], C.c_int32),
                                           _ptr(d["col"], C.c_int32), _ptr(d["val"], C.c_double)),
           "uc_presolved_strided_groups")
    d.update(groups=ng, strided_groups=int(counts[1]), entries=int(counts[2]),
             strided_entries=int(counts[3]), slots=slots)
    return d


class _TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        try:
            p = self.torch.cuda.caching_allocator_alloc(int(nbytes), stream=self.torch.cuda.current_stream())
        except Exception:
            return None
        self.live[p] = nbytes
        return p

    def _free(self, ptr, nbytes, stream, ctx):
        if ptr in self.live:
            del self.live[ptr]
            self.torch.cuda.caching_allocator_delete(ptr)


_allocator = None


def _torch_stream_and_allocator():
    global _allocator
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("uc_solve needs a CUDA device (there is no CPU fallback)")
    if _allocator is None:
        _allocator = _TorchAllocator()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream), _allocator


def solve_opts(tol: float = 1e-4, max_iter: int = 100_000, n_eval: int = 64, use_graph: bool = True,
               kernel_timing: bool = False, timeout_ms: float = 0.0, warm_x=None, warm_y=None, warm_omega=0.0,
               cancel=None, spmv_kernel: int = 0, algorithm: str = "halpern",
               restart_metric: str = "kkt", cta_rows: int = 0,
               rows_per_thread=None, pdl: bool = True, reorder: bool = True,
               stages: int = 0, lanes: bool = False, adaptive_step: bool = False,
               pw_gains=None, polish: bool = False, polish_max_iter: int = 0,
               tol_abs_feas: float = 1e-5, pw_guard=None) -> tuple[uc_solve_opts, list]:
    o = uc_solve_opts()
    lib.uc_default_solve_opts(C.byref(o))
    keep = []
    o.tol_rel_kkt = tol
    o.max_iter = int(max_iter)
    o.n_eval = int(n_eval)
    o.use_graph = int(bool(use_graph))
    o.kernel_timing = int(bool(kernel_timing))
    o.timeout_ms = float(timeout_ms)
    o.warm_omega = float(warm_omega or 0.0)
    o.spmv_kernel = int(spmv_kernel)
    o.cta_rows = int(cta_rows)
    o.no_pdl = 0 if pdl else 1
    o.no_reorder = 0 if reorder else 1
    o.stages = int(stages)
    o.lanes = int(bool(lanes))
    o.adaptive_step = int(bool(adaptive_step))
    o.polish = int(bool(polish))
    o.polish_max_iter = int(polish_max_iter)
    o.tol_abs_feas = float(tol_abs_feas)
    if pw_gains is not None:   # (kp, ki, kd) of the primal-weight controller
        o.pw_kp, o.pw_ki, o.pw_kd = (float(v) for v in pw_gains)
    if pw_guard is not None:   # residual-balance guard kappa (0: off)
        o.pw_guard = float(pw_guard)
    if rows_per_thread is not None:
        rp = np.ascontiguousarray(rows_per_thread, dtype=np.int32)
        keep.append(rp)
        o.rows_per_thread = _ptr(rp, C.c_int32)
    o.algorithm = {"halpern": 0, "average": 1}[algorithm]
    o.restart_metric = {"kkt": 0, "fpr": 1, "fprp": 2}[restart_metric]
    if warm_x is not None:
        wx = _f64(warm_x); keep.append(wx); o.warm_x = _ptr(wx, C.c_double)
    if warm_y is not None:
        wy = _f64(warm_y); keep.append(wy); o.warm_y = _ptr(wy, C.c_double)
    if cancel is not None:
        o.cancel = C.cast(C.addressof(cancel), _P(C.c_int))
        keep.append(cancel)
    return o, keep


def uc_solve(ps, **kw) -> tuple[ResultHandle, int]:
    """Solve one presolved LP on PyTorch's current device and stream.  Returns
    (result, status); raises UCError for statuses without a result."""
    stream, alloc = _torch_stream_and_allocator()
    o, keep = solve_opts(**kw)
    o.alloc = alloc.alloc
    o.free = alloc.free
    out = C.c_void_p()
    rc = lib.uc_solve(ps.ptr, C.byref(o), stream, C.byref(out))
    if not out.value:
        raise UCError(rc, "uc_solve")
    return ResultHandle(out.value, keep=ps), rc


def uc_solve_batch(ps_list, **kw) -> tuple[list, int]:
    stream, alloc = _torch_stream_and_allocator()
    o, keep = solve_opts(**kw)
    o.alloc = alloc.alloc
    o.free = alloc.free
    k = len(ps_list)
    arr = (C.c_void_p * k)(*[p.ptr.value for p in ps_list])
    outs = (C.c_void_p * k)()
    rc = lib.uc_solve_batch(arr, k, C.byref(o), stream, outs)
    if not all(outs[i] for i in range(k)):
        raise UCError(rc, "uc_solve_batch")
    return [ResultHandle(outs[i], keep=ps_list[i]) for i in range(k)], rc


def uc_get_solution(res, T: int, B: int, L: int, G: int) -> dict:
    d = dict(p=np.zeros((T, G)), u=np.zeros((T, G)), v=np.zeros((T, G)), theta=np.zeros((T, B)),
             f=np.zeros((T, L)), shed=np.zeros((T, B)), lmp=np.zeros((T, B)))
    st = uc_stats()
    _check(lib.uc_get_solution(res.ptr, *[_ptr(d[k], C.c_double) for k in
                                          ("p", "u", "v", "theta", "f", "shed", "lmp")], C.byref(st)),
           "uc_get_solution")
    d["stats"] = st.as_dict()
    return d


def uc_crossover(res, max_pivots: int = 0):
    """A vertex of the presolved LP from a result's returned point (host);
    returns (vertex result, status)."""
    out = C.c_void_p()
    rc = lib.uc_crossover(res.ptr, int(max_pivots), C.byref(out))
    if not out.value:
        raise UCError(rc, "uc_crossover")
    return ResultHandle(out.value, keep=res), rc


def uc_simplex_solve(ps, max_pivots: int = 0, cancel=None):
    """The host simplex from the cold start (CPU arm); returns (result, status).
    ``cancel``: a ctypes.c_int another thread may set to stop it."""
    out = C.c_void_p()
    rc = lib.uc_simplex_solve(ps.ptr, int(max_pivots), None if cancel is None else C.byref(cancel),
                              C.byref(out))
    if not out.value:
        raise UCError(rc, "uc_simplex_solve")
    return ResultHandle(out.value, keep=ps), rc


def uc_solve_concurrent(ps, **kw):
    """Alg. 1: device PDHG and host simplex at once, the first optimal one wins;
    returns (result, status, winner) with winner 0 (device) or 1 (host)."""
    stream, alloc = _torch_stream_and_allocator()
    o, keep = solve_opts(**kw)
    o.alloc = alloc.alloc
    o.free = alloc.free
    out = C.c_void_p()
    win = C.c_int(-1)
    rc = lib.uc_solve_concurrent(ps.ptr, C.byref(o), stream, C.byref(out), C.byref(win))
    if not out.value:
        raise UCError(rc, "uc_solve_concurrent")
    return ResultHandle(out.value, keep=ps), rc, win.value


def uc_result_from_point(ps, x, y):
    """A result holding the scaled presolved point (x, y) (host only)."""
    xa, ya = _f64(x), _f64(y)
    out = C.c_void_p()
    _check(lib.uc_result_from_point(ps.ptr, _ptr(xa, C.c_double), _ptr(ya, C.c_double), C.byref(out)),
           "uc_result_from_point")
    return ResultHandle(out.value, keep=ps)


def uc_get_raw_solution(res, raw_n: int, raw_m: int):
    x = np.zeros(raw_n)
    y = np.zeros(raw_m)
    _check(lib.uc_get_raw_solution(res.ptr, _ptr(x, C.c_double), _ptr(y, C.c_double)),
           "uc_get_raw_solution")
    return x, y


def uc_get_iterate(res, which: int, n: int, m: int):
    x = np.zeros(n)
    y = np.zeros(m)
    _check(lib.uc_get_iterate(res.ptr, int(which), _ptr(x, C.c_double), _ptr(y, C.c_double)),
           "uc_get_iterate")
    return x, y


def uc_get_stats(res) -> dict:
    st = uc_stats()
    _check(lib.uc_get_solution(res.ptr, None, None, None, None, None, None, None, C.byref(st)),
           "uc_get_solution")
    return st.as_dict()


class Session:
    """Device-resident LPs (uc_session_*): upload once, then reset / run /
    harvest / refill.  Device memory from PyTorch's caching allocator; work on
    PyTorch's current stream at creation."""

    def __init__(self, ps_list, **kw):
        stream, alloc = _torch_stream_and_allocator()
        self._opts, self._keep = solve_opts(**kw)
        self._opts.alloc = alloc.alloc
        self._opts.free = alloc.free
        self._alloc = alloc
        self.ps = list(ps_list)
        self.k = len(self.ps)
        arr = (C.c_void_p * self.k)(*[p.ptr.value for p in self.ps])
        out = C.c_void_p()
        _check(lib.uc_session_create(arr, self.k, C.byref(self._opts), stream, C.byref(out)),
               "uc_session_create")
        self.ptr = out

    def reset(self, i: int = -1):
        _check(lib.uc_session_reset(self.ptr, int(i)), "uc_session_reset")

    def run(self, max_replays: int = 0) -> tuple[int, int]:
        nr = C.c_int(0)
        rc = lib.uc_session_run(self.ptr, int(max_replays), C.byref(nr))
        if rc not in (UC_OK, UC_ECANCELLED, UC_ETIMEOUT):
            raise UCError(rc, "uc_session_run")
        return rc, nr.value

    def status(self, i: int) -> int:
        return lib.uc_session_status(self.ptr, int(i))

    def result(self, i: int) -> tuple[ResultHandle, int]:
        out = C.c_void_p()
        rc = lib.uc_session_result(self.ptr, int(i), C.byref(out))
        if not out.value:
            raise UCError(rc, "uc_session_result")
        return ResultHandle(out.value, keep=self.ps[i]), rc

    def set_start(self, i: int, x=None, y=None, omega: float = 0.0):
        xa = _f64(x) if x is not None else None
        ya = _f64(y) if y is not None else None
        _check(lib.uc_session_set_start(self.ptr, int(i), _ptr(xa, C.c_double), _ptr(ya, C.c_double),
                                        float(omega or 0.0)), "uc_session_set_start")

    def update_lp(self, i: int, ps):
        _check(lib.uc_session_update_lp(self.ptr, int(i), ps.ptr), "uc_session_update_lp")
        self.ps[i] = ps

    def device_bytes(self) -> int:
        return int(lib.uc_session_device_bytes(self.ptr))

    def close(self):
        if self.ptr:
            lib.uc_session_free(self.ptr)
            self.ptr = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def uc_kkt_noalloc(dev_lp: uc_device_lp, x_ptr: int, y_ptr: int, omega: float, out_ptr: int,
                   stream: int | None = None) -> int:
    """Relative KKT of a device-resident point with no device allocation
    (see include/uc_pdhg.h); all pointers are device addresses.  Returns the
    status code; the 8 results land in `out_ptr` on `stream`."""
    return lib.uc_kkt_noalloc(C.byref(dev_lp), C.c_void_p(x_ptr), C.c_void_p(y_ptr), float(omega),
                              C.c_void_p(out_ptr), C.c_void_p(stream or 0))
