"""GB300 (sm_103a) solver for the LP relaxation of multi-period DC unit
commitment: host presolve + scaling in C++, restarted PDHG in hand-written
CUDA kernels, behind the C ABI of include/uc_pdhg.h.

The ctypes binding (``binding``) is loaded lazily so that ``_build`` can run
before the library exists; any attribute access that needs the library
fails loudly if it has not been built.
"""
from ._build import build  # noqa: F401

_BINDING_NAMES = {
    "uc_build_lp", "uc_lp_dims", "uc_lp_export", "uc_presolve", "uc_presolved_dims",
    "uc_presolved_export", "uc_solve", "uc_solve_batch", "uc_get_solution", "uc_get_raw_solution",
    "uc_get_iterate", "uc_get_stats", "UCError", "STATUS_NAMES", "UC_OK", "UC_EITERLIMIT",
    "UC_ECANCELLED", "UC_ETIMEOUT", "Session",
}


def __getattr__(name):
    if name in _BINDING_NAMES or name == "binding":
        import importlib
        binding = importlib.import_module(__name__ + ".binding")
        return binding if name == "binding" else getattr(binding, name)
    raise AttributeError(name)
