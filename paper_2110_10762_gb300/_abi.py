"""ctypes view of libparareal.so (include/parareal.h): structs and prototypes.

Loading fails loudly (ImportError) when the library has not been built;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libparareal.so")

PR_OK, PR_EINVAL, PR_ENOMEM, PR_ECUDA, PR_ETIMEOUT, PR_ENOTCONV, PR_ESTATE, PR_ELOGFULL = range(8)
STATUS_NAMES = {0: "PR_OK", 1: "PR_EINVAL", 2: "PR_ENOMEM", 3: "PR_ECUDA", 4: "PR_ETIMEOUT",
                5: "PR_ENOTCONV", 6: "PR_ESTATE", 7: "PR_ELOGFULL"}
PR_EXPLICIT_EULER, PR_IMPLICIT_EULER, PR_CRANK_NICOLSON = 0, 1, 2
PR_SOLVER_THOMAS, PR_SOLVER_CG = 0, 1
PR_OPT_PIPELINE, PR_OPT_PIPELINE_CHUNKS, PR_OPT_CG_BLOCKS_PER_SM, PR_OPT_G_CHEBYSHEV = 1, 2, 3, 4
PR_OPT_G_CG = 5
PR_OPT_F_STEPS_PER_PASS = 6


class pr_problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("T0", C.c_double), ("T", C.c_double),
                ("N", C.c_int), ("u0_dev", C.c_void_p), ("kappa_dev", C.c_void_p),
                ("f_scheme", C.c_int), ("f_steps", C.c_int), ("f_prec", C.c_int),
                ("g_solver", C.c_int), ("g_steps", C.c_int), ("g_rtol", C.c_double),
                ("g_maxit", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int),
                ("f_rtol", C.c_double), ("f_maxit", C.c_int)]


class pr_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("max_delta", C.c_double),
                ("fine_lups", C.c_longlong), ("cg_iterations", C.c_longlong),
                ("coarse_solves", C.c_longlong), ("t_total_ms", C.c_double),
                ("t_fine_ms", C.c_double), ("t_coarse_ms", C.c_double), ("events", C.c_longlong),
                ("launches", C.c_longlong), ("fine_cg_iterations", C.c_longlong),
                ("verify_rounds", C.c_int), ("residual", C.c_double),
                ("predictor_cg_iterations", C.c_longlong), ("t_predictor_ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pr_async_opts(C.Structure):
    _fields_ = [("paper_literal", C.c_int), ("timeout_s", C.c_double),
                ("delays_dev", C.c_void_p), ("delay_cols", C.c_int),
                ("delay_unit_ns", C.c_double), ("ctas_per_slice", C.c_int),
                ("quiescence", C.c_int), ("lazy", C.c_int), ("verify", C.c_int)]


class pr_event(C.Structure):
    _fields_ = [("slice", C.c_int32), ("version", C.c_int32), ("vF", C.c_int32),
                ("vG", C.c_int32), ("cg_iters", C.c_int32), ("team", C.c_int32),
                ("delta", C.c_double), ("t_start", C.c_uint64), ("t_end", C.c_uint64)]


EXPORTS = {
    # name: (restype, argtypes)
    "parareal_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "parareal_set_problem": (C.c_int, [C.c_void_p, C.POINTER(pr_problem)]),
    "parareal_run_sync": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(pr_stats)]),
    "parareal_run_sync_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(pr_stats)]),
    "parareal_run_async": (C.c_int, [C.c_void_p, C.POINTER(pr_async_opts), C.c_void_p,
                                     C.POINTER(pr_stats), C.POINTER(pr_event), C.c_size_t,
                                     C.POINTER(C.c_size_t)]),
    "parareal_serial_fine": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(pr_stats)]),
    "parareal_fine": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "parareal_coarse": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.POINTER(C.c_int)]),
    "parareal_correct": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.POINTER(C.c_double)]),
    "parareal_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "parareal_adjoint_async": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]),
    "parareal_slice_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "parareal_set_option": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "parareal_coarse_noalloc": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.c_double, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                          C.POINTER(C.c_int), C.c_void_p]),
    "parareal_probe_fp64": (C.c_int, [C.c_int, C.c_longlong, C.c_void_p, C.POINTER(C.c_double),
                                      C.POINTER(C.c_longlong), C.c_void_p]),
    "parareal_probe_convert": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_longlong, C.c_void_p]),
    "parareal_destroy": (None, [C.c_void_p]),
    "parareal_last_error": (C.c_char_p, [C.c_void_p]),
    "parareal_version": (C.c_char_p, []),
}


def header_declared_names(header_path: str) -> list[str]:
    """Names of the functions include/parareal.h declares (parsed from text)."""
    import re
    src = open(header_path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(parareal_\w+)\s*\(", src)))


_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library and attach prototypes (cached)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libparareal.so not built at {path}; run paper_2110_10762_gb300.build")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
