"""ctypes binding of the C ABI in include/chase_gb300.h (argument marshalling only).

The shared library is built in-tree by ``paper_2205_02491_gb300.build``.  There is
no fallback: if the library is missing or fails to load, importing this module
raises, so nothing silently runs elsewhere.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchase_gb300.so")

CHASE_R64, CHASE_C128 = 0, 1
CHASE_FP64, CHASE_FP64_NATIVE, CHASE_BF16x3, CHASE_BF16x6 = 0, 1, 2, 3
MODES = {"fp64": CHASE_FP64, "fp64_native": CHASE_FP64_NATIVE, "bf16x3": CHASE_BF16x3, "bf16x6": CHASE_BF16x6}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_NOCONV", 4: "ERR_QR_BREAKDOWN", 5: "ERR_NAN",
          6: "ERR_CUDA", 7: "ERR_STATE", 8: "ERR_TIMEOUT", 9: "ERR_UNSUPPORTED"}

# every symbol include/chase_gb300.h declares
EXPORTED = ["chase_default_opts", "chase_create", "chase_destroy", "chase_last_error", "chase_workspace_bytes",
            "chase_solve", "chase_solve_batched", "chase_eigvals", "chase_eigvecs", "chase_stats", "chase_backward",
            "chase_kernel_launch_count", "chase_lanczos", "chase_filter", "chase_qr", "chase_rayleigh_ritz", "chase_heevj", "chase_heevj_noalloc", "chase_hemm",
            "chase_generate", "chase_perturb", "chase_set_wait_limit_ns", "chase_measure_fp64_peak",
            "chase_measure_mma_issue"]


class Opts(C.Structure):
    _fields_ = [("maxdeg", C.c_int), ("lanczos_steps", C.c_int), ("lanczos_runs", C.c_int), ("maxiter", C.c_int),
                ("extra_deg", C.c_int), ("nfinal", C.c_int), ("oz_slices", C.c_int),
                ("native_below_mflop", C.c_int), ("batch_workers", C.c_int), ("batch_grouped", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("locked", C.c_int), ("matvecs", C.c_int64), ("matvecs_lowp", C.c_int64),
                ("lowp_iterations", C.c_int), ("ms_total", C.c_double), ("ms_lanczos", C.c_double),
                ("ms_filter", C.c_double), ("ms_qr", C.c_double), ("ms_rr", C.c_double), ("ms_resid", C.c_double),
                ("b_sup", C.c_double), ("mu_1", C.c_double), ("mu_ne", C.c_double), ("norm_est", C.c_double),
                ("max_resid", C.c_double), ("qr_fallbacks", C.c_int), ("filter_launches", C.c_int),
                ("ms_filter_kernel", C.c_double), ("filter_kernel_launches", C.c_int),
                ("ms_filter_kernel_lowp", C.c_double), ("ms_backward", C.c_double),
                ("minres_iterations", C.c_int), ("rr_clusters", C.c_int), ("rr_fallbacks", C.c_int),
                ("qr_householder", C.c_int), ("filter_reorth", C.c_int),
                ("rr_sweeps", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ChaseError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; g.build()'` "
                          "(or python paper_2205_02491_gb300/build.py) first")
    lib = C.CDLL(LIB_PATH)
    P, I64, I, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "chase_default_opts": (None, [C.POINTER(Opts)]),
        "chase_create": (I, [C.POINTER(P), I64, I, I, C.POINTER(Opts), P]),
        "chase_destroy": (None, [P]),
        "chase_last_error": (C.c_char_p, [P]),
        "chase_workspace_bytes": (I64, [I64, I, I, C.POINTER(Opts)]),
        "chase_kernel_launch_count": (I64, []),
        "chase_solve": (I, [P, P, I64, I64, I, I, D, I, I, P, P]),
        "chase_solve_batched": (I, [P, I, P, P, P, P, D, I, I, P, P, P, P]),
        "chase_eigvals": (I, [P, P, I]),
        "chase_eigvecs": (I, [P, P, I64, I]),
        "chase_stats": (I, [P, C.POINTER(Stats)]),
        "chase_backward": (I, [P, P, I64, P, P, I64, P, I64, D, I]),
        "chase_lanczos": (I, [P, P, I64, I64, I, P, I, I, P]),
        "chase_filter": (I, [P, P, I64, I64, P, I64, I, P, D, D, D, I]),
        "chase_qr": (I, [P, P, I64, I64, I, I]),
        "chase_rayleigh_ritz": (I, [P, P, I64, I64, P, I64, I, P, P]),
        "chase_heevj": (I, [P, P, I64, I, P, P, I64]),
        "chase_heevj_noalloc": (I, [P, I64, I, I, P, P, I64, P]),
        "chase_hemm": (I, [P, P, I64, I64, P, I64, I, P, I64, I]),
        "chase_generate": (I, [P, P, I64, I64, P, P, P, P, I]),
        "chase_perturb": (I, [P, P, I64, I64, D, C.c_uint64]),
        "chase_set_wait_limit_ns": (None, [C.c_uint64]),
        "chase_measure_fp64_peak": (I, [I, C.POINTER(D), C.POINTER(D)]),
        "chase_measure_mma_issue": (I, [I, I, C.POINTER(D)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(ctx, status: int):
    if status != 0:
        lib = load()
        msg = lib.chase_last_error(ctx)
        raise ChaseError(status, msg.decode() if msg else "")
