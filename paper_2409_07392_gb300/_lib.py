"""ctypes declarations of the C-ABI in include/firal.h and the loader of the in-tree library.

The library must have been built (``python -m paper_2409_07392_gb300.build`` or
``__graft_entry__.build()``); there is no fallback implementation.
"""
import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_size_t, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfiral.so")

FIRAL_FP64, FIRAL_FP32, FIRAL_MIXED_BF16, FIRAL_MIXED_BF16_FAST = 0, 1, 2, 3
FIRAL_DT_F64, FIRAL_DT_F32, FIRAL_DT_BF16 = 0, 1, 2
STATUS = {0: "FIRAL_OK", -1: "FIRAL_ERR_ARG", -2: "FIRAL_ERR_CUDA", -3: "FIRAL_ERR_NOT_SPD",
          -4: "FIRAL_ERR_CG_NOT_CONVERGED", -5: "FIRAL_ERR_NONFINITE", -6: "FIRAL_ERR_TIMEOUT",
          -7: "FIRAL_ERR_NOMEM", -8: "FIRAL_ERR_UNSUPPORTED", -9: "FIRAL_ERR_COMM"}
(FIRAL_OK, FIRAL_ERR_ARG, FIRAL_ERR_CUDA, FIRAL_ERR_NOT_SPD, FIRAL_ERR_CG_NOT_CONVERGED,
 FIRAL_ERR_NONFINITE, FIRAL_ERR_TIMEOUT, FIRAL_ERR_NOMEM, FIRAL_ERR_UNSUPPORTED,
 FIRAL_ERR_COMM) = range(0, -10, -1)
FIRAL_REDUCE_SUM, FIRAL_REDUCE_MAX = 0, 1

# int32 allreduce(void* buf, int64 count, int32 dtype, int32 op, void* stream, void* user)
ALLREDUCE_FN = ctypes.CFUNCTYPE(c_int32, c_void_p, c_int64, c_int32, c_int32, c_void_p, c_void_p)


class FiralPool(ctypes.Structure):
    _fields_ = [("X", c_void_p), ("h", c_void_p), ("n", c_int64), ("d", c_int32),
                ("c", c_int32), ("x_dtype", c_int32), ("h_dtype", c_int32)]


class FiralHess0(ctypes.Structure):
    _fields_ = [("Xo", c_void_p), ("ho", c_void_p), ("m", c_int64), ("lam", c_double)]


class FiralCGOpts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("maxit", c_int32), ("fixed_iters", c_int32),
                ("block", c_int32), ("reserved", c_int32)]


class FiralRelaxOpts(ctypes.Structure):
    _fields_ = [("s", c_int32), ("T", c_int32), ("cg", FiralCGOpts), ("beta0", c_double),
                ("seed", c_uint64), ("precision", c_int32), ("estimator", c_int32),
                ("md_tol", c_double)]


class FiralAlOpts(ctypes.Structure):
    _fields_ = [("rounds", c_int32), ("budget", c_int32), ("lam", c_double),
                ("lr_gamma", c_double), ("lr_max_newton", c_int32), ("reserved", c_int32),
                ("lr_tol", c_double), ("relax", FiralRelaxOpts), ("eta", c_double)]


class FiralTuning(ctypes.Structure):
    _fields_ = [("dterm_splits", c_int32), ("bsum_splits", c_int32), ("sm_budget", c_int32),
                ("reserved", c_int32)]


class FiralStepStats(ctypes.Structure):
    _fields_ = [("fhat", c_double), ("gmax", c_double), ("zmax", c_double),
                ("cg_iters", c_int32 * 2), ("cg_relres", c_double * 2)]


class FiralRelaxStats(ctypes.Structure):
    _fields_ = [("iters_done", c_int32), ("fhat_last", c_double), ("cg_iters_total", c_int32)]


class FiralComm(ctypes.Structure):
    _fields_ = [("rank", c_int32), ("world", c_int32), ("allreduce", ALLREDUCE_FN),
                ("user", c_void_p)]


class FiralRoundOpts(ctypes.Structure):
    _fields_ = [("eta", c_double), ("exclude_selected", c_int32), ("precision", c_int32)]


class FiralRoundStats(ctypes.Structure):
    _fields_ = [("nu_last", c_double), ("score_last", c_double)]


# (name, restype, argtypes) of every exported symbol
SIGNATURES = [
    ("firal_status_string", c_char_p, [c_int32]),
    ("firal_build_info", c_int32, []),
    ("firal_launch_count", c_int64, []),
    ("firal_profile", c_int32, [c_int32]),
    ("firal_profile_read", c_int32, [POINTER(c_double), POINTER(c_int64), c_int32]),
    ("firal_profile_name", c_char_p, [c_int32]),
    ("firal_create", c_int32, [POINTER(c_void_p), c_void_p]),
    ("firal_destroy", c_int32, [c_void_p]),
    ("firal_set_stream", c_int32, [c_void_p, c_void_p]),
    ("firal_last_error", c_int32, [c_void_p, c_char_p, c_size_t]),
    ("firal_problem_create", c_int32, [c_void_p, POINTER(FiralPool), POINTER(FiralHess0), c_int32,
                                       POINTER(c_void_p)]),
    ("firal_problem_destroy", c_int32, [c_void_p]),
    ("firal_relax", c_int32, [c_void_p, POINTER(FiralPool), POINTER(FiralHess0), c_double,
                              c_void_p, POINTER(FiralRelaxOpts), c_void_p, POINTER(c_double),
                              POINTER(FiralRelaxStats)]),
    ("firal_relax_step", c_int32, [c_void_p, POINTER(FiralRelaxOpts), c_int32, c_double, c_void_p,
                                   POINTER(FiralStepStats)]),
    ("firal_batched_relax", c_int32, [c_void_p, c_int32, POINTER(FiralPool), POINTER(FiralHess0),
                                      POINTER(c_double), POINTER(FiralRelaxOpts),
                                      POINTER(c_void_p)]),
    ("firal_round", c_int32, [c_void_p, POINTER(FiralPool), POINTER(FiralHess0), c_void_p,
                              c_int32, POINTER(FiralRoundOpts), c_void_p,
                              POINTER(FiralRoundStats)]),
    ("firal_round_problem", c_int32, [c_void_p, c_void_p, c_int32, POINTER(FiralRoundOpts),
                                      c_void_p, POINTER(FiralRoundStats)]),
    ("firal_round_sweep", c_int32, [c_void_p, c_void_p, c_int32, POINTER(c_double), c_int32,
                                    POINTER(FiralRoundOpts), c_void_p, POINTER(c_double),
                                    POINTER(c_int32)]),
    ("firal_probes", c_int32, [c_void_p, c_uint64, c_int32, c_int32, c_void_p]),
    ("firal_hessian_apply", c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_void_p]),
    ("firal_precond_blocks", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("firal_pcg", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, POINTER(FiralCGOpts),
                            c_void_p, POINTER(c_int32), POINTER(c_double)]),
    ("firal_quad_forms", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_double, c_void_p]),
    ("firal_md_step", c_int32, [c_void_p, c_void_p, c_void_p, c_double, c_double]),
    ("firal_md_step_static", c_int32, [c_void_p, c_void_p, c_int64, c_int32, c_double, c_double,
                                       c_void_p]),
    ("firal_objective_fwd", c_int32, [c_void_p, c_void_p, c_uint64, c_int32, c_int32,
                                      POINTER(FiralCGOpts), POINTER(c_double), c_void_p,
                                      c_void_p]),
    ("firal_objective_bwd", c_int32, [c_void_p, c_void_p, c_uint64, c_int32, c_int32,
                                      POINTER(FiralCGOpts), c_void_p, c_void_p, c_double,
                                      c_void_p]),
    ("firal_block_eigvals", c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p,
                                      c_void_p]),
    ("firal_nu_bisect", c_int32, [c_void_p, c_void_p, c_int64, POINTER(c_double)]),
    ("firal_exact_objective", c_int32, [c_void_p, c_void_p, POINTER(c_double), c_void_p]),
    ("firal_exact_relax", c_int32, [c_void_p, c_double, c_int32, c_double, c_void_p, c_void_p,
                                    POINTER(c_double)]),
    ("firal_exact_round", c_int32, [c_void_p, c_void_p, c_int32, c_double, c_int32, c_void_p,
                                    POINTER(c_double), POINTER(c_double)]),
    ("firal_cache_trim", c_int32, []),
    ("firal_cache_bytes", c_int64, []),
    ("firal_problem_set_tuning", c_int32, [c_void_p, POINTER(FiralTuning)]),
    ("firal_problem_get_tuning", c_int32, [c_void_p, POINTER(FiralTuning)]),
    ("firal_set_default_tuning", c_int32, [c_void_p, POINTER(FiralTuning)]),
    ("firal_problem_set_comm", c_int32, [c_void_p, POINTER(FiralComm)]),
    ("firal_lr_probs", c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_int64, c_int32,
                                 c_int32, c_int32, c_void_p]),
    ("firal_lr_fit", c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_int64, c_int32, c_int32,
                               c_double, c_int32, c_int32, c_double, c_void_p,
                               POINTER(c_int32), POINTER(c_double)]),
    ("firal_active_learning", c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p,
                                        c_void_p, c_int64, c_int32, c_int32, c_int32,
                                        POINTER(FiralAlOpts), c_void_p, c_void_p,
                                        POINTER(c_double)]),
]

_lib = None


def load():
    """Load ``_build/libfiral.so`` once; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run paper_2409_07392_gb300.build.build())")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class FiralError(RuntimeError):
    def __init__(self, code, detail):
        super().__init__(f"{STATUS.get(code, code)}: {detail}")
        self.code = code


def check(code, handle=None):
    if code != 0:
        buf = ctypes.create_string_buffer(512)
        load().firal_last_error(handle, buf, 512)
        raise FiralError(code, buf.value.decode(errors="replace"))
