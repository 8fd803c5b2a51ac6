"""ctypes declarations of the C ABI in include/mgdg.h and include/mgdg_server.h
(argument marshalling only)."""
import ctypes
import glob
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmgdg.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

MG_OK, MG_EINVAL, MG_ENOMEM, MG_ECUDA, MG_ENOCONV, MG_ENOTREADY = range(6)
STATUS_NAMES = {0: "MG_OK", 1: "MG_EINVAL", 2: "MG_ENOMEM", 3: "MG_ECUDA", 4: "MG_ENOCONV", 5: "MG_ENOTREADY"}


class MgOpts(ctypes.Structure):
    _fields_ = [
        ("overlap_mode", ctypes.c_int),
        ("overlap_frac", ctypes.c_double),
        ("weight_profile", ctypes.c_int),
        ("ns_pre", ctypes.c_int),
        ("ns_post", ctypes.c_int),
        ("ns_growth", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("fdm_tensor_cores", ctypes.c_int),
        ("outer_df64", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("weight_delta", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("fdm_operands", ctypes.c_int),
        ("persistent", ctypes.c_int),
    ]


FILL_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double),
                           ctypes.c_size_t)


class MgRequest(ctypes.Structure):
    _fields_ = [
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("P", ctypes.c_int),
        ("overlap", ctypes.c_int),
        ("penalty", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("f", ctypes.c_void_p),
        ("fill", FILL_FN),
        ("user", ctypes.c_void_p),
        ("u", ctypes.c_void_p),
        ("footprint", ctypes.c_size_t),
    ]


EXECUTE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong, ctypes.POINTER(MgRequest),
                              ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double))


class MgServerOpts(ctypes.Structure):
    _fields_ = [
        ("slots", ctypes.c_int),
        ("budget", ctypes.c_size_t),
        ("policy", ctypes.c_int),
        ("max_wait", ctypes.c_double),
        ("device", ctypes.c_int),
        ("use_cg", ctypes.c_int),
        ("maxit", ctypes.c_int),
        ("opts", MgOpts),
        ("execute", EXECUTE_FN),
        ("execute_user", ctypes.c_void_p),
        ("batch_max", ctypes.c_int),
        ("batch_dofs", ctypes.c_size_t),
    ]


class MgResult(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("iterations", ctypes.c_int),
        ("relres", ctypes.c_double),
        ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
        ("concurrency", ctypes.c_int),
        ("batch", ctypes.c_int),
        ("slot", ctypes.c_int),
        ("footprint", ctypes.c_size_t),
        ("error", ctypes.c_char * 160),
    ]


class MgServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
        ("queued", ctypes.c_int), ("running", ctypes.c_int), ("max_running", ctypes.c_int),
        ("budget", ctypes.c_size_t), ("used", ctypes.c_size_t), ("peak_used", ctypes.c_size_t),
    ]


MG_SCHED_FCFS, MG_SCHED_SMALLEST = 0, 1

_c = ctypes
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_LL = ctypes.c_longlong
_S = ctypes.c_int  # mg_status

SIGNATURES = {
    "mg_default_opts": (None, [ctypes.POINTER(MgOpts)]),
    "mg_setup": (_S, [_D, _D, _D, _I, _I, _I, _I, _D, _I, ctypes.POINTER(MgOpts), ctypes.POINTER(_P)]),
    "mg_workspace_size": (_S, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "mg_bind_workspace": (_S, [_P, _P, ctypes.c_size_t]),
    "mg_num_levels": (_I, [_P]),
    "mg_num_dofs": (_LL, [_P, _I]),
    "mg_level_layers": (_I, [_P, _I]),
    "mg_level_layers_dir": (_I, [_P, _I, _I]),
    "mg_level_fdm_tensor_cores": (_I, [_P, _I]),
    "mg_level_kernel_variant": (_I, [_P, _I, _I]),
    "mg_apply_sipg_df64": (_S, [_P, _I, _P, _P]),
    "mg_vcycle_df64": (_S, [_P, _P, _P]),
    "mg_smooth_df64": (_S, [_P, _I, _P, _P, _I]),
    "mg_selftest_bounded_wait": (_S, [_P, _I, ctypes.POINTER(ctypes.c_int)]),
    "mg_node_coords": (_S, [_P, _I, _P, _P, _P]),
    "mg_rhs": (_S, [_P, _P, _P]),
    "mg_apply_sipg": (_S, [_P, _I, _P, _P]),
    "mg_residual": (_S, [_P, _I, _P, _P, _P]),
    "mg_smooth": (_S, [_P, _I, _P, _P, _I]),
    "mg_restrict_residual": (_S, [_P, _I, _P, _P, _P]),
    "mg_prolongate": (_S, [_P, _I, _P, _P]),
    "mg_coarse_solve": (_S, [_P, _P, _P]),
    "mg_vcycle": (_S, [_P, _P, _P]),
    "mg_solve": (_S, [_P, _P, _P, _D, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "mg_solve_batch": (_S, [_P, _I, _P, _P, _D, _I, _P, _P, _P]),
    "mg_solve_host": (_S, [_P, _P, _P, _D, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "mg_apply_sipg_f32": (_S, [_P, _I, _P, _P]),
    "mg_smooth_f32": (_S, [_P, _I, _P, _P, _I]),
    "mg_vcycle_f32": (_S, [_P, _P, _P]),
    "mg_get_table": (_S, [_P, _I, _I, _I, _P, _I, ctypes.POINTER(_I)]),
    "mg_setup_graded": (_S, [_P, _P, _P, _I, _I, _I, _I, _D, _I, ctypes.POINTER(MgOpts), ctypes.POINTER(_P)]),
    "mg_is_graded": (_I, [_P]),
    "mg_get_line_table": (_S, [_P, _I, _I, _I, _I, _P, _I, ctypes.POINTER(_I)]),
    "mg_coarse_solve_noalloc": (_S, [_D, _D, _D, _I, _I, _I, _D, _P, _P, _P]),
    "mg_kernel_launches": (_LL, [_P]),
    "mg_batch_launches": (_LL, [_P]),
    "mg_profile": (_S, [_P, _I]),
    "mg_profile_result": (_S, [_P, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_LL)]),
    "mg_server_default_opts": (None, [ctypes.POINTER(MgServerOpts)]),
    "mg_server_create": (_S, [ctypes.POINTER(MgServerOpts), ctypes.POINTER(_P)]),
    "mg_request_footprint": (_S, [ctypes.POINTER(MgRequest), ctypes.POINTER(MgOpts), ctypes.POINTER(ctypes.c_size_t)]),
    "mg_submit": (_S, [_P, ctypes.POINTER(MgRequest), ctypes.POINTER(_LL)]),
    "mg_poll": (_S, [_P, _LL, ctypes.POINTER(MgResult)]),
    "mg_wait": (_S, [_P, _LL, _D, ctypes.POINTER(MgResult)]),
    "mg_server_get_stats": (_S, [_P, ctypes.POINTER(MgServerStats)]),
    "mg_server_destroy": (None, [_P]),
    "mg_sched_pick": (_I, [_I, _D, _D, ctypes.c_size_t, ctypes.c_size_t, _I, _P, _P, _P]),
    "mg_last_error": (ctypes.c_char_p, [_P]),
    "mg_destroy": (None, [_P]),
}

_lib = None


def header_symbols(include=INCLUDE):
    """Names of the functions declared in the headers under include/."""
    names = set()
    for path in sorted(glob.glob(os.path.join(include, "*.h"))):
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"\(\s*\*\s*\w+\s*\)\s*\(", "(", text)  # function-pointer members
        names.update(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def load_library(path=LIB_PATH):
    """Load libmgdg.so (built by libbuild.py) and declare every entry point.
    Raises if the library is missing: there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libmgdg.so not found at %s; run paper_1612_04796_gb300.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
