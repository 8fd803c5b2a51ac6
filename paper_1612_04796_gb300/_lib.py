"""ctypes declarations of the C ABI in include/mgdg.h (argument marshalling only)."""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmgdg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mgdg.h")

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
    ]


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
    "mg_apply_sipg_df64": (_S, [_P, _I, _P, _P]),
    "mg_vcycle_df64": (_S, [_P, _P, _P]),
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
    "mg_solve_host": (_S, [_P, _P, _P, _D, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "mg_apply_sipg_f32": (_S, [_P, _I, _P, _P]),
    "mg_smooth_f32": (_S, [_P, _I, _P, _P, _I]),
    "mg_vcycle_f32": (_S, [_P, _P, _P]),
    "mg_get_table": (_S, [_P, _I, _I, _I, _P, _I, ctypes.POINTER(_I)]),
    "mg_coarse_solve_noalloc": (_S, [_D, _D, _D, _I, _I, _I, _D, _P, _P, _P]),
    "mg_kernel_launches": (_LL, [_P]),
    "mg_profile": (_S, [_P, _I]),
    "mg_profile_result": (_S, [_P, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_LL)]),
    "mg_last_error": (ctypes.c_char_p, [_P]),
    "mg_destroy": (None, [_P]),
}

_lib = None


def header_symbols(path=HEADER):
    """Names of the functions declared in include/mgdg.h."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", text)))


def load_library(path=LIB_PATH):
    """Load libmgdg.so (built by build.py) and declare every entry point.
    Raises if the library is missing: there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libmgdg.so not found at %s; run paper_1612_04796_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
