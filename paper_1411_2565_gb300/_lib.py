"""ctypes declarations of the C ABI in include/grace.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# GRACE_DEBUG=1 selects the checked build (device-side index checks, workspace guards)
DEBUG = os.environ.get("GRACE_DEBUG", "0") not in ("", "0")
LIB_PATH = os.path.join(HERE, "libgrace_debug.so" if DEBUG else "libgrace.so")

GRACE_OK = 0
STATUS = {0: "GRACE_OK", -1: "GRACE_EINVAL", -2: "GRACE_EWORKSPACE", -3: "GRACE_ECUDA",
          -4: "GRACE_ETIMEOUT", -5: "GRACE_ESTATE", -6: "GRACE_ENONFINITE",
          -7: "GRACE_EUNSUPPORTED"}
TERM_DEMAG, TERM_EXCH, TERM_ANIS, TERM_ZEEMAN, TERM_ALL = 1, 2, 4, 8, 15
OPT_GRAPH, OPT_GRAPH_STEPS, OPT_TILE_X, OPT_TILE_YZ, OPT_PDL, OPT_INTEGRATOR = 1, 2, 3, 4, 5, 6
OPT_TILE_Z, OPT_SIDE_STREAMS = 7, 8
OPT_PERSISTENT, OPT_BARRIER_TIMEOUT_US, OPT_TEST_SKIP_ARRIVE = 9, 10, 11
OPT_NAMES = {OPT_GRAPH: "graph", OPT_GRAPH_STEPS: "graph_steps", OPT_TILE_X: "tile_x",
             OPT_TILE_YZ: "tile_yz", OPT_PDL: "pdl", OPT_INTEGRATOR: "integrator", OPT_TILE_Z: "tile_z",
             OPT_SIDE_STREAMS: "side_streams", OPT_PERSISTENT: "persistent",
             OPT_BARRIER_TIMEOUT_US: "barrier_timeout_us", OPT_TEST_SKIP_ARRIVE: "test_skip_arrive"}
KERNEL_NAMES = ("yz_fast", "x_fast", "yz", "y", "z", "x", "y_fast", "z_fast")

_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_SZ = C.c_size_t
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)

SIGNATURES = {
    "grace_create": (_I, [C.POINTER(_P), _IP, _DP, _D, _D, _D, _D, _D]),
    "grace_batch_create": (_I, [C.POINTER(_P), _I, _IP, _DP, _DP, _DP, _DP, _DP, _DP]),
    "grace_workspace_size": (_I, [_P, C.POINTER(_SZ)]),
    "grace_ncells": (_I, [_P, C.POINTER(C.c_longlong)]),
    "grace_bind": (_I, [_P, _P, _SZ, _P]),
    "grace_set_m": (_I, [_P, _P]),
    "grace_sync": (_I, [_P]),
    "grace_debug_check": (_I, [_P, C.POINTER(C.c_uint)]),
    "grace_get_m": (_I, [_P, _P]),
    "grace_set_m_host": (_I, [_P, _P]),
    "grace_get_m_host": (_I, [_P, _P]),
    "grace_get_m_host_async": (_I, [_P, _P]),
    "grace_set_hext": (_I, [_P, _DP]),
    "grace_set_film_hext": (_I, [_P, _I, _DP]),
    "grace_set_hext_field": (_I, [_P, _P]),
    "grace_set_ms_field": (_I, [_P, _P]),
    "grace_set_hext_pulse": (_I, [_P, _DP]),
    "grace_set_time": (_I, [_P, _D]),
    "grace_get_time": (_I, [_P, _DP]),
    "grace_heff": (_I, [_P, _P, C.c_uint]),
    "grace_step": (_I, [_P, _I, _D]),
    "grace_energy": (_I, [_P, _DP, _DP]),
    "grace_backward_workspace_size": (_I, [_P, _I, _I, C.POINTER(_SZ)]),
    "grace_backward": (_I, [_P, _P, _I, _D, _I, _P, _SZ, _P, _P, _P]),
    "grace_step_checkpointed": (_I, [_P, _I, _D, _I, _P, _SZ]),
    "grace_backward_checkpointed": (_I, [_P, _P, _I, _D, _I, _P, _SZ, _P, _P, _P]),
    "grace_set_option": (_I, [_P, _I, C.c_longlong]),
    "grace_trace": (_I, [_P, _I]),
    "grace_trace_read": (_I, [_P, _DP, C.POINTER(C.c_longlong)]),
    "grace_energy_noalloc": (_I, [_IP, _DP, _D, _D, _D, _DP, _P, _P, _P, _DP, _DP]),
    "grace_last_error": (C.c_char_p, [_P]),
    "grace_destroy": (_I, [_P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libgrace.so (built in-tree by ``paper_1411_2565_gb300.build``); fails loudly if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1411_2565_gb300.build.build("
                           f"debug={DEBUG}) (there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GraceError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str = ""):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} {msg}".rstrip())


def check(code: int, where: str, ctx=None):
    if code != GRACE_OK:
        msg = ""
        if ctx:
            msg = (load().grace_last_error(ctx) or b"").decode(errors="replace")
        raise GraceError(code, where, msg)


def dvec(values):
    return (C.c_double * len(values))(*values)


def ivec(values):
    return (C.c_int * len(values))(*values)
