"""ctypes prototypes of libisg's C ABI (include/isg.h), under the same names.

This module only declares argument and result types; all computation happens
in libisg.so.  Importing it loads the library and raises if it is missing:
there is no fallback implementation.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libisg.so")

ISG_OK = 0
ISG_ERR_INVALID = -1
ISG_ERR_OOM = -2
ISG_ERR_CUDA = -3
ISG_ERR_DEVICE_TIMEOUT = -4
ISG_ERR_BUSY = -5
ISG_ERR_UNSUPPORTED = -6
ISG_NOALLOC_MAX_L = 1 << 18
ISG_SW_MAX_L = 32768
ISG_REQ_QUEUED, ISG_REQ_RUNNING, ISG_REQ_DONE = 0, 1, 2
ISG_REQ_CANCELLED, ISG_REQ_EXPIRED, ISG_REQ_FAILED = 3, 4, 5
ISG_INJECT_ALLOC, ISG_INJECT_LAUNCH, ISG_INJECT_WAIT = 1, 2, 3
ISG_ISING = 0
ISG_BLUME_CAPEL = 1

STATUS_NAMES = {0: "ISG_OK", -1: "ISG_ERR_INVALID", -2: "ISG_ERR_OOM", -3: "ISG_ERR_CUDA",
                -4: "ISG_ERR_DEVICE_TIMEOUT", -5: "ISG_ERR_BUSY", -6: "ISG_ERR_UNSUPPORTED"}


class isg_lattice_desc(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("L", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("delta", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("device_buf", ctypes.c_void_p), ("device_buf_bytes", ctypes.c_size_t),
                ("record_capacity", ctypes.c_int64)]


class isg_obs(ctypes.Structure):
    _fields_ = [("sweep", ctypes.c_int64), ("B", ctypes.c_int64), ("M", ctypes.c_int64),
                ("Q", ctypes.c_int64), ("row_sums", ctypes.POINTER(ctypes.c_int32)),
                ("col_sums", ctypes.POINTER(ctypes.c_int32))]


class isg_ensemble_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("L", ctypes.POINTER(ctypes.c_int64)),
                ("model", ctypes.POINTER(ctypes.c_int32)), ("seed", ctypes.POINTER(ctypes.c_uint64)),
                ("delta", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("record_capacity", ctypes.c_int64)]


class isg_ensemble_tuning(ctypes.Structure):
    _fields_ = [("threads_per_cta", ctypes.c_int32), ("half_teams", ctypes.c_int32),
                ("sweeps_per_launch", ctypes.c_int64), ("multi_words", ctypes.c_int32),
                ("multi_band", ctypes.c_int32), ("ms", ctypes.c_double), ("part", ctypes.c_int32)]


class isg_server_desc(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_active", ctypes.c_int32),
                ("chunk_sweeps", ctypes.c_int64), ("stream", ctypes.c_void_p)]


class isg_request(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("L", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("delta", ctypes.c_double), ("n_sweeps", ctypes.c_int64),
                ("n_pieces", ctypes.c_int64), ("t_start", ctypes.POINTER(ctypes.c_int64)),
                ("beta", ctypes.POINTER(ctypes.c_double)), ("record_every", ctypes.c_int64),
                ("keep_result", ctypes.c_int32), ("arrival_time", ctypes.c_double),
                ("deadline", ctypes.c_double)]


class isg_result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("sweeps_done", ctypes.c_int64),
                ("B", ctypes.c_int64), ("M", ctypes.c_int64), ("Q", ctypes.c_int64),
                ("t_arrival", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("records", ctypes.c_int64),
                ("error", ctypes.c_int32)]


class isg_slab_desc(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("L", ctypes.c_int64), ("y0", ctypes.c_int64),
                ("rows", ctypes.c_int64), ("seed", ctypes.c_uint64), ("delta", ctypes.c_double),
                ("stream", ctypes.c_void_p)]


class isg_schedule(ctypes.Structure):
    _fields_ = [("n_pieces", ctypes.c_int64), ("t_start", ctypes.POINTER(ctypes.c_int64)),
                ("beta", ctypes.POINTER(ctypes.c_double))]


_P = ctypes.c_void_p
_I32, _I64, _U64, _F64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
_I8P = ctypes.POINTER(ctypes.c_int8)
_I32P = ctypes.POINTER(ctypes.c_int32)
_I64P = ctypes.POINTER(ctypes.c_int64)
_U64P = ctypes.POINTER(ctypes.c_uint64)
_F64P = ctypes.POINTER(ctypes.c_double)

# name: (restype, argtypes)
PROTOTYPES = {
    "isg_lattice_bytes": (ctypes.c_size_t, [_I32, _I64]),
    "isg_lattice_create": (_I32, [ctypes.POINTER(isg_lattice_desc), ctypes.POINTER(_P)]),
    "isg_lattice_destroy": (None, [_P]),
    "isg_lattice_init_random": (_I32, [_P]),
    "isg_lattice_init_uniform": (_I32, [_P, ctypes.c_int8]),
    "isg_lattice_set": (_I32, [_P, _I8P, _I64]),
    "isg_lattice_get_rect": (_I32, [_P, _I64, _I64, _I64, _I64, _I8P]),
    "isg_lattice_get": (_I32, [_P, _I8P]),
    "isg_lattice_info": (_I32, [_P, _I64P, _I64P, _I32P, _U64P]),
    "isg_save": (_I32, [_P, ctypes.c_char_p]),
    "isg_load": (_I32, [ctypes.c_char_p, _P, _I64, ctypes.POINTER(_P)]),
    "isg_sweep": (_I32, [_P, _I64, _F64P, _F64, _I64]),
    "isg_sweep_schedule": (_I32, [_P, _I64, ctypes.POINTER(isg_schedule), _I64]),
    "isg_half_sweep": (_I32, [_P, _I32, _F64]),
    "isg_record": (_I32, [_P]),
    "isg_read_records": (_I32, [_P, ctypes.POINTER(isg_obs), _I64, _I64P]),
    "isg_pending_records": (_I32, [_P, _I64P]),
    "isg_measure": (_I32, [_P, ctypes.POINTER(isg_obs)]),
    "isg_measure_planes_noalloc": (_I32, [_I32, _I64, _P, _P, _I64, ctypes.POINTER(isg_obs)]),
    "isg_xi2": (_F64, [_I64, _I64, _I64P, _I32P, _I32P]),
    "isg_correlation": (_I32, [_P, _I64, _I64P, _I64P, _I64P]),
    "isg_xi_integral": (_F64, [_I64, _F64P, _F64P, _F64]),
    "isg_swendsen_wang": (_I32, [_P, _F64]),
    "isg_sw_labels": (_I32, [_P, _I32P]),
    "isg_sw_iterations": (_I32, [_P, _I64P]),
    "isg_energy_density": (_F64, [ctypes.POINTER(isg_obs), _I64, _F64]),
    "isg_last_error": (ctypes.c_char_p, []),
    "isg_ensemble_create": (_I32, [ctypes.POINTER(isg_ensemble_desc), ctypes.POINTER(_P)]),
    "isg_ensemble_destroy": (None, [_P]),
    "isg_ensemble_init_random": (_I32, [_P]),
    "isg_ensemble_sweep": (_I32, [_P, _I64, _F64P, _F64, _I64]),
    "isg_ensemble_read_records": (_I32, [_P, _I64, ctypes.POINTER(isg_obs), _I64P]),
    "isg_ensemble_get": (_I32, [_P, _I64, _I8P]),
    "isg_ensemble_info": (_I32, [_P, _I64P, _I64P, _I64P, _I32P]),
    "isg_ensemble_autotune": (_I32, [_P, _I64, ctypes.POINTER(isg_ensemble_tuning),
                                     ctypes.POINTER(isg_ensemble_tuning), _I64, _I64P]),
    "isg_ensemble_set_tuning": (_I32, [_P, ctypes.POINTER(isg_ensemble_tuning)]),
    "isg_ensemble_get_tuning": (_I32, [_P, ctypes.POINTER(isg_ensemble_tuning)]),
    "isg_server_create": (_I32, [ctypes.POINTER(isg_server_desc), ctypes.POINTER(_P)]),
    "isg_server_destroy": (None, [_P]),
    "isg_server_submit": (_I32, [_P, ctypes.POINTER(isg_request), _U64P]),
    "isg_server_step": (_I32, [_P, _I32P, _I32P]),
    "isg_server_cancel": (_I32, [_P, _U64]),
    "isg_debug_inject": (_I32, [_I32, _I64]),
    "isg_server_drain": (_I32, [_P]),
    "isg_server_poll": (_I32, [_P, _U64, ctypes.POINTER(isg_result)]),
    "isg_server_read_records": (_I32, [_P, _U64, ctypes.POINTER(isg_obs), _I64, _I64P]),
    "isg_server_get_lattice": (_I32, [_P, _U64, _I8P]),
    "isg_server_release": (_I32, [_P, _U64]),
    "isg_server_clock": (_F64, [_P]),
    "isg_server_stats": (_I32, [_P, _F64P, ctypes.POINTER(ctypes.c_size_t),
                                ctypes.POINTER(ctypes.c_size_t)]),
    "isg_slab_edge_bytes": (ctypes.c_size_t, [_I32, _I64]),
    "isg_slab_create": (_I32, [ctypes.POINTER(isg_slab_desc), ctypes.POINTER(_P)]),
    "isg_slab_destroy": (None, [_P]),
    "isg_slab_init_random": (_I32, [_P]),
    "isg_slab_set": (_I32, [_P, _I8P, _I64]),
    "isg_slab_get": (_I32, [_P, _I8P]),
    "isg_slab_edges": (_I32, [_P, _I32, _P, _P]),
    "isg_slab_set_halos": (_I32, [_P, _I32, _P, _P]),
    "isg_slab_half_sweep": (_I32, [_P, _I32, _F64]),
    "isg_slab_measure": (_I32, [_P, ctypes.POINTER(isg_obs)]),
    "isg_slab_info": (_I32, [_P, _I64P, _I64P, _I64P, _I64P, _I32P]),
}

_lib = None


def lib():
    """The loaded libisg with prototypes set; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                "libisg.so is not built (run __graft_entry__.build() or "
                "python -m paper_2503_14688_b300.build); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class IsgError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status):
    if status != ISG_OK:
        msg = lib().isg_last_error()
        raise IsgError(status, msg.decode() if msg else "")
    return status
