"""ctypes declarations of libqs.so (the C ABI in include/qs.h).

Argument marshalling only: every step of the hot path runs in the library's CUDA
kernels.  Loading fails loudly when the library is missing; there is no CPU path.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqs.so")

# enums (include/qs.h)
QS_C64, QS_C128 = 0, 1
QS_OK, QS_EINVAL, QS_ENOMEM, QS_ECUDA, QS_ETIMEOUT, QS_EBUSY, QS_EUNSUPPORTED, QS_ECANCELED = range(8)
QS_ARITH_AUTO, QS_ARITH_DF, QS_ARITH_F64 = 0, 1, 2
QS_MODE_PERGATE, QS_MODE_PAPER, QS_MODE_TILE = 0, 1, 2
QS_ORDER_LOGICAL, QS_ORDER_STORAGE = 0, 1
QS_DENSE_AUTO, QS_DENSE_CUDA_CORES, QS_DENSE_TENSOR = 0, 1, 2
QS_FLAG_FULL_RX, QS_FLAG_NO_DENSE, QS_FLAG_NO_FUSE = 1, 2, 4
OP_CODES = {"U1": 0, "H": 1, "X": 2, "Y": 3, "Z": 4, "S": 5, "T": 6, "RZ": 7, "RX": 8, "RY": 9, "P": 10,
            "CNOT": 11, "CZ": 12, "CP": 13, "CU": 14, "SWAP": 15, "U2": 16, "UK": 17, "RELABEL": 18}
STATUS_NAMES = {0: "QS_OK", 1: "QS_EINVAL", 2: "QS_ENOMEM", 3: "QS_ECUDA", 4: "QS_ETIMEOUT", 5: "QS_EBUSY",
                6: "QS_EUNSUPPORTED", 7: "QS_ECANCELED"}


class qs_op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nq", ctypes.c_int32), ("q", ctypes.c_int32 * 6),
                ("param", ctypes.c_double), ("mat", ctypes.c_int64)]


class qs_cost_model(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_double * 3), ("gate", ctypes.c_double * 3), ("permute", ctypes.c_double * 3),
                ("dense", ctypes.c_double * 3)]


class qs_compile_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("dtype", ctypes.c_int32), ("arith", ctypes.c_int32),
                ("tile_bits", ctypes.c_int32), ("low_bits", ctypes.c_int32), ("max_ops", ctypes.c_int32),
                ("scoring", ctypes.c_int32), ("flags", ctypes.c_int32), ("reg_bits", ctypes.c_int32),
                ("renorm_every", ctypes.c_int32), ("cost", ctypes.POINTER(qs_cost_model))]


class qs_plan_stats(ctypes.Structure):
    _fields_ = [("n_gates", ctypes.c_int64), ("n_passes", ctypes.c_int64), ("n_pergate", ctypes.c_int64),
                ("n_permutes", ctypes.c_int64), ("n_comm_gates", ctypes.c_int64), ("hbm_bytes", ctypes.c_double),
                ("alu_instr", ctypes.c_double), ("compile_ms", ctypes.c_double), ("n_dense", ctypes.c_int64),
                ("predicted_ms", ctypes.c_double), ("n_permute_kernels", ctypes.c_int64),
                ("n_fused", ctypes.c_int64)]


class qs_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("alu", ctypes.c_double)]


class qs_batch_stats(ctypes.Structure):
    _fields_ = [("n_circuits", ctypes.c_int64), ("n_gates", ctypes.c_int64), ("n_passes", ctypes.c_int64),
                ("n_waves", ctypes.c_int64), ("state_bytes", ctypes.c_double), ("hbm_bytes", ctypes.c_double),
                ("alu_instr", ctypes.c_double), ("compile_ms", ctypes.c_double)]


class qs_server_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("compile_threads", ctypes.c_int32), ("mem_budget", ctypes.c_int64),
                ("readout", ctypes.c_int32), ("batch_small_n", ctypes.c_int32), ("batch_max", ctypes.c_int32),
                ("order", ctypes.c_int32), ("max_wait_ms", ctypes.c_int32), ("tile_bits", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class qs_server_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("n", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("batched", ctypes.c_int32), ("norm", ctypes.c_double), ("t_submit_s", ctypes.c_double),
                ("t_admit_s", ctypes.c_double), ("t_done_s", ctypes.c_double), ("amplitudes", ctypes.c_uint64),
                ("error", ctypes.c_char * 128)]


class qs_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("waiting", ctypes.c_int64), ("batches", ctypes.c_int64), ("batched_requests", ctypes.c_int64),
                ("peak_in_flight", ctypes.c_int64), ("peak_mem_bytes", ctypes.c_double),
                ("mem_used_bytes", ctypes.c_double), ("now_s", ctypes.c_double)]


assert ctypes.sizeof(qs_op) == 48

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_H = ctypes.c_void_p
_I = ctypes.c_int
_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
_I32P = ctypes.POINTER(ctypes.c_int32)

# name -> (restype, argtypes); every symbol declared in include/qs.h
SIGNATURES = {
    "qs_last_error": (ctypes.c_char_p, []),
    "qs_version": (ctypes.c_char_p, []),
    "qs_set_allocator": (_I, [ALLOC_FN, FREE_FN, _P]),
    "qs_create": (_I, [_I, _I, ctypes.POINTER(_H)]),
    "qs_create_async": (_I, [_I, _I, _P, ctypes.POINTER(_H)]),
    "qs_destroy": (_I, [_H]),
    "qs_set_stream": (_I, [_H, _P]),
    "qs_set_arith": (_I, [_H, _I]),
    "qs_set_profiling": (_I, [_H, _I]),
    "qs_get_kernel_stats": (_I, [_H, ctypes.POINTER(qs_kernel_stat), _I, _IP]),
    "qs_reset_kernel_stats": (_I, [_H]),
    "qs_reset": (_I, [_H]),
    "qs_get_info": (_I, [_H, _IP, _IP, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_size_t)]),
    "qs_sync": (_I, [_H]),
    "qs_apply_1q": (_I, [_H, _DP, _I]),
    "qs_apply_2q": (_I, [_H, _DP, _I, _I]),
    "qs_apply_controlled": (_I, [_H, _DP, _I, _I]),
    "qs_apply_dense": (_I, [_H, _DP, _I, _IP]),
    "qs_permute": (_I, [_H, _IP]),
    "qs_get_permutation": (_I, [_H, _IP]),
    "qs_compile": (_I, [_I, ctypes.POINTER(qs_op), ctypes.c_size_t, _DP, ctypes.c_size_t, _IP,
                        ctypes.POINTER(qs_compile_opts), ctypes.POINTER(_H)]),
    "qs_plan_destroy": (_I, [_H]),
    "qs_default_cost_model": (_I, [_I, _I, ctypes.POINTER(qs_cost_model)]),
    "qs_plan_get_stats": (_I, [_H, ctypes.POINTER(qs_plan_stats)]),
    "qs_plan_final_permutation": (_I, [_H, _IP]),
    "qs_plan_get_trace": (_I, [_H, _I32P, _I32P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "qs_execute": (_I, [_H, _H]),
    "qs_run": (_I, [_H, ctypes.POINTER(qs_op), ctypes.c_size_t, _DP, ctypes.c_size_t,
                    ctypes.POINTER(qs_compile_opts)]),
    "qs_probabilities": (_I, [_H, _DP, _I]),
    "qs_get_amplitudes": (_I, [_H, _P, ctypes.c_uint64, ctypes.c_uint64, _I]),
    "qs_set_amplitudes": (_I, [_H, _P]),
    "qs_copy_range_device": (_I, [_H, _P, ctypes.c_uint64, ctypes.c_uint64, _I]),
    "qs_gate_matrix": (_I, [_I, ctypes.POINTER(qs_op), _DP, ctypes.c_size_t, _DP, _IP]),
    "qs_norm": (_I, [_H, _DP]),
    "qs_norm_noalloc": (_I, [_P, _I, _I, _P, _P]),
    "qs_inner": (_I, [_H, _H, _DP]),
    "qs_set_dense_path": (_I, [_H, _I]),
    "qs_selftest_bounded_wait": (_I, [_I, _IP]),
    "qs_renormalize": (_I, [_H, _DP]),
    "qs_batch_create": (_I, [_I, _IP, ctypes.POINTER(qs_op), ctypes.POINTER(ctypes.c_int64), _DP, ctypes.c_size_t,
                             ctypes.POINTER(qs_compile_opts), ctypes.POINTER(_H)]),
    "qs_batch_set_stream": (_I, [_H, _P]),
    "qs_batch_set_graph": (_I, [_H, _I]),
    "qs_batch_run": (_I, [_H]),
    "qs_batch_sync": (_I, [_H]),
    "qs_batch_norms": (_I, [_H, _DP]),
    "qs_batch_get_amplitudes": (_I, [_H, _I, _P, ctypes.c_uint64, ctypes.c_uint64]),
    "qs_batch_get_stats": (_I, [_H, ctypes.POINTER(qs_batch_stats)]),
    "qs_batch_destroy": (_I, [_H]),
    "qs_server_create": (_I, [ctypes.POINTER(qs_server_opts), ctypes.POINTER(_H)]),
    "qs_server_submit": (_I, [_H, _I, _I, ctypes.POINTER(qs_op), ctypes.c_size_t, _DP, ctypes.c_size_t,
                              ctypes.POINTER(ctypes.c_int64)]),
    "qs_server_poll": (_I, [_H, ctypes.POINTER(qs_server_result), _I, _IP, _I]),
    "qs_server_take": (_I, [_H, ctypes.c_int64, _P, ctypes.c_uint64]),
    "qs_server_cancel": (_I, [_H, ctypes.c_int64]),
    "qs_server_get_stats": (_I, [_H, ctypes.POINTER(qs_server_stats)]),
    "qs_server_destroy": (_I, [_H]),
}

_lib = None


def load():
    """Load libqs.so (building it first if the toolkit is present and it is stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        try:
            from . import build as _b
            _b.build()
        except Exception as e:  # noqa: BLE001
            raise ImportError(f"libqs.so is missing and could not be built: {e}") from e
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class QSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status):
    if status != QS_OK:
        raise QSError(status, load().qs_last_error().decode(errors="replace"))
