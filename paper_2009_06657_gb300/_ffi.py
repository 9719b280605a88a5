"""ctypes binding of liblret (include/lret.h): argument marshalling only.

The shared library is built in-tree by build.py; importing this module without
it raises immediately (there is no fallback path).
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblret.so")

LR_OK = 0
LR_EINVAL = -1
LR_EKRAUS = -2
LR_ECAPACITY = -3
LR_ENOMEM = -4
LR_ETIMEOUT = -5
LR_ECUDA = -6
LR_ESTATE = -7
LR_ENOCONV = -8
LR_C64 = 0
LR_C128 = 1
LR_DEPOLARIZING = 0
LR_AMPLITUDE_DAMPING = 1
LR_BIT_FLIP = 2
LR_STATIC_MAX_TERMS = 256
KCLASSES = ["expand", "gram", "eigh", "project", "readout", "pauli", "small", "refine"]
LR_TRUNC_LOG_FIELDS = 8
LR_EIGP_REFINED = 0
LR_EIGP_FP32 = 1
LR_EIGP_FP64 = 2
LR_NKCLASS = 8


class LRError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: status {status} ({lib.lr_status_string(status).decode()})")


class lr_info(C.Structure):
    _fields_ = [("n", C.c_int), ("columns", C.c_int), ("capacity", C.c_int), ("dtype", C.c_int),
                ("compressions", C.c_int64), ("stages", C.c_int64), ("discarded", C.c_double),
                ("last_gap", C.c_double)]


class lr_op(C.Structure):
    _fields_ = [("kind", C.c_int), ("q0", C.c_int), ("q1", C.c_int), ("theta", C.c_double), ("p", C.c_double)]


class lr_circuit(C.Structure):
    _fields_ = [("n", C.c_int), ("r", C.c_int), ("nops", C.c_int), ("ops", C.POINTER(lr_op))]


class lr_batch_opts(C.Structure):
    _fields_ = [("dtype", C.c_int), ("eig_precision", C.c_int), ("eig_iters", C.c_int),
                ("rows_per_split", C.c_int), ("splits", C.POINTER(C.c_int)), ("use_graph", C.c_int),
                ("stream", C.c_void_p), ("tensor_cores", C.c_int), ("cluster_min_m", C.c_int)]


OP_KIND = {"rx": 0, "ry": 1, "rz": 2, "cnot": 3, "cz": 4, "dep": 5, "ad": 6, "bf": 7}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"liblret.so not found at {LIB_PATH}; build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    return C.CDLL(LIB_PATH)


lib = _load()

_H = C.c_void_p
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_U64 = C.POINTER(C.c_uint64)
_I = C.POINTER(C.c_int)

_SIGS = {
    "lr_init": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, C.POINTER(_H)]),
    "lr_init_ex": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, _P, C.POINTER(_H)]),
    "lr_free": (C.c_int, [_H]),
    "lr_reset": (C.c_int, [_H]),
    "lr_apply_gate": (C.c_int, [_H, C.c_int, _I, _D, _D, C.c_int]),
    "lr_apply_diagonal": (C.c_int, [_H, C.c_int, _I, _D]),
    "lr_apply_gate_device": (C.c_int, [_H, C.c_int, _I, C.c_void_p]),
    "lr_apply_rotation": (C.c_int, [_H, C.c_int, C.c_int, C.c_double, C.c_int]),
    "lr_apply_kraus": (C.c_int, [_H, C.c_int, C.c_int, _D]),
    "lr_kraus_preset": (C.c_int, [C.c_int, C.c_double, _D, _I]),
    "lr_compress": (C.c_int, [_H, C.c_int, _D]),
    "lr_set_eps": (C.c_int, [_H, C.c_double]),
    "lr_set_eigensolver": (C.c_int, [_H, C.c_int]),
    "lr_set_eig_precision": (C.c_int, [_H, C.c_int, C.c_int]),
    "lr_last_eig": (C.c_int, [_H, _I, _I, _D, _D, _D]),
    "lr_set_trunc_log": (C.c_int, [_H, C.c_int]),
    "lr_get_trunc_log": (C.c_int, [_H, _D, C.c_int, C.POINTER(C.c_int64)]),
    "lr_set_path": (C.c_int, [_H, C.c_int]),
    "lr_set_tensor_cores": (C.c_int, [_H, C.c_int]),
    "lr_probs": (C.c_int, [_H, _P]),
    "lr_expect": (C.c_int, [_H, C.c_int, _U64, _U64, _D, _D]),
    "lr_z_expect": (C.c_int, [_H, _D]),
    "lr_set_record": (C.c_int, [_H, C.c_int]),
    "lr_set_checkpoint": (C.c_int, [_H, C.c_int]),
    "lr_backward": (C.c_int, [_H, C.c_int, _U64, _U64, _D, C.c_int, _D]),
    "lr_get_info": (C.c_int, [_H, C.POINTER(lr_info)]),
    "lr_get_state": (C.c_int, [_H, _P]),
    "lr_device_bytes": (C.c_int64, [_H]),
    "lr_last_eig_stats": (C.c_int, [_H, C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    "lr_set_timing": (C.c_int, [_H, C.c_int]),
    "lr_kernel_times": (C.c_int, [_H, _D, C.POINTER(C.c_int64)]),
    "lr_expect_static": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _U64, _U64, _D, _D, _P]),
    "lr_batch_create": (C.c_int, [C.POINTER(lr_circuit), C.c_int, C.c_int, C.c_int, C.c_int, _P, C.POINTER(_H)]),
    "lr_batch_opts_default": (None, [C.POINTER(lr_batch_opts)]),
    "lr_batch_create_ex": (C.c_int, [C.POINTER(lr_circuit), C.c_int, C.POINTER(lr_batch_opts), C.POINTER(_H)]),
    "lr_batch_run": (C.c_int, [_H]),
    "lr_batch_reset": (C.c_int, [_H]),
    "lr_batch_info": (C.c_int, [_H, C.c_int, C.POINTER(lr_info)]),
    "lr_batch_probs": (C.c_int, [_H, C.c_int, _P]),
    "lr_batch_stats": (C.c_int, [_H, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64)]),
    "lr_batch_free": (C.c_int, [_H]),
    "lr_status_string": (C.c_char_p, [C.c_int]),
    "lr_selftest_wait": (C.c_int, [C.c_longlong, C.c_int, _P]),
    "lr_launch_count": (C.c_int64, []),
    "lr_sample": (C.c_int, [_H, C.c_int, _D, C.POINTER(C.c_int64)]),
    "lr_entropy": (C.c_int, [_H, _D]),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def check(status, where):
    if status != LR_OK:
        raise LRError(status, where)
    return status


def exported_symbols():
    return sorted(_SIGS)
