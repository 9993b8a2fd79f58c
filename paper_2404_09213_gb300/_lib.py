"""ctypes declarations of the C ABI in ``include/qsim.h`` and the loader of ``libqsim.so``.

The library is built in-tree (``python -m paper_2404_09213_gb300.build``); importing this module
without it raises immediately — there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqsim.so")

QSIM_RX, QSIM_RY, QSIM_RZ, QSIM_H, QSIM_X, QSIM_CNOT, QSIM_CZ = range(7)
QSIM_C64, QSIM_C128 = 0, 1
QSIM_FUSED, QSIM_PER_GATE = 0, 1
ERRORS = {0: "QSIM_OK", -1: "QSIM_ERR_ARG", -2: "QSIM_ERR_QUBIT", -3: "QSIM_ERR_PARAM", -4: "QSIM_ERR_GATE",
          -5: "QSIM_ERR_NO_FORWARD", -6: "QSIM_ERR_OOM", -7: "QSIM_ERR_CUDA", -8: "QSIM_ERR_TIMEOUT",
          -9: "QSIM_ERR_UNSUPPORTED"}


class QsimGate(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("targets", ctypes.c_int32 * 2), ("controls", ctypes.c_int32 * 2),
                ("param", ctypes.c_int32)]


class QsimPlanOpts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("dtype", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("contiguous_bits", ctypes.c_int32), ("checkpoint_passes", ctypes.c_int32),
                ("sample_block", ctypes.c_int32), ("bwd_reg_bits", ctypes.c_int32),
                ("fwd_reg_bits", ctypes.c_int32), ("weight_remap", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("max_regs", ctypes.c_int32), ("rotate_low_bits", ctypes.c_int32),
                ("pauli_frame", ctypes.c_int32), ("scalar_bwd", ctypes.c_int32),
                ("product_prefix", ctypes.c_int32), ("split_diagonal", ctypes.c_int32),
                ("large_circuit_qubits", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_int64)]


class QsimPlanInfo(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_gates", ctypes.c_int32), ("n_params", ctypes.c_int32),
                ("n_inputs", ctypes.c_int32), ("n_passes", ctypes.c_int32), ("k", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("mode", ctypes.c_int32), ("n_checkpoints", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64)]


class QsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None

# name -> (restype, argtypes)
SIGNATURES = {
    "qsim_default_opts": (None, [ctypes.POINTER(QsimPlanOpts)]),
    "qsim_plan": (ctypes.c_int, [ctypes.POINTER(QsimGate), ctypes.c_int32, ctypes.c_int32,
                                 ctypes.POINTER(QsimPlanOpts), ctypes.POINTER(ctypes.c_void_p)]),
    "qsim_plan_info_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(QsimPlanInfo)]),
    "qsim_plan_describe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t,
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "qsim_plan_kernel_source": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t,
                                               ctypes.POINTER(ctypes.c_size_t)]),
    "qsim_plan_compile_kernels": (ctypes.c_int, [ctypes.c_void_p]),
    "qsim_tile_index_map": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_int64)]),
    "qsim_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "qsim_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "qsim_sync_status": (ctypes.c_int, [ctypes.c_void_p]),
    "qsim_expval_z": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "qsim_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "qsim_read_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                         ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "qsim_kernel_launches": (ctypes.c_int64, []),
    "qsim_expval_z_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_void_p, ctypes.c_void_p]),
    "qsim_multi_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.POINTER(QsimGate)), ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.POINTER(QsimPlanOpts),
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_void_p)]),
    "qsim_parse_qasm": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(QsimGate), ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "qsim_export_qasm": (ctypes.c_int, [ctypes.POINTER(QsimGate), ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "qsim_landscape": (ctypes.c_int, [ctypes.POINTER(QsimGate), ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(QsimPlanOpts), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "qsim_autotune": (ctypes.c_int, [ctypes.POINTER(QsimGate), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(QsimPlanOpts),
                                     ctypes.POINTER(ctypes.c_float), ctypes.c_void_p]),
    "qsim_multi_autotune": (ctypes.c_int, [ctypes.POINTER(ctypes.POINTER(QsimGate)), ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(QsimPlanOpts),
                                           ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "qsim_multi_offsets": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32] + [ctypes.POINTER(ctypes.c_int64)] * 4),
    "qsim_multi_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "qsim_multi_backward": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "qsim_multi_sync_status": (ctypes.c_int, [ctypes.c_void_p]),
    "qsim_multi_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32)]),
    "qsim_multi_kernel_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
    "qsim_multi_set_test_hooks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]),
    "qsim_multi_destroy": (None, [ctypes.c_void_p]),
    "qsim_plan_destroy": (None, [ctypes.c_void_p]),
    "qsim_frame_walk_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64),
                                            ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32)]),
    "qsim_landscape_clear_cache": (None, []),
    "qsim_last_error": (ctypes.c_char_p, []),
}


def lib():
    """The loaded ``libqsim.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2404_09213_gb300.build` "
                              "(or __graft_entry__.build()); there is no non-CUDA fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code: int):
    if code != 0:
        raise QsimError(code, lib().qsim_last_error().decode())
    return code
