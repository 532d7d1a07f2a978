"""ctypes declarations of libsimplexenc's C ABI (``include/simplexenc.h``).

This module only loads the shared library and declares argument types.  There
is no fallback: if the library is missing or fails to load, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsimplexenc.so")

SXE_OK, SXE_EINVAL, SXE_EUNSUPPORTED, SXE_ECUDA, SXE_ENOMEM = 0, -1, -2, -3, -4
SXE_SIMPLEX, SXE_GRID = 0, 1
SXE_F32, SXE_F16, SXE_BF16 = 0, 1, 2
SXE_RES_RAW, SXE_RES_EQUAL_MEM = 0, 1
SXE_INDEX_HASH, SXE_INDEX_DENSE_COARSE = 0, 1
SXE_MAX_LEVELS = 32
SXE_MLP_KERNEL_AUTO, SXE_MLP_KERNEL_MMA_SYNC, SXE_MLP_KERNEL_TCGEN05, SXE_MLP_KERNEL_TCGEN05_PIPELINED = 0, 1, 2, 3
SXE_MLP_KERNEL_TCGEN05_3TILE = 4
SXE_FWD_ORDER_AUTO, SXE_FWD_ORDER_POINT_MAJOR, SXE_FWD_ORDER_LEVEL_MAJOR = 0, 1, 2

#: every function the header declares (checked by the export test)
EXPORTS = (
    "sxe_encoder_create", "sxe_encoder_destroy", "sxe_encoder_level_params", "sxe_encoder_level_index",
    "sxe_encoder_set_bwd_aggregation", "sxe_encoder_set_fwd_order",
    "sxe_encode_fwd", "sxe_encode_fwd_marked", "sxe_encode_bwd", "sxe_encode_bwd_levels", "sxe_encode_bwd_kernel_count",
    "sxe_encode_bwd_levels_kernel_count", "sxe_encode_bwd_coarse_levels", "sxe_encode_bwd_input",
    "sxe_encode_vertices",
    "sxe_encode_plain_fwd", "sxe_encode_plain_bwd", "sxe_vr_samples", "sxe_vr_field", "sxe_vr_field_mlp", "sxe_vr_field_mlp_saved", "sxe_vr_composite",
    "sxe_vr_composite_bwd", "sxe_vr_field_bwd",
    "sxe_adam_advance", "sxe_step_dev", "sxe_step_touched_dev",
    "sxe_mlp_n_params", "sxe_mlp_fwd", "sxe_mlp_bwd_workspace_bytes", "sxe_mlp_bwd", "sxe_mlp_train_l2",
    "sxe_loss_l2", "sxe_step", "sxe_step_touched", "sxe_last_error", "sxe_version",
    "sxe_mlp_train_l2_static", "sxe_mlp_train_l2_grouped", "sxe_mlp_train_l2_part",
    "sxe_mlp_set_kernel", "sxe_mlp_get_kernel", "sxe_device_error", "sxe_selftest_wait",
    "sxe_server_create", "sxe_server_add_field", "sxe_server_start", "sxe_server_submit", "sxe_server_wait",
    "sxe_server_stop", "sxe_server_stats", "sxe_server_destroy",
)


class EncodingDesc(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("n_levels", ctypes.c_int32), ("n_features", ctypes.c_int32),
                ("log2_T", ctypes.c_int32), ("base_res", ctypes.c_double), ("growth", ctypes.c_double),
                ("kind", ctypes.c_int32), ("res_mode", ctypes.c_int32), ("table_dtype", ctypes.c_int32),
                ("out_dtype", ctypes.c_int32), ("index_mode", ctypes.c_int32)]


class MlpDesc(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("width", ctypes.c_int32), ("n_hidden", ctypes.c_int32),
                ("n_out", ctypes.c_int32), ("dtype", ctypes.c_int32)]


class AdamDesc(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("skip_zero_grad", ctypes.c_int32)]


class ServerDesc(ctypes.Structure):
    _fields_ = [("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_int64), ("n_slots", ctypes.c_int32),
                ("max_batch_points", ctypes.c_int64), ("priority_points", ctypes.c_int64)]


_lib = None


def _declare(L):
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    E = ctypes.POINTER(EncodingDesc)
    M = ctypes.POINTER(MlpDesc)
    A = ctypes.POINTER(AdamDesc)
    sig = {
        "sxe_encoder_create": (i32, [E, ctypes.POINTER(vp)]),
        "sxe_encoder_destroy": (i32, [vp]),
        "sxe_encoder_level_params": (i32, [vp, vp, vp]),
        "sxe_encoder_level_index": (i32, [vp, vp]),
        "sxe_encoder_set_bwd_aggregation": (i32, [vp, i32]),
        "sxe_encoder_set_fwd_order": (i32, [vp, i32]),
        "sxe_encode_fwd": (i32, [vp, vp, i64, vp, vp, vp]),
        "sxe_encode_fwd_marked": (i32, [vp, vp, i64, vp, vp, vp, vp]),
        "sxe_encode_bwd": (i32, [vp, vp, i64, vp, vp, i64, vp, vp]),
        "sxe_encode_bwd_input": (i32, [vp, vp, i64, vp, vp, vp, vp]),
        "sxe_encode_bwd_kernel_count": (i32, [vp, i64]),
        "sxe_encode_bwd_levels": (i32, [vp, vp, i64, vp, vp, i64, vp, i32, i32, vp]),
        "sxe_encode_bwd_levels_kernel_count": (i32, [vp, i64, i32, i32]),
        "sxe_encode_bwd_coarse_levels": (i32, [vp, i64]),
        "sxe_encode_vertices": (i32, [vp, vp, i64, vp, vp, vp]),
        "sxe_encode_plain_fwd": (i32, [vp, vp, i64, vp, vp, vp]),
        "sxe_vr_samples": (i32, [vp, vp, vp, vp, i64, i32, vp, vp, vp]),
        "sxe_adam_advance": (i32, [A, vp, vp, vp]),
        "sxe_step_dev": (i32, [A, vp, i64, vp, vp, vp, vp, vp, i32, vp]),
        "sxe_step_touched_dev": (i32, [A, vp, i64, i32, vp, vp, vp, i32, vp]),
        "sxe_vr_field": (i32, [vp, vp, i64, i32, i32, vp, vp, vp]),
        "sxe_vr_composite_bwd": (i32, [vp, vp, vp, vp, vp, i64, i32, vp, vp, vp]),
        "sxe_vr_field_bwd": (i32, [vp, vp, vp, vp, i64, i32, vp, vp]),
        "sxe_vr_field_mlp": (i32, [M, vp, M, vp, vp, vp, i64, i32, vp, vp, vp]),
        "sxe_vr_field_mlp_saved": (i32, [M, vp, M, vp, vp, vp, i64, i32, vp, vp, vp, vp, vp]),
        "sxe_vr_composite": (i32, [vp, vp, vp, i64, i32, vp, vp, vp, vp]),
        "sxe_encode_plain_bwd": (i32, [vp, vp, i64, vp, vp, vp]),
        "sxe_mlp_n_params": (i64, [M]),
        "sxe_mlp_fwd": (i32, [M, vp, vp, i64, vp, vp, vp]),
        "sxe_mlp_bwd_workspace_bytes": (i64, [M, i64]),
        "sxe_mlp_bwd": (i32, [M, vp, vp, vp, f32, i64, vp, vp, vp, i64, vp]),
        "sxe_mlp_train_l2": (i32, [M, vp, vp, vp, f32, i64, vp, vp, vp, vp, i64, vp]),
        "sxe_loss_l2": (i32, [vp, vp, i64, i32, vp, vp, vp]),
        "sxe_step": (i32, [A, i64, i64, vp, vp, vp, vp, vp, i32, vp]),
        "sxe_step_touched": (i32, [A, i64, i64, i32, vp, vp, vp, i32, vp]),
        "sxe_mlp_train_l2_grouped": (i32, [M, vp, vp, vp, f32, i64, vp, i32, vp, vp, vp, i64, vp]),
        "sxe_mlp_train_l2_static": (i32, [M, vp, vp, vp, f32, i64, vp, vp, vp, vp]),
        "sxe_mlp_train_l2_part": (i32, [M, vp, vp, vp, f32, i64, i64, vp, vp, vp, vp, i64, vp]),
        "sxe_mlp_set_kernel": (i32, [i32]),
        "sxe_mlp_get_kernel": (i32, []),
        "sxe_device_error": (i32, [ctypes.POINTER(i32), i32]),
        "sxe_selftest_wait": (i32, [i32, i64, vp]),
        "sxe_server_create": (i32, [ctypes.POINTER(ServerDesc), ctypes.POINTER(vp)]),
        "sxe_server_add_field": (i32, [vp, vp, vp, M, vp]),
        "sxe_server_start": (i32, [vp]),
        "sxe_server_submit": (i32, [vp, i32, vp, i64, vp, ctypes.POINTER(i64)]),
        "sxe_server_wait": (i32, [vp, i64, i64, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]),
        "sxe_server_stop": (i32, [vp, i32]),
        "sxe_server_stats": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "sxe_server_destroy": (i32, [vp]),
        "sxe_last_error": (ctypes.c_char_p, []),
        "sxe_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def lib(path: str | None = None):
    """The loaded library (loaded once).  Raises if it is not built."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                "libsimplexenc.so is not built (%s); run paper_2311_15439_gb300.build.build() "
                "or __graft_entry__.build() first -- there is no CPU fallback" % p)
        L = ctypes.CDLL(p)
        _declare(L)
        _lib = L
    return _lib


class SxeError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().sxe_last_error().decode(errors="replace")
        super().__init__("%s failed with status %d: %s" % (where, status, msg))
        self.status = status


def check(status: int, where: str) -> None:
    if status != SXE_OK:
        raise SxeError(status, where)
