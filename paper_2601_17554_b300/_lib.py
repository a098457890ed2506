"""ctypes declarations of the C ABI in include/mlpf.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmlpf.so")

MLPF_OK, MLPF_E_INVALID, MLPF_E_FORMAT, MLPF_E_CUDA, MLPF_E_OOM, MLPF_E_TIMEOUT, \
    MLPF_E_NONFINITE, MLPF_E_UNSUPPORTED = range(8)
MLPF_FP32, MLPF_BF16, MLPF_FP8, MLPF_FP16 = 0, 1, 2, 3
OPT_USE_GRAPHS, OPT_WAIT_LIMIT_NS, OPT_DEBUG_STALL, OPT_ATTN_CTAS_PER_SM, OPT_ATTN_KV_STAGES, \
    OPT_PROFILE, OPT_ATTN_VARIANT_BF16, OPT_ATTN_VARIANT_FP16, OPT_ATTN_VARIANT_FP8, \
    OPT_ATTN_WINDOW, OPT_GATE_CONFIDENCE, OPT_HOST_CHUNKS, OPT_HOST_STREAMS, OPT_WIDE_ATTN_KERNEL = range(1, 15)

# every symbol include/mlpf.h declares
EXPORTS = ("mlpf_load_weights", "mlpf_free", "mlpf_get_config", "mlpf_forward",
           "mlpf_forward_host", "mlpf_forward_noalloc", "mlpf_calibrate_fp8",
           "mlpf_get_fp8_scales", "mlpf_autotune", "mlpf_measure_unit_rates",
           "mlpf_eval_activation", "mlpf_forward_gated", "mlpf_trainer_create",
           "mlpf_trainer_free", "mlpf_trainer_num_params", "mlpf_trainer_step",
           "mlpf_trainer_step_supervised", "mlpf_trainer_export", "mlpf_sync", "mlpf_set_option", "mlpf_get_option",
           "mlpf_last_launch_count", "mlpf_profile_get", "mlpf_last_error", "mlpf_abi_version",
           "mlpf_cluster_jets", "mlpf_measure_ex2_packed_rate", "mlpf_trainer_forward",
           "mlpf_trainer_backward", "mlpf_trainer_params", "mlpf_shard_events",
           "mlpf_trainer_set_precision", "mlpf_gemm_tc")


class MlpfConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("in_dim", "d", "heads", "ffn", "l_pid", "l_reg", "n_cls", "n_reg", "act", "arch")]


_handle = None


def load(build_if_missing: bool = True):
    """Load libmlpf.so (building it with nvcc first if it is missing)."""
    global _handle
    if _handle is not None:
        return _handle
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(f"{LIB_PATH} is missing; run python -m paper_2601_17554_b300.build")
        from .build import build
        build()
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    L.mlpf_load_weights.argtypes = [vp, sz, ctypes.c_int, ctypes.POINTER(vp)]
    L.mlpf_load_weights.restype = ctypes.c_int
    L.mlpf_free.argtypes = [vp]
    L.mlpf_free.restype = None
    L.mlpf_get_config.argtypes = [vp, ctypes.POINTER(MlpfConfig)]
    L.mlpf_get_config.restype = ctypes.c_int
    fwd = [vp, i32, vp, vp, i32, i32, i32, vp, vp, vp, vp, vp]
    L.mlpf_forward.argtypes = fwd
    L.mlpf_forward.restype = ctypes.c_int
    L.mlpf_forward_host.argtypes = fwd
    L.mlpf_forward_host.restype = ctypes.c_int
    L.mlpf_forward_noalloc.argtypes = fwd
    L.mlpf_forward_noalloc.restype = ctypes.c_int
    L.mlpf_calibrate_fp8.argtypes = [vp, vp, vp, i32, i32, i32, vp]
    L.mlpf_calibrate_fp8.restype = ctypes.c_int
    L.mlpf_measure_unit_rates.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
    L.mlpf_measure_unit_rates.restype = ctypes.c_int
    L.mlpf_measure_ex2_packed_rate.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    L.mlpf_measure_ex2_packed_rate.restype = ctypes.c_int
    L.mlpf_cluster_jets.argtypes = [vp, vp, vp, vp, i32, i32, ctypes.c_float, vp, vp, vp, vp]
    L.mlpf_cluster_jets.restype = ctypes.c_int
    L.mlpf_eval_activation.argtypes = [i32, i32, vp, vp, i32, vp]
    L.mlpf_eval_activation.restype = ctypes.c_int
    L.mlpf_autotune.argtypes = [vp, i32, vp, vp, i32, i32, i32, ctypes.c_char_p, vp]
    L.mlpf_autotune.restype = ctypes.c_int
    L.mlpf_get_fp8_scales.argtypes = [vp, i32, ctypes.c_char_p, ctypes.POINTER(ctypes.c_float)]
    L.mlpf_get_fp8_scales.restype = i32
    L.mlpf_forward_gated.argtypes = [vp, vp, ctypes.c_float, i32, i32, vp, vp, i32, i32, i32, vp, vp, vp,
                                     vp, vp, ctypes.POINTER(i32), vp]
    L.mlpf_forward_gated.restype = ctypes.c_int
    L.mlpf_trainer_create.argtypes = [vp, sz, ctypes.c_int, ctypes.POINTER(vp)]
    L.mlpf_trainer_create.restype = ctypes.c_int
    L.mlpf_trainer_free.argtypes = [vp]
    L.mlpf_trainer_free.restype = None
    L.mlpf_trainer_num_params.argtypes = [vp]
    L.mlpf_trainer_num_params.restype = i64
    L.mlpf_trainer_step.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, ctypes.c_float, i32, vp,
                                    ctypes.POINTER(ctypes.c_double), vp]
    L.mlpf_trainer_step.restype = ctypes.c_int
    L.mlpf_trainer_step_supervised.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, ctypes.c_float,
                                               ctypes.c_float, ctypes.c_float, ctypes.c_float, i32, vp,
                                               ctypes.POINTER(ctypes.c_double), vp]
    L.mlpf_trainer_step_supervised.restype = ctypes.c_int
    L.mlpf_trainer_forward.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, vp]
    L.mlpf_trainer_forward.restype = ctypes.c_int
    L.mlpf_trainer_backward.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, vp, vp]
    L.mlpf_trainer_backward.restype = ctypes.c_int
    L.mlpf_trainer_params.argtypes = [vp, vp, vp, vp]
    L.mlpf_trainer_params.restype = ctypes.c_int
    L.mlpf_trainer_set_precision.argtypes = [vp, i32]
    L.mlpf_trainer_set_precision.restype = ctypes.c_int
    L.mlpf_gemm_tc.argtypes = [i32, vp, i64, vp, i64, i32, i32, i32, vp, i64, vp, vp, i64, i32, i32, i32, vp, vp]
    L.mlpf_gemm_tc.restype = ctypes.c_int
    L.mlpf_trainer_export.argtypes = [vp, vp, sz, ctypes.POINTER(sz)]
    L.mlpf_trainer_export.restype = ctypes.c_int
    L.mlpf_sync.argtypes = [vp, vp]
    L.mlpf_sync.restype = ctypes.c_int
    L.mlpf_set_option.argtypes = [vp, i32, i64]
    L.mlpf_set_option.restype = ctypes.c_int
    L.mlpf_get_option.argtypes = [vp, i32, ctypes.POINTER(i64)]
    L.mlpf_get_option.restype = ctypes.c_int
    L.mlpf_last_launch_count.argtypes = [vp]
    L.mlpf_last_launch_count.restype = i64
    L.mlpf_profile_get.argtypes = [vp, i32, ctypes.c_char_p, ctypes.POINTER(ctypes.c_float)]
    L.mlpf_profile_get.restype = i32
    L.mlpf_last_error.argtypes = []
    L.mlpf_last_error.restype = ctypes.c_char_p
    L.mlpf_shard_events.argtypes = [vp, i32, i32, vp, vp]
    L.mlpf_shard_events.restype = ctypes.c_int
    L.mlpf_abi_version.argtypes = []
    L.mlpf_abi_version.restype = i32
    _handle = L
    return L


class MlpfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mlpf status {status}: {msg}")
        self.status = status


def check(status: int):
    if status != MLPF_OK:
        raise MlpfError(status, load().mlpf_last_error().decode(errors="replace"))
