"""B300 (sm_103a) MLPF full-event transformer forward behind a C ABI.

This module is a thin binding: it passes torch tensors' device pointers, sizes
and the current CUDA stream to the C entry points of libmlpf.so
(include/mlpf.h).  Every step of the forward runs in the library's CUDA
kernels; there is no CPU or PyTorch fallback: if the library cannot be loaded
or the GPU path fails, the calls raise.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import (MLPF_FP32, MLPF_BF16, MLPF_FP8, MLPF_FP16, MlpfError, check,  # noqa: F401
                   OPT_USE_GRAPHS, OPT_WAIT_LIMIT_NS, OPT_DEBUG_STALL, OPT_ATTN_VARIANT_BF16,
                   OPT_ATTN_VARIANT_FP16, OPT_ATTN_VARIANT_FP8, OPT_ATTN_WINDOW)

PRECISIONS = {"fp32": MLPF_FP32, "bf16": MLPF_BF16, "fp8": MLPF_FP8, "fp16": MLPF_FP16}


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def measure_unit_rates(device: int = 0) -> dict:
    """Measured MUFU exp2 (FP32 and packed BF16) and FP32 FMA rates (results per
    second) of a device."""
    L = _lib.load()
    ex2, ffma = ctypes.c_double(), ctypes.c_double()
    check(L.mlpf_measure_unit_rates(device, ctypes.byref(ex2), ctypes.byref(ffma)))
    packed = ctypes.c_double()
    check(L.mlpf_measure_ex2_packed_rate(device, ctypes.byref(packed)))
    return {"ex2_per_s": ex2.value, "ffma_per_s": ffma.value, "ex2_bf16x2_per_s": packed.value}


def shard_events(sizes, n_shards: int):
    """Cost-balanced split of a batch's events over n_shards devices (LPT on N^2, in the
    library; host arrays).  Returns (shard_of_event int32 [n_events], shard_cost
    float64 [n_shards])."""
    import numpy as np
    L = _lib.load()
    sz = np.ascontiguousarray(sizes, np.int32)
    shard = np.empty(len(sz), np.int32)
    cost = np.empty(int(n_shards), np.float64)
    check(L.mlpf_shard_events(sz.ctypes.data_as(ctypes.c_void_p), len(sz), int(n_shards),
                              shard.ctypes.data_as(ctypes.c_void_p), cost.ctypes.data_as(ctypes.c_void_p)))
    return shard, cost


class Model:
    """A loaded MLPF model on one CUDA device (owns weights and workspace)."""

    def __init__(self, blob: bytes, device: int = 0):
        self.L = _lib.load()
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(blob, len(blob))
        check(self.L.mlpf_load_weights(buf, len(blob), device, ctypes.byref(h)))
        self.h = h
        self.device = device
        cfg = _lib.MlpfConfig()
        check(self.L.mlpf_get_config(self.h, ctypes.byref(cfg)))
        self.config = {n: getattr(cfg, n) for n, _ in _lib.MlpfConfig._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.L.mlpf_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option: int, value: int):
        check(self.L.mlpf_set_option(self.h, option, int(value)))

    def get_option(self, option: int) -> int:
        v = ctypes.c_int64()
        check(self.L.mlpf_get_option(self.h, option, ctypes.byref(v)))
        return v.value

    @property
    def last_launch_count(self) -> int:
        return int(self.L.mlpf_last_launch_count(self.h))

    def forward(self, x, cu_seqlens, max_n: int, precision="bf16", logits=None, reg=None,
                cls=None, event_sums=None, want_cls=True, want_sums=True, stream=None):
        """Batched forward over packed events (device tensors).

        x: float32 [total, 42] CUDA tensor; cu_seqlens: int32 [n_events+1] CUDA
        tensor.  Returns (logits [total,6], reg [total,5], cls [total] | None,
        event_sums [n_events,3] float64 | None), asynchronous on `stream`
        (default: torch's current stream).
        """
        import torch
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        total = x.shape[0]
        n_events = cu_seqlens.shape[0] - 1
        dev = x.device
        if logits is None:
            logits = torch.empty((total, 6), dtype=torch.float32, device=dev)
        if reg is None:
            reg = torch.empty((total, 5), dtype=torch.float32, device=dev)
        if cls is None and want_cls:
            cls = torch.empty((total,), dtype=torch.int32, device=dev)
        if event_sums is None and want_sums:
            event_sums = torch.empty((n_events, 3), dtype=torch.float64, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        check(self.L.mlpf_forward(self.h, prec, _ptr(x), _ptr(cu_seqlens), n_events, total,
                                  int(max_n), _ptr(logits), _ptr(reg), _ptr(cls),
                                  _ptr(event_sums), ctypes.c_void_p(stream)))
        return logits, reg, cls, event_sums

    def forward_host(self, x, cu_seqlens, max_n: int, precision="bf16", logits=None, reg=None,
                     cls=None, event_sums=None, stream=None):
        """Forward with host (CPU) tensors; copies in and out inside the call."""
        import torch
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        total = x.shape[0]
        n_events = cu_seqlens.shape[0] - 1
        if logits is None:
            logits = torch.empty((total, 6), dtype=torch.float32)
        if reg is None:
            reg = torch.empty((total, 5), dtype=torch.float32)
        s = ctypes.c_void_p(stream if stream is not None else
                            torch.cuda.current_stream(self.device).cuda_stream)
        check(self.L.mlpf_forward_host(self.h, prec, _ptr(x), _ptr(cu_seqlens), n_events, total,
                                       int(max_n), _ptr(logits), _ptr(reg), _ptr(cls),
                                       _ptr(event_sums), s))
        return logits, reg, cls, event_sums

    def cluster_jets(self, reg, cls, cu_seqlens, R: float = 0.4, jet_of: bool = True, stream=None):
        """Anti-kt jets of every event's reconstructed particles from the decoded
        outputs (device tensors): returns (jets [total, 4] (px, py, pz, E), event e's
        jets in rows cu[e] .. cu[e] + n_jets[e] - 1; n_jets [n_events] int32; jet_of
        [total] int32 or None).  Asynchronous on the stream."""
        import torch
        total = reg.shape[0]
        n_events = cu_seqlens.shape[0] - 1
        dev = reg.device
        jets = torch.empty((total, 4), dtype=torch.float32, device=dev)
        n_jets = torch.empty((n_events,), dtype=torch.int32, device=dev)
        jof = torch.empty((total,), dtype=torch.int32, device=dev) if jet_of else None
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        check(self.L.mlpf_cluster_jets(self.h, _ptr(reg), _ptr(cls), _ptr(cu_seqlens), n_events, total,
                                       float(R), _ptr(jets), _ptr(n_jets), _ptr(jof), ctypes.c_void_p(s)))
        return jets, n_jets, jof

    def autotune(self, x, cu_seqlens, max_n: int, precision="bf16", cache_path=None, stream=None):
        """Keep the fastest attention variant of `precision` on this batch (device
        tensors); returns the chosen variant index (None for fp32).  For models on the
        generic-width path the choice is the attention kernel (MLPF_OPT_WIDE_ATTN_KERNEL,
        read it with get_option); the returned variant then does not apply."""
        import torch
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        check(self.L.mlpf_autotune(self.h, prec, _ptr(x), _ptr(cu_seqlens), cu_seqlens.shape[0] - 1,
                                   x.shape[0], int(max_n),
                                   cache_path.encode() if cache_path else None, ctypes.c_void_p(s)))
        opt = {MLPF_BF16: OPT_ATTN_VARIANT_BF16, MLPF_FP16: OPT_ATTN_VARIANT_FP16,
               MLPF_FP8: OPT_ATTN_VARIANT_FP8}.get(prec)
        return self.get_option(opt) if opt else None

    def calibrate_fp8(self, x, cu_seqlens, max_n: int, stream=None):
        """Static FP8 activation scales from an FP16 run on these events (device tensors)."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        check(self.L.mlpf_calibrate_fp8(self.h, _ptr(x), _ptr(cu_seqlens), cu_seqlens.shape[0] - 1,
                                        x.shape[0], int(max_n), ctypes.c_void_p(s)))

    def fp8_scales(self) -> dict:
        """Activation scales of the FP8 calibration, by GEMM input."""
        n = self.L.mlpf_get_fp8_scales(self.h, 0, None, None)
        if n <= 0:
            return {}
        names = ctypes.create_string_buffer(32 * n)
        vals = (ctypes.c_float * n)()
        self.L.mlpf_get_fp8_scales(self.h, n, names, vals)
        return {names.raw[32 * i:32 * (i + 1)].split(b"\0")[0].decode(): vals[i] for i in range(n)}

    def sync(self, stream=None):
        """Wait for the stream and raise on a device-side timeout / non-finite output."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        check(self.L.mlpf_sync(self.h, ctypes.c_void_p(s)))


class Trainer:
    """Trainer of a model (hand-written forward/backward kernels, LAMB): distillation
    (arch 0, step) or the supervised loss of Eq. 1 (arch 1, step_supervised).
    precision: "fp32" (SIMT GEMMs) or "bf16" / "fp16" (linear-layer GEMMs on the tensor
    cores with 16-bit operands and FP32 accumulation; everything else FP32)."""

    def __init__(self, blob: bytes, device: int = 0, precision: str = "fp32"):
        self.L = _lib.load()
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(blob, len(blob))
        check(self.L.mlpf_trainer_create(buf, len(blob), device, ctypes.byref(h)))
        self.h = h
        self.device = device
        self.num_params = int(self.L.mlpf_trainer_num_params(self.h))
        self.set_precision(precision)

    def set_precision(self, precision):
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        check(self.L.mlpf_trainer_set_precision(self.h, p))
        self.precision = precision

    def close(self):
        if getattr(self, "h", None):
            self.L.mlpf_trainer_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, x, cu_seqlens, max_n: int, t_logits, t_reg, lr: float, update: bool = True,
             grads=None, want_loss: bool = True, stream=None):
        """One step on device tensors; returns the batch loss (or None if not wanted)."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        loss = ctypes.c_double(0.0)
        check(self.L.mlpf_trainer_step(self.h, _ptr(x), _ptr(cu_seqlens), cu_seqlens.shape[0] - 1,
                                       x.shape[0], int(max_n), _ptr(t_logits), _ptr(t_reg),
                                       float(lr), int(bool(update)), _ptr(grads),
                                       ctypes.byref(loss) if want_loss else None, ctypes.c_void_p(s)))
        return loss.value if want_loss else None

    def step_supervised(self, x, cu_seqlens, max_n: int, cls_target, reg_target, lr: float,
                        update: bool = True, grads=None, want_loss: bool = True, beta: float = 0.01,
                        focal_gamma: float = 2.0, delta: float = 1.0, stream=None):
        """One step on the loss of Eq. 1 (arch-1 model; device tensors); returns the loss."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        loss = ctypes.c_double(0.0)
        check(self.L.mlpf_trainer_step_supervised(
            self.h, _ptr(x), _ptr(cu_seqlens), cu_seqlens.shape[0] - 1, x.shape[0], int(max_n),
            _ptr(cls_target), _ptr(reg_target), float(beta), float(focal_gamma), float(delta), float(lr),
            int(bool(update)), _ptr(grads), ctypes.byref(loss) if want_loss else None, ctypes.c_void_p(s)))
        return loss.value if want_loss else None

    def export(self) -> bytes:
        """Current weights as a weight blob (loadable with Model)."""
        n = ctypes.c_size_t(0)
        check(self.L.mlpf_trainer_export(self.h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        check(self.L.mlpf_trainer_export(self.h, buf, n.value, ctypes.byref(n)))
        return buf.raw


def gemm_tc(A, B, C, bias=None, R=None, act: int = -1, mode: int = 0, kchunk: int = 0, status=None,
            stream=None):
    """C (op)= act(A B^T + bias) + R on the tensor cores (mlpf_gemm_tc): A [M, >=K], B [N, >=K]
    torch.bfloat16 or torch.float16 CUDA tensors with K = A's logical width (a multiple of 64),
    C [M, >=N] float32.  status: int32 CUDA tensor of one element (allocated if None);
    returned."""
    import torch
    L = _lib.load()
    prec = PRECISIONS["bf16"] if A.dtype == torch.bfloat16 else PRECISIONS["fp16"]
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=A.device)
    s = stream if stream is not None else torch.cuda.current_stream(A.device).cuda_stream
    M, K = A.shape
    N = B.shape[0]
    check(L.mlpf_gemm_tc(prec, _ptr(A), A.stride(0), _ptr(B), B.stride(0), M, N, K, _ptr(C), C.stride(0),
                         _ptr(bias), _ptr(R), R.stride(0) if R is not None else 0, act, mode, kchunk,
                         _ptr(status), ctypes.c_void_p(s)))
    return status


def forward_gated(student: Model, teacher: Model, threshold: float, x, cu_seqlens, max_n: int,
                  student_precision="bf16", teacher_precision="fp32", stream=None):
    """Student forward with per-event fallback to the teacher (device tensors).

    Returns (logits, reg, cls, event_sums, used_teacher [n_events] int32, n_fallback).
    """
    import torch
    sp = PRECISIONS[student_precision] if isinstance(student_precision, str) else int(student_precision)
    tp = PRECISIONS[teacher_precision] if isinstance(teacher_precision, str) else int(teacher_precision)
    total, n_events, dev = x.shape[0], cu_seqlens.shape[0] - 1, x.device
    logits = torch.empty((total, 6), dtype=torch.float32, device=dev)
    reg = torch.empty((total, 5), dtype=torch.float32, device=dev)
    cls = torch.empty((total,), dtype=torch.int32, device=dev)
    sums = torch.empty((n_events, 3), dtype=torch.float64, device=dev)
    used = torch.empty((n_events,), dtype=torch.int32, device=dev)
    nfb = ctypes.c_int32(0)
    s = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    check(student.L.mlpf_forward_gated(student.h, teacher.h, float(threshold), sp, tp, _ptr(x),
                                       _ptr(cu_seqlens), n_events, total, int(max_n), _ptr(logits),
                                       _ptr(reg), _ptr(cls), _ptr(sums), _ptr(used),
                                       ctypes.byref(nfb), ctypes.c_void_p(s)))
    return logits, reg, cls, sums, used, nfb.value
