"""torch.autograd.Function over the library's hand-written training kernels.

`StudentMLPF` is a torch.nn.Module whose one parameter is the flat parameter
vector of an MLPF model (blob tensor order).  Its forward runs the library's FP32
training forward (mlpf_trainer_forward) and its backward the hand-written backward
kernels (mlpf_trainer_backward: GEMMs, LayerNorm, GELU, varlen attention with the
probabilities recomputed from Q, K and the saved log-sum-exp), so any torch loss
and optimizer can drive them.  This module only marshals pointers; every step of
the forward and backward runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import Trainer, _ptr, check


class StudentFunction(torch.autograd.Function):
    """(params, x, cu_seqlens, max_n, trainer) -> (logits [T, 6], raw [T, 5]).

    The trainer keeps the activations of the last forward: call backward before
    the next forward on the same trainer (torch's usual forward/backward order).
    """

    @staticmethod
    def forward(ctx, params, x, cu_seqlens, max_n, trainer):
        L = trainer.L
        T, n = x.shape[0], cu_seqlens.shape[0] - 1
        s = ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
        params = params.detach().contiguous()
        check(L.mlpf_trainer_params(trainer.h, None, _ptr(params), s))
        logits = torch.empty((T, 6), dtype=torch.float32, device=x.device)
        raw = torch.empty((T, 5), dtype=torch.float32, device=x.device)
        check(L.mlpf_trainer_forward(trainer.h, _ptr(x), _ptr(cu_seqlens), n, T, int(max_n),
                                     _ptr(logits), _ptr(raw), s))
        ctx.trainer, ctx.x, ctx.cu, ctx.max_n = trainer, x, cu_seqlens, int(max_n)
        ctx.n_params = params.shape[0]
        return logits, raw

    @staticmethod
    def backward(ctx, dlogits, draw):
        trainer, x, cu = ctx.trainer, ctx.x, ctx.cu
        T, n = x.shape[0], cu.shape[0] - 1
        dev = x.device
        dlogits = torch.zeros((T, 6), device=dev) if dlogits is None else dlogits.float().contiguous()
        draw = torch.zeros((T, 5), device=dev) if draw is None else draw.float().contiguous()
        g = torch.empty((ctx.n_params,), dtype=torch.float32, device=dev)
        s = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        check(trainer.L.mlpf_trainer_backward(trainer.h, _ptr(x), _ptr(cu), n, T, ctx.max_n,
                                              _ptr(dlogits), _ptr(draw), _ptr(g), s))
        return g, None, None, None, None


class StudentMLPF(torch.nn.Module):
    """An MLPF model (weight blob) as a torch module trained through the library's
    hand-written forward and backward kernels."""

    def __init__(self, blob: bytes, device: int = 0, precision: str = "fp32"):
        super().__init__()
        self.trainer = Trainer(blob, device, precision)
        p = torch.empty((self.trainer.num_params,), dtype=torch.float32, device=torch.device("cuda", device))
        s = ctypes.c_void_p(torch.cuda.current_stream(p.device).cuda_stream)
        check(self.trainer.L.mlpf_trainer_params(self.trainer.h, _ptr(p), None, s))
        self.params = torch.nn.Parameter(p)

    def forward(self, x, cu_seqlens, max_n: int):
        """(logits [T, 6], raw head outputs [T, 5]) of a packed batch (device tensors)."""
        return StudentFunction.apply(self.params, x, cu_seqlens, max_n, self.trainer)

    def export(self) -> bytes:
        """The current parameters as a weight blob (loadable with Model)."""
        s = ctypes.c_void_p(torch.cuda.current_stream(self.params.device).cuda_stream)
        check(self.trainer.L.mlpf_trainer_params(self.trainer.h, None, _ptr(self.params.detach()), s))
        torch.cuda.current_stream(self.params.device).synchronize()
        return self.trainer.export()

    def close(self):
        self.trainer.close()


def distill_loss(logits, raw, x, t_logits, t_reg):
    """The distillation loss (KL of the class probabilities plus the squared error of
    the raw regression outputs against the teacher's raw values recovered from its
    decoded ones, Eq. 2), averaged over elements, in torch (for the autograd path)."""
    lt = torch.log_softmax(t_logits, dim=1)
    ls = torch.log_softmax(logits, dim=1)
    kl = (lt.exp() * (lt - ls)).sum(dim=1)
    traw = t_reg.clone()
    traw[:, 0] = torch.log(t_reg[:, 0]) - x[:, 8]
    traw[:, 4] = torch.log(t_reg[:, 4]) - x[:, 9]
    return (kl + ((raw - traw) ** 2).sum(dim=1)).mean()
