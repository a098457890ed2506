"""Shared helpers for the GPU parity tests: run the library, compare to the oracle."""
from __future__ import annotations

import numpy as np

import synth


def rel_err_cols(y, ref):
    """Per-column normwise relative error ||y - ref||_2 / ||ref||_2."""
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    num = np.sqrt(((y - ref) ** 2).sum(axis=0))
    den = np.sqrt((ref ** 2).sum(axis=0))
    return num / np.maximum(den, 1e-300)


def max_scaled_err(y, ref):
    """max |y - ref| / max(|ref|, rms(ref column)) over all elements."""
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    rms = np.sqrt((ref ** 2).mean(axis=0, keepdims=True))
    return float((np.abs(y - ref) / np.maximum(np.abs(ref), rms)).max())


def run_gpu(model, x, cu, precision, max_n=None):
    """Run the library on numpy inputs; returns numpy (logits, reg, cls, sums)."""
    import torch
    xt = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    ct = torch.from_numpy(np.ascontiguousarray(cu, np.int32)).cuda()
    sizes = np.diff(np.asarray(cu, np.int64))
    mn = int(sizes.max()) if max_n is None and len(sizes) else (max_n or 0)
    lo, rg, cl, su = model.forward(xt, ct, mn, precision=precision)
    model.sync()
    return (lo.cpu().numpy(), rg.cpu().numpy(), cl.cpu().numpy(), su.cpu().numpy())


def make_model(cfg, seed, perturbed=False, cls_scale=1.0):
    from paper_2601_17554_b300 import Model
    w = synth.make_weights(cfg, seed, perturbed=perturbed, cls_scale=cls_scale)
    return Model(synth.pack_blob(cfg, w)), w
