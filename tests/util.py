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


def f64_distill_reference(W, cfg, x, cu, tl, tr, operand_format=None):
    """The distillation loss of a sequential-architecture model and its gradient
    from an independent torch float64 model (torch.nn.functional layers, exact
    scaled-dot-product attention, autograd).  Returns (loss, {name: grad}).

    operand_format "bf16" / "fp16": every linear layer rounds its GEMM operands to that
    format, in the forward (input and weight) and in the backward (the output gradient,
    with the rounded weight for the input gradient and the rounded input for the weight
    gradient), and attention rounds the operands of its products (RoundedAttention): the
    arithmetic of a mixed-precision training step whose GEMMs and attention products run
    on 16-bit tensor cores with exact accumulation; everything else stays float64."""
    import torch
    import torch.nn.functional as F

    import oracle
    P = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True) for k, v in W.items()}
    act = (lambda t: F.relu(t)) if cfg.act == 1 else (lambda t: F.gelu(t, approximate="none"))
    if operand_format is not None:
        dt = {"bf16": torch.bfloat16, "fp16": torch.float16}[operand_format]
        rnd = lambda t: t.float().to(dt).double()

        class RoundedLinear(torch.autograd.Function):
            @staticmethod
            def forward(ctx, t, w, b):
                tr_, wr = rnd(t), rnd(w)
                ctx.save_for_backward(tr_, wr)
                return tr_ @ wr.T + b

            @staticmethod
            def backward(ctx, gy):
                tr_, wr = ctx.saved_tensors
                gr = rnd(gy)
                return gr @ wr, gr.T @ tr_, gy.sum(0)

        LOG2E = 1.0 / np.log(2.0)

        class RoundedAttention(torch.autograd.Function):
            """softmax(q k^T / sqrt(dh)) v per head with the operands of its four products
            rounded: q / sqrt(dh) log2(e), k, v and the unnormalised probabilities in the
            forward; the output gradient, the probabilities and the score gradient in the
            backward (probabilities recomputed from the log-sum-exp)."""

            @staticmethod
            def forward(ctx, q, k, v):
                sc = 1.0 / np.sqrt(q.shape[-1])
                qr, kr, vr = rnd(q * sc * LOG2E), rnd(k), rnd(v)
                s2 = qr @ kr.transpose(-1, -2)
                m = s2.amax(-1, keepdim=True)
                e = torch.exp2(s2 - m)
                l = e.sum(-1, keepdim=True)
                o = (rnd(e) @ vr) / l
                ctx.save_for_backward(qr, kr, vr, m + torch.log2(l), o)
                ctx.sc = sc
                return o

            @staticmethod
            def backward(ctx, go):
                qr, kr, vr, lse2, o = ctx.saved_tensors
                p = torch.exp2(qr @ kr.transpose(-1, -2) - lse2)
                Dr = (go * o).sum(-1, keepdim=True)
                gr = rnd(go)
                ds = p * (gr @ vr.transpose(-1, -2) - Dr)
                dsr = rnd(ds)
                return ctx.sc * (dsr @ kr), (dsr.transpose(-1, -2) @ qr) / LOG2E, rnd(p).transpose(-1, -2) @ gr

        F = type("F", (), {k: staticmethod(getattr(torch.nn.functional, k)) for k in
                           ("relu", "gelu", "layer_norm", "log_softmax")})
        F.linear = staticmethod(lambda t, w, b: RoundedLinear.apply(t, w, b))
        F.scaled_dot_product_attention = staticmethod(lambda q, k, v: RoundedAttention.apply(q, k, v))
    mlp = lambda t, p: F.linear(act(F.linear(t, P[p + "w1"], P[p + "b1"])), P[p + "w2"], P[p + "b2"])
    ln = lambda t, p: F.layer_norm(t, (cfg.d,), P[p + ".g"], P[p + ".b"], eps=1e-5)

    def stack(z, pre, n):
        for l in range(n):
            p = f"{pre}.{l}."
            zn = ln(z, p + "ln1")
            split = lambda t: t.view(-1, cfg.heads, cfg.dh).transpose(0, 1)
            q, k, v = (split(F.linear(zn, P[p + "w" + c], P[p + "b" + c])) for c in "qkv")
            o = F.scaled_dot_product_attention(q, k, v).transpose(0, 1).reshape(-1, cfg.d)
            z = z + F.linear(o, P[p + "wo"], P[p + "bo"])
            z = z + F.linear(act(F.linear(ln(z, p + "ln2"), P[p + "ffn.w1"], P[p + "ffn.b1"])),
                             P[p + "ffn.w2"], P[p + "ffn.b2"])
        return ln(z, pre + ".lnf")

    total = 0.0
    for e in range(len(cu) - 1):
        if cu[e + 1] == cu[e]:
            continue
        xe = torch.tensor(x[cu[e]:cu[e + 1]], dtype=torch.float64)
        hp = stack(mlp(xe, "emb."), "pid", cfg.l_pid)
        hr = stack(mlp(torch.cat([xe, hp], 1), "remb."), "reg", cfg.l_reg)
        logits = mlp(hp, "head.cls.")
        raw = torch.cat([mlp(hr, f"head.{n}.") for n, _ in synth.REG_HEADS], 1)
        tlog = torch.tensor(tl[cu[e]:cu[e + 1]], dtype=torch.float64)
        traw = torch.tensor(oracle.raw_from_decoded(x[cu[e]:cu[e + 1]], tr[cu[e]:cu[e + 1]]))
        lt = F.log_softmax(tlog, 1)
        kl = (lt.exp() * (lt - F.log_softmax(logits, 1))).sum(1)
        total = total + (kl + ((raw - traw) ** 2).sum(1)).sum()
    loss = total / x.shape[0]
    loss.backward()
    return float(loss.detach()), {n: P[n].grad.numpy() for n in W}
