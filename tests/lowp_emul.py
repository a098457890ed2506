"""Float64 emulation of the tensor-core path's roundings, one stage at a time.

TEST INFRASTRUCTURE (error-budget ablation of the 16-bit and E4M3 forward).

The tensor-core forward keeps LayerNorm moments, softmax statistics, the
residual stream and every accumulator in FP32 and rounds values only where they
become a GEMM operand or are stored in 16 bits.  This module takes the oracle's
float64 forward (same order of steps, Sec. 5.3) and inserts those roundings,
each switchable by name, so that the error each one contributes to the class
argmax and the regressions can be measured on the CPU:

  x        element features as the embedding GEMM's A operand
  w_emb    embedding weights (42 -> d -> d, and the regression-stack input FFN)
  emb_h    embedding hidden layer (after the activation)
  ln1      LN1 output, A operand of the fused Q/K/V projection
  w_qkv    Q/K/V projection weights
  qk       stored Q (pre-multiplied by log2(e)/sqrt(dh)) and K
  v        stored V
  p_arg    exponent argument S - max of the softmax numerators (a packed 16-bit
           exponential rounds it before the exponential)
  p        softmax numerators P (the row sums are taken from the rounded P)
  o        stored attention output (A operand of the out-projection)
  w_o      out-projection weights
  ln2      LN2 output (A operand of FFN up)
  w_ffn    FFN weights
  ffn_h    FFN hidden layer (after the activation)
  hpid     final-normed PID-stack output (stored; A operand of the class head
           and part of the regression-stack input)
  hreg     final-normed regression-stack output (A operand of the heads)
  w_head1  first layers of the output heads
  head_h   head hidden layers (after the activation)
  w_head2  last layers of the output heads

`fmt` maps a stage to a format: "bf16", "fp16", "e4m3" (with a per-tensor
scale, Sec. 8 of the paper names quantisation as an optimisation) or None
(float64, no rounding).  With every stage None the emulation is the oracle's
forward; `tests/test_lowp_emul.py` pins that.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

F64 = np.float64
STAGES = ("x", "w_emb", "emb_h", "ln1", "w_qkv", "qk", "v", "p_arg", "p", "o", "w_o", "ln2", "w_ffn",
          "ffn_h", "hpid", "hreg", "w_head1", "head_h", "w_head2")


# --------------------------------------------------------------- roundings

def round_bf16(a):
    """Round to the nearest BF16 (ties to even), via FP32 as the GPU does."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(F64)


def round_fp16(a):
    """Round to the nearest IEEE half (ties to even), via FP32."""
    return np.asarray(np.asarray(a, np.float32).astype(np.float16), F64)


def round_e4m3(a):
    """Round to the nearest E4M3 value (ties to even), saturating at +-448.

    E4M3: 3 mantissa bits, exponent bias 7, normal range 2^-6 .. 448,
    subnormals with spacing 2^-9.
    """
    a = np.asarray(a, F64)
    m = np.abs(a)
    e = np.floor(np.log2(np.where(m > 0, m, 1.0)))
    e = np.maximum(e, -6.0)
    q = np.exp2(e - 3.0)
    r = np.round(m / q) * q          # numpy rounds half to even
    r = np.minimum(r, 448.0)
    return np.copysign(r, a)


def rounder(fmt, scale=None):
    """A function rounding a float64 array to `fmt`; E4M3 values are divided by
    the per-tensor scale before and multiplied after the rounding."""
    if fmt is None:
        return lambda a: np.asarray(a, F64)
    if fmt == "bf16":
        return round_bf16
    if fmt == "fp16":
        return round_fp16
    if fmt == "e4m3":
        s = float(scale) if scale else 1.0
        return lambda a: round_e4m3(np.asarray(a, F64) / s) * s
    raise ValueError(fmt)


def amax_scale(a):
    """Per-tensor E4M3 scale amax / 448."""
    m = float(np.abs(np.asarray(a, F64)).max()) if np.size(a) else 0.0
    return m / 448.0 if m > 0 else 1.0


# ----------------------------------------------------------- the emulation

class Emulation:
    """Forward of the sequential architecture (arch 0) with rounding at named stages.

    fmt: dict stage -> format (missing = no rounding).  act_scales: dict of
    per-tensor E4M3 activation scales keyed "<stage>:<tensor>" (from
    `calibrate`); weight scales are amax/448 of each weight matrix.
    """

    def __init__(self, W, cfg, fmt=None, act_scales=None):
        assert getattr(cfg, "arch", 0) == 0
        self.W = W
        self.cfg = cfg
        self.fmt = dict(fmt or {})
        self.act_scales = dict(act_scales or {})
        self.record = None   # calibration: dict key -> running amax
        self._wcache = {}

    # a weight matrix rounded per its stage's format
    def wt(self, stage, name):
        key = (stage, name)
        if key not in self._wcache:
            w = np.asarray(self.W[name], F64)
            f = self.fmt.get(stage)
            sw = None
            if f == "e4m3":
                # per-tensor scale; the Q, K and V projections are one merged tensor
                grp = [name]
                for t in ("wq", "wk", "wv"):
                    if name.endswith("." + t):
                        grp = [name[:-len(t)] + u for u in ("wq", "wk", "wv")]
                sw = max(amax_scale(self.W[g]) for g in grp)
            self._wcache[key] = rounder(f, sw)(w)
        return self._wcache[key]

    # an activation rounded per its stage's format (key names the tensor)
    def act(self, stage, key, a):
        if self.record is not None:
            m = float(np.abs(a).max()) if np.size(a) else 0.0
            self.record[key] = max(self.record.get(key, 0.0), m)
        f = self.fmt.get(stage)
        return rounder(f, self.act_scales.get(key, 1.0) if f == "e4m3" else None)(a)

    def linear(self, a, wstage, name, bias):
        return a @ self.wt(wstage, name).T + np.asarray(self.W[bias], F64)

    def actf(self, v):
        return (oracle.relu if self.cfg.act == 1 else oracle.gelu)(v)

    def attention(self, q, k, v, tag):
        """One event's attention per head: scores in base 2 from the stored Q
        (pre-scaled by log2(e)/sqrt(dh)) and K, P = 2^(s - row max) rounded,
        O = (P V) / (P 1) from the rounded P and stored V, then O rounded."""
        d = q.shape[1]
        dh = d // self.cfg.heads
        c = math.log2(math.e) / math.sqrt(dh)
        rq = self.act("qk", tag + "q", q * c)
        rk = self.act("qk", tag + "k", k)
        rv = self.act("v", tag + "v", v)
        o = np.empty_like(q)
        for h in range(self.cfg.heads):
            sl = slice(h * dh, (h + 1) * dh)
            s = rq[:, sl] @ rk[:, sl].T
            p = np.exp2(self.act("p_arg", tag + "parg", s - s.max(axis=1, keepdims=True)))
            p = self.act("p", tag + "p", p)
            o[:, sl] = (p @ rv[:, sl]) / p.sum(axis=1, keepdims=True)
        return self.act("o", tag + "o", o)

    def block(self, z, p):
        W = self.W
        zn = self.act("ln1", p + "ln1", oracle.layer_norm(z, W[p + "ln1.g"], W[p + "ln1.b"]))
        q = self.linear(zn, "w_qkv", p + "wq", p + "bq")
        k = self.linear(zn, "w_qkv", p + "wk", p + "bk")
        v = self.linear(zn, "w_qkv", p + "wv", p + "bv")
        o = self.attention(q, k, v, p)
        z = z + self.linear(o, "w_o", p + "wo", p + "bo")
        zn = self.act("ln2", p + "ln2", oracle.layer_norm(z, W[p + "ln2.g"], W[p + "ln2.b"]))
        hid = self.act("ffn_h", p + "ffn_h", self.actf(self.linear(zn, "w_ffn", p + "ffn.w1", p + "ffn.b1")))
        return z + self.linear(hid, "w_ffn", p + "ffn.w2", p + "ffn.b2")

    def stack(self, z, prefix, n):
        for l in range(n):
            z = self.block(z, f"{prefix}.{l}.")
        return oracle.layer_norm(z, self.W[prefix + ".lnf.g"], self.W[prefix + ".lnf.b"])

    def head(self, h, name):
        pre = f"head.{name}."
        hid = self.actf(self.linear(h, "w_head1", pre + "w1", pre + "b1"))
        hid = self.act("head_h", pre + "h", hid)
        return self.linear(hid, "w_head2", pre + "w2", pre + "b2")

    def event(self, x):
        """x [N, 42] -> (logits [N, 6], raw [N, 5])."""
        cfg = self.cfg
        x = np.asarray(x, F64)
        xr = self.act("x", "x", x)
        e = self.act("emb_h", "emb_h", self.actf(self.linear(xr, "w_emb", "emb.w1", "emb.b1")))
        e = self.linear(e, "w_emb", "emb.w2", "emb.b2")
        h_pid = self.act("hpid", "hpid", self.stack(e, "pid", cfg.l_pid))
        logits = self.head(h_pid, "cls")
        xin = np.concatenate([xr, h_pid], axis=1)
        r = self.act("emb_h", "remb_h", self.actf(self.linear(xin, "w_emb", "remb.w1", "remb.b1")))
        r = self.linear(r, "w_emb", "remb.w2", "remb.b2")
        h_reg = self.act("hreg", "hreg", self.stack(r, "reg", cfg.l_reg))
        raw = np.concatenate([self.head(h_reg, n) for n, _ in (("pt", 1), ("eta", 1), ("phi", 2), ("e", 1))],
                             axis=1)
        return logits, raw

    def forward(self, x, cu, events=None):
        """Packed batch -> (logits, raw, reg, cls) over the listed events (all by default)."""
        x = np.asarray(x, F64)
        cu = np.asarray(cu, np.int64)
        todo = range(len(cu) - 1) if events is None else events
        rows = np.concatenate([np.arange(cu[e], cu[e + 1]) for e in todo]) if len(todo) else np.zeros(0, int)
        lo = np.zeros((len(rows), self.cfg.n_cls))
        raw = np.zeros((len(rows), self.cfg.n_reg))
        off = 0
        for e in todo:
            n = int(cu[e + 1] - cu[e])
            if n:
                lo[off:off + n], raw[off:off + n] = self.event(x[cu[e]:cu[e + 1]])
            off += n
        cls, reg = oracle.decode(x[rows], lo, raw)
        return lo, raw, reg, cls, rows

    def calibrate(self, x, cu):
        """Static per-tensor activation scales amax/448 from a run of this
        emulation (its own formats, typically FP16 everywhere)."""
        self.record = {}
        self.forward(x, cu)
        rec, self.record = self.record, None
        return {k: (m / 448.0 if m > 0 else 1.0) for k, m in rec.items()}


# formats of the GPU's precision modes (which stages round, to what)
def gpu_formats(mode):
    """Stage formats of the library's MLPF_BF16 / MLPF_FP16 / MLPF_FP8 modes."""
    if mode == "fp16":
        return {s: "fp16" for s in STAGES}     # packed FP16 exponentials: p_arg in FP16 too
    if mode == "bf16_all":
        f = {s: "bf16" for s in STAGES}
        f["p_arg"] = None                       # FP32 exponentials
        return f
    if mode == "bf16":
        f = {s: "fp16" for s in STAGES}
        for s in ("qk", "v", "p_arg", "p"):
            f[s] = "bf16"
        return f
    if mode == "fp8":
        f = {s: "fp16" for s in STAGES}
        for s in ("ln1", "w_qkv", "o", "w_o", "ln2", "w_ffn", "ffn_h"):
            f[s] = "e4m3"
        return f
    raise ValueError(mode)
