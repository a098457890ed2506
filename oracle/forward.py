"""FP64 oracle: the MLPF transformer forward written out step by step.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The architecture follows Sec. 5.3 of the paper (arXiv 2601.17554): PF elements
are embedded by a feed-forward network, processed by a classification (PID)
transformer encoder and a regression encoder, and decoded by two-layer FFN
heads.  Readings of points the paper leaves open (all listed in the design
notes) are marked "reading:" below.

Parity status: every function here is pinned by tests/test_oracle_pins.py
(brute-force attention, closed forms, invariants, an independent torch.nn
float64 model); none is "parity unpinned".
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.special import erf

F64 = np.float64


# ---------------------------------------------------------------- primitives

def layer_norm(x, g, b, eps=1e-5):
    """Layer normalisation over the last axis (pre-LN blocks, Sec. 5.3).

    reading: eps = 1e-5, biased variance.
    """
    x = np.asarray(x, F64)
    mu = x.mean(axis=-1, keepdims=True)
    var = ((x - mu) ** 2).mean(axis=-1, keepdims=True)
    return (x - mu) / np.sqrt(var + eps) * np.asarray(g, F64) + np.asarray(b, F64)


def gelu(x):
    """Exact GELU x * Phi(x), Phi the standard normal CDF written with erf."""
    x = np.asarray(x, F64)
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def relu(x):
    """Rectified linear unit (the paper's activation, Sec. 5.3)."""
    return np.maximum(np.asarray(x, F64), 0.0)


def activation(cfg_act):
    return relu if cfg_act == 1 else gelu


def linear(x, w, b):
    """y = x W^T + b with W stored [out, in]."""
    return np.asarray(x, F64) @ np.asarray(w, F64).T + np.asarray(b, F64)


def softmax_rows(s):
    """Row softmax: positive entries that sum to one per row (Sec. 5.3, Eq. 4).

    A key masked with -inf gets weight exactly zero.
    """
    s = np.asarray(s, F64)
    m = s.max(axis=-1, keepdims=True)
    p = np.exp(s - m)
    return p / p.sum(axis=-1, keepdims=True)


def attention_matrix(q, k, key_mask=None):
    """A = softmax(Q K^T / sqrt(d_k)) (Sec. 5.3, Eq. 4).

    q [N, dk], k [M, dk]; key_mask [M] bool (True = real key) restricts the
    softmax to real keys (padding keys get weight zero); a [N, M] key_mask
    restricts each query row to its own keys (windowed attention).
    """
    q = np.asarray(q, F64)
    k = np.asarray(k, F64)
    s = q @ k.T / math.sqrt(q.shape[-1])
    if key_mask is not None:
        km = np.asarray(key_mask, bool)
        s = np.where(km if km.ndim == 2 else km[None, :], s, -np.inf)
    return softmax_rows(s)


def sdpa(q, k, v, key_mask=None):
    """Scaled dot-product attention A V (Sec. 5.3, Eq. 4; FlashAttention computes
    the same values exactly, Sec. 5.3)."""
    return attention_matrix(q, k, key_mask) @ np.asarray(v, F64)


# ------------------------------------------------------------------- blocks

def multi_head_attention(zn, W, p, heads, key_mask=None):
    """Multi-head self-attention over one event's elements.

    reading: Q, K, V and output projections carry biases; heads split the
    model width into `heads` contiguous slices of d/heads.
    """
    q = linear(zn, W[p + "wq"], W[p + "bq"])
    k = linear(zn, W[p + "wk"], W[p + "bk"])
    v = linear(zn, W[p + "wv"], W[p + "bv"])
    d = q.shape[1]
    dh = d // heads
    o = np.empty_like(q)
    for h in range(heads):
        sl = slice(h * dh, (h + 1) * dh)
        o[:, sl] = sdpa(q[:, sl], k[:, sl], v[:, sl], key_mask)
    return linear(o, W[p + "wo"], W[p + "bo"])


def encoder_block(z, W, p, heads, act, key_mask=None):
    """Pre-LN transformer block (Sec. 5.3): z += MHA(LN1 z); z += FFN(LN2 z)."""
    z = np.asarray(z, F64)
    z = z + multi_head_attention(layer_norm(z, W[p + "ln1.g"], W[p + "ln1.b"]),
                                 W, p, heads, key_mask)
    zn = layer_norm(z, W[p + "ln2.g"], W[p + "ln2.b"])
    hid = act(linear(zn, W[p + "ffn.w1"], W[p + "ffn.b1"]))
    return z + linear(hid, W[p + "ffn.w2"], W[p + "ffn.b2"])


def encoder_stack(z, W, prefix, n_layers, heads, act, key_mask=None):
    """A stack of encoder blocks followed by a final LayerNorm.

    reading: pre-LN stacks end with one LayerNorm (prefix.lnf).
    """
    for l in range(n_layers):
        z = encoder_block(z, W, f"{prefix}.{l}.", heads, act, key_mask)
    return layer_norm(z, W[prefix + ".lnf.g"], W[prefix + ".lnf.b"])


def embed(x, W, act):
    """Element embedding, a two-layer FFN 42 -> d -> d (Sec. 5.3).

    reading: one shared FFN for all element types (the type one-hot is part
    of x); activation between the layers, none after the second.
    """
    return linear(act(linear(x, W["emb.w1"], W["emb.b1"])), W["emb.w2"], W["emb.b2"])


def is_track(x):
    """Element types embedded by the track FFN: track, GSF track, brem (x[:, 0:8]
    is the type one-hot: track, ECAL, HCAL, HF-EM, HF-HAD, GSF track, brem,
    supercluster).

    reading: "tracks and clusters are each embedded" (Sec. 5.3) = one FFN for the
    three track-like types and one for the five calorimeter-cluster types.
    """
    x = np.asarray(x, F64)
    return (x[:, 0] + x[:, 5] + x[:, 6]) > 0.5


def embed_per_type(x, W, act):
    """Per-type embedding (Sec. 5.3 as printed): a two-layer FFN 42 -> d -> d for
    track-like elements (emb.trk) and another for clusters (emb.clu)."""
    x = np.asarray(x, F64)
    e_trk = linear(act(linear(x, W["emb.trk.w1"], W["emb.trk.b1"])), W["emb.trk.w2"], W["emb.trk.b2"])
    e_clu = linear(act(linear(x, W["emb.clu.w1"], W["emb.clu.b1"])), W["emb.clu.w2"], W["emb.clu.b2"])
    return np.where(is_track(x)[:, None], e_trk, e_clu)


def reg_embed(x, h_pid, W, act):
    """Input of the regression encoder: FFN over concat(x, h_pid), (42+d) -> d -> d.

    reading: the regression stack takes the PID stack's (final-normed) output
    concatenated with the raw input features.
    """
    xin = np.concatenate([np.asarray(x, F64), np.asarray(h_pid, F64)], axis=1)
    return linear(act(linear(xin, W["remb.w1"], W["remb.b1"])), W["remb.w2"], W["remb.b2"])


def ffn_head(h, W, name, act):
    """Two-layer FFN output head (Sec. 5.3): d -> d -> k."""
    p = f"head.{name}."
    return linear(act(linear(h, W[p + "w1"], W[p + "b1"])), W[p + "w2"], W[p + "b2"])


# ------------------------------------------------------------------ forward

@dataclasses.dataclass
class OracleOutput:
    logits: np.ndarray      # [T, 6] raw class scores
    raw: np.ndarray         # [T, 5] head outputs (pT', eta, sin, cos, E')
    reg: np.ndarray         # [T, 5] decoded (pT, eta, sin phi, cos phi, E)
    cls: np.ndarray         # [T] argmax class (0 = none)
    sums: np.ndarray        # [n_events, 3] (METx, METy, sum pT)
    h_pid: np.ndarray | None = None
    h_reg: np.ndarray | None = None


def forward_event(W, cfg, x, key_mask=None, keep_hidden=False):
    """Forward of one event: x [N, 42] -> (logits [N, 6], raw [N, 5]).

    Attention runs over this event's elements only (a set; no positional
    encoding, Sec. 5.3).
    """
    act = activation(cfg.act)
    x = np.asarray(x, F64)
    if getattr(cfg, "arch", 0) == 1:
        # Sec. 5.3 as printed: per-type embedding; two parallel encoders on it;
        # binary and multi-class PID heads on the classification encoder
        e = embed_per_type(x, W, act)
        h_pid = encoder_stack(e, W, "pid", cfg.l_pid, cfg.heads, act, key_mask)
        h_reg = encoder_stack(e, W, "reg", cfg.l_reg, cfg.heads, act, key_mask)
        logits = np.concatenate([ffn_head(h_pid, W, "bin", act), ffn_head(h_pid, W, "pid", act)],
                                axis=1)
    else:
        e = embed(x, W, act)
        h_pid = encoder_stack(e, W, "pid", cfg.l_pid, cfg.heads, act, key_mask)
        r = reg_embed(x, h_pid, W, act)
        h_reg = encoder_stack(r, W, "reg", cfg.l_reg, cfg.heads, act, key_mask)
        logits = ffn_head(h_pid, W, "cls", act)
    raw = np.concatenate([ffn_head(h_reg, W, "pt", act), ffn_head(h_reg, W, "eta", act),
                          ffn_head(h_reg, W, "phi", act), ffn_head(h_reg, W, "e", act)],
                         axis=1)
    if keep_hidden:
        return logits, raw, h_pid, h_reg
    return logits, raw


def decode(x, logits, raw, arch=0):
    """Candidates from head outputs (Sec. 5.3, Eq. 2 inverted).

    arch 0: class = argmax of the 6 scores, lowest index on ties (0 = no
    particle).  arch 1 (Sec. 5.3 as printed): a particle where the binary score
    is above 0.5, i.e. its logit (column 0) > 0, with PID = 1 + argmax of the 5
    PID scores (columns 1-5, lowest index on ties); otherwise class 0.
    pT = pT_elem * exp(pT'), E = E_elem * exp(E'), with log pT_elem = x[:, 8]
    and log E_elem = x[:, 9]; eta, sin phi, cos phi as predicted.
    """
    x = np.asarray(x, F64)
    raw = np.asarray(raw, F64)
    lg = np.asarray(logits, F64)
    if arch == 1:
        cls = np.where(lg[:, 0] > 0, 1 + np.argmax(lg[:, 1:], axis=1), 0).astype(np.int32)
    else:
        cls = np.argmax(lg, axis=1).astype(np.int32)
    reg = np.empty_like(raw)
    reg[:, 0] = np.exp(x[:, 8] + raw[:, 0])
    reg[:, 1] = raw[:, 1]
    reg[:, 2] = raw[:, 2]
    reg[:, 3] = raw[:, 3]
    reg[:, 4] = np.exp(x[:, 9] + raw[:, 4])
    return cls, reg


def event_sums(cls, reg, cu_seqlens):
    """Per-event (METx, METy, sum pT) over predicted particles (cls != 0).

    The missing-pT vector is the negative vector pT sum of the candidates
    (Sec. 3.3, uncorrected and unweighted here).  phi enters through
    (sin, cos) normalised by r = sqrt(s^2 + c^2); an element with r = 0 adds
    its pT to the scalar sum but nothing to the vector sum.
    """
    cls = np.asarray(cls)
    reg = np.asarray(reg, F64)
    cu = np.asarray(cu_seqlens, np.int64)
    out = np.zeros((len(cu) - 1, 3), F64)
    for ev in range(len(cu) - 1):
        sl = slice(cu[ev], cu[ev + 1])
        keep = cls[sl] != 0
        pt = reg[sl, 0][keep]
        s = reg[sl, 2][keep]
        c = reg[sl, 3][keep]
        r = np.sqrt(s * s + c * c)
        ok = r > 0
        px = np.where(ok, pt * np.divide(c, r, out=np.zeros_like(c), where=ok), 0.0)
        py = np.where(ok, pt * np.divide(s, r, out=np.zeros_like(s), where=ok), 0.0)
        out[ev, 0] = -px.sum()
        out[ev, 1] = -py.sum()
        out[ev, 2] = pt.sum()
    return out


# ------------------------------------------------------ windowed attention
# The paper names sparse or block attention as a way to cut the inference cost
# (Sec. 9) and suggests partitioning the event before the correlation layers
# (Sec. 5.3).  This variant (not the paper's model) orders each event's elements
# by eta and lets query block b (of WINDOW_BLOCK elements) attend to the keys of
# blocks b - window .. b + window only; window 0 in forward() = full attention.

WINDOW_BLOCK = 128


def eta_order(x):
    """Order of an event's elements by eta (x[:, 10]); ties keep their input order."""
    return np.argsort(np.asarray(x, F64)[:, 10], kind="stable")


def window_mask(n, window, block=WINDOW_BLOCK):
    """[n, n] allowed (query, key) pairs in eta order: |i // block - j // block| <= window."""
    b = np.arange(n) // block
    return np.abs(b[:, None] - b[None, :]) <= window


def forward(W, cfg, x, cu_seqlens, events=None, keep_hidden=False, window=0):
    """Forward over a packed batch; events are independent.

    events: optional list of event indices to evaluate (the others are left
    as NaN rows / NaN sums), for sampled checks of large batches.
    window > 0: windowed attention in eta order (see window_mask); outputs are
    returned in the input order.
    """
    x = np.asarray(x, F64)
    cu = np.asarray(cu_seqlens, np.int64)
    total = int(cu[-1])
    n = len(cu) - 1
    logits = np.full((total, cfg.n_cls), np.nan)
    raw = np.full((total, cfg.n_reg), np.nan)
    hp = np.full((total, cfg.d), np.nan) if keep_hidden else None
    hr = np.full((total, cfg.d), np.nan) if keep_hidden else None
    todo = range(n) if events is None else events
    for ev in todo:
        sl = slice(cu[ev], cu[ev + 1])
        if cu[ev + 1] == cu[ev]:
            continue
        if window > 0:
            xe = x[sl]
            order = eta_order(xe)
            res = forward_event(W, cfg, xe[order], key_mask=window_mask(len(order), window),
                                keep_hidden=keep_hidden)
            inv = np.empty_like(order)
            inv[order] = np.arange(len(order))
            res = tuple(r[inv] for r in res)
        else:
            res = forward_event(W, cfg, x[sl], keep_hidden=keep_hidden)
        logits[sl], raw[sl] = res[0], res[1]
        if keep_hidden:
            hp[sl], hr[sl] = res[2], res[3]
    cls = np.zeros(total, np.int32)
    reg = np.full((total, cfg.n_reg), np.nan)
    done = ~np.isnan(logits[:, 0])
    if done.any():
        c, r = decode(x[done], logits[done], raw[done], getattr(cfg, "arch", 0))
        cls[done] = c
        reg[done] = r
    sums = np.full((n, 3), np.nan)
    for ev in todo:
        sums[ev] = event_sums(cls[cu[ev]:cu[ev + 1]], reg[cu[ev]:cu[ev + 1]],
                              [0, cu[ev + 1] - cu[ev]])[0]
    return OracleOutput(logits=logits, raw=raw, reg=reg, cls=cls, sums=sums,
                        h_pid=hp, h_reg=hr)


# ---------------------------------------------------------- distillation loss

def raw_from_decoded(x, reg):
    """Raw head outputs (pT', eta, sin, cos, E') from decoded ones: the log-ratio
    targets of Eq. 2 with the element's pT and E (x[:, 8], x[:, 9] in log GeV)."""
    x = np.asarray(x, F64)
    reg = np.asarray(reg, F64)
    raw = reg.copy()
    raw[:, 0] = np.log(reg[:, 0]) - x[:, 8]
    raw[:, 4] = np.log(reg[:, 4]) - x[:, 9]
    return raw


def log_softmax_rows(s):
    s = np.asarray(s, F64)
    m = s.max(axis=-1, keepdims=True)
    return s - m - np.log(np.exp(s - m).sum(axis=-1, keepdims=True))


def distill_loss(W, cfg, x, cu_seqlens, t_logits, t_reg):
    """Distillation loss of a student with weights W on a teacher's outputs.

    reading: mean over elements of KL(p_teacher || p_student) over the classes
    plus the squared error of the five raw regression outputs (the regression
    part of the paper's loss, Eq. 3, with unit weights), the teacher's raw
    outputs recovered from its decoded ones (Eq. 2).
    """
    out = forward(W, cfg, x, cu_seqlens)
    lt = log_softmax_rows(t_logits)
    ls = log_softmax_rows(out.logits)
    kl = (np.exp(lt) * (lt - ls)).sum(axis=1)
    mse = ((out.raw - raw_from_decoded(x, t_reg)) ** 2).sum(axis=1)
    return float((kl + mse).mean())


# ------------------------------------------------------- supervised loss (Eq. 1)

# readings of the points the paper leaves open:
SUP_BETA = 0.01      # weight of the binary term: the later, more specific value (Sec. 5.3)
SUP_FOCAL = 2.0      # focusing parameter of the focal loss (unstated; the value of Lin et al.)
SUP_DELTA = 1.0      # weight of the angular regression terms (unstated)


def softplus(z):
    z = np.asarray(z, F64)
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def supervised_loss(x, logits, raw, cls_target, reg_target, beta=SUP_BETA, focal=SUP_FOCAL,
                    delta=SUP_DELTA):
    """Per-element loss of Eq. 1 for the printed architecture, averaged over elements.

    logits [T, 6]: binary logit, then the 5 PID logits; raw [T, 5]: (pT', eta, sin phi,
    cos phi, E'); cls_target [T]: 0 = no target particle, k = 1..5 = particle of PID
    class k; reg_target [T, 5]: the target particle's (pT, eta, sin phi, cos phi, E).

      L_i = beta BCE(b_i, sigmoid(z_i))
            + b_i [ FL(k_i) + g_i (dpT'^2 + dE'^2) + delta (deta^2 + dsin^2 + dcos^2) ]
    b_i = [cls_target > 0]; BCE = softplus(z) - b z; the focal loss (Lin et al. 2017)
    FL = -(1 - p_t)^focal log p_t with p_t the PID softmax probability of the target
    class; pT' and E' targets from Eq. 2 (log of the target over the element's value);
    g_i = sqrt(pT target) (Sec. 5.3).

    reading: the PID and regression terms apply to elements that have a target
    particle only; the sum over elements is divided by their number.
    """
    x = np.asarray(x, F64)
    lg = np.asarray(logits, F64)
    raw = np.asarray(raw, F64)
    k = np.asarray(cls_target, np.int64)
    b = (k > 0).astype(F64)
    z = lg[:, 0]
    bce = softplus(z) - b * z
    lp = log_softmax_rows(lg[:, 1:])
    kk = np.clip(k - 1, 0, 4)
    logpt = lp[np.arange(len(k)), kk]
    fl = -((1.0 - np.exp(logpt)) ** focal) * logpt
    reg_target = np.asarray(reg_target, F64)
    ok = k > 0
    rt = np.zeros_like(raw)
    rt[ok] = raw_from_decoded(x[ok], reg_target[ok])
    g = np.sqrt(np.where(ok, reg_target[:, 0], 1.0))
    d2 = (raw - rt) ** 2
    lreg = g * (d2[:, 0] + d2[:, 4]) + delta * (d2[:, 1] + d2[:, 2] + d2[:, 3])
    per = beta * bce + b * (fl + lreg)
    return float(per.mean())
