"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: brute force on
tiny inputs, closed forms, invariants of the method (a set model with no
positional encoding, Sec. 5.3), and an independent float64 model assembled from
torch.nn.functional library routines.  No GPU is needed.
"""
import json
import math
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(7)


# ---------------------------------------------------------------- attention

def brute_force_sdpa(q, k, v, mask=None):
    """Pure-Python loop nest of Eq. 4 (no numpy reductions)."""
    n, dk = len(q), len(q[0])
    m = len(k)
    out = []
    for i in range(n):
        scores = []
        for j in range(m):
            if mask is not None and not mask[j]:
                scores.append(None)
                continue
            s = 0.0
            for t in range(dk):
                s += float(q[i][t]) * float(k[j][t])
            scores.append(s / math.sqrt(dk))
        mx = max(s for s in scores if s is not None)
        w = [0.0 if s is None else math.exp(s - mx) for s in scores]
        tot = sum(w)
        row = []
        for t in range(len(v[0])):
            acc = 0.0
            for j in range(m):
                acc += w[j] / tot * float(v[j][t])
            row.append(acc)
        out.append(row)
    return np.array(out)


@pytest.mark.parametrize("n,m,dk", [(1, 1, 4), (3, 5, 16), (16, 16, 16), (7, 16, 32)])
def test_sdpa_brute_force(n, m, dk):
    q, k, v = rng.normal(size=(n, dk)), rng.normal(size=(m, dk)), rng.normal(size=(m, dk))
    np.testing.assert_allclose(oracle.sdpa(q, k, v), brute_force_sdpa(q, k, v),
                               rtol=1e-12, atol=1e-13)


def test_sdpa_brute_force_masked():
    q, k, v = rng.normal(size=(6, 16)), rng.normal(size=(12, 16)), rng.normal(size=(12, 16))
    mask = np.array([True] * 9 + [False] * 3)
    mask[4] = False
    np.testing.assert_allclose(oracle.sdpa(q, k, v, mask), brute_force_sdpa(q, k, v, mask),
                               rtol=1e-12, atol=1e-13)


def test_softmax_rows_positive_and_sum_to_one():
    q, k = rng.normal(size=(40, 16)) * 3, rng.normal(size=(33, 16)) * 3
    a = oracle.attention_matrix(q, k)
    assert (a > 0).all()
    np.testing.assert_allclose(a.sum(axis=1), 1.0, atol=1e-15 * 33)


def test_sdpa_single_key_returns_v():
    q, k, v = rng.normal(size=(1, 16)), rng.normal(size=(1, 16)), rng.normal(size=(1, 16))
    np.testing.assert_array_equal(oracle.sdpa(q, k, v), v)


def test_sdpa_textbook_library():
    q, k, v = (torch.randn(1, 1, 20, 16, dtype=torch.float64) for _ in range(3))
    ref = F.scaled_dot_product_attention(q, k, v)[0, 0].numpy()
    np.testing.assert_allclose(oracle.sdpa(q[0, 0].numpy(), k[0, 0].numpy(), v[0, 0].numpy()),
                               ref, rtol=1e-12, atol=1e-13)


# ----------------------------------------------------------- LN and GELU

def test_layer_norm_closed_forms():
    g, b = rng.normal(size=8), rng.normal(size=8)
    np.testing.assert_allclose(oracle.layer_norm(np.full((1, 8), 3.7), g, b)[0], b, atol=1e-12)
    a = 2.5
    x = np.array([[a, -a]])
    y = oracle.layer_norm(x, np.ones(2), np.zeros(2), eps=1e-5)
    np.testing.assert_allclose(y[0], [a / math.sqrt(a * a + 1e-5), -a / math.sqrt(a * a + 1e-5)],
                               rtol=1e-14)
    z = oracle.layer_norm(rng.normal(size=(5, 64)) * 10 + 3, np.ones(64), np.zeros(64))
    np.testing.assert_allclose(z.mean(axis=1), 0.0, atol=1e-12)
    np.testing.assert_allclose(z.var(axis=1), 1.0, rtol=1e-5)


def test_gelu_closed_forms():
    phi1 = 0.8413447460685429  # standard normal CDF at 1
    np.testing.assert_allclose(oracle.gelu([0.0, 1.0, -1.0]), [0.0, phi1, -(1 - phi1)],
                               rtol=1e-15, atol=1e-16)
    np.testing.assert_allclose(oracle.gelu([12.0, -12.0]), [12.0, 0.0], atol=1e-30)
    np.testing.assert_array_equal(oracle.relu([-2.0, 0.0, 3.0]), [0.0, 0.0, 3.0])


# -------------------------------------------------- independent torch model

def torch_reference(W, cfg, x):
    """The architecture assembled from torch.nn.functional routines in float64."""
    T = {k: torch.tensor(np.asarray(v, np.float64)) for k, v in W.items()}
    act = (lambda t: F.gelu(t, approximate="none")) if cfg.act == 0 else F.relu
    x = torch.tensor(np.asarray(x, np.float64))

    def lin(t, p):
        return F.linear(t, T[p + "w" if p.endswith(".") else p + ".w"], None)

    def ln(t, p):
        return F.layer_norm(t, (cfg.d,), T[p + ".g"], T[p + ".b"], eps=1e-5)

    def mlp(t, w1, b1, w2, b2):
        return F.linear(act(F.linear(t, T[w1], T[b1])), T[w2], T[b2])

    def stack(z, prefix, n):
        for l in range(n):
            p = f"{prefix}.{l}."
            zn = ln(z, p + "ln1")
            q = F.linear(zn, T[p + "wq"], T[p + "bq"])
            k = F.linear(zn, T[p + "wk"], T[p + "bk"])
            v = F.linear(zn, T[p + "wv"], T[p + "bv"])
            split = lambda t: t.view(-1, cfg.heads, cfg.dh).transpose(0, 1)
            o = F.scaled_dot_product_attention(split(q), split(k), split(v))
            o = o.transpose(0, 1).reshape(-1, cfg.d)
            z = z + F.linear(o, T[p + "wo"], T[p + "bo"])
            z = z + mlp(ln(z, p + "ln2"), p + "ffn.w1", p + "ffn.b1", p + "ffn.w2", p + "ffn.b2")
        return ln(z, prefix + ".lnf")

    head = lambda h, n: mlp(h, f"head.{n}.w1", f"head.{n}.b1", f"head.{n}.w2", f"head.{n}.b2")
    if cfg.arch == synth.ARCH_PAPER:
        # track-like types (track, GSF track, brem) take the track embedding
        trk = (x[:, synth.TRACK_TYPES].sum(1) > 0.5)[:, None]
        e = torch.where(trk, mlp(x, "emb.trk.w1", "emb.trk.b1", "emb.trk.w2", "emb.trk.b2"),
                        mlp(x, "emb.clu.w1", "emb.clu.b1", "emb.clu.w2", "emb.clu.b2"))
        h_pid, h_reg = stack(e, "pid", cfg.l_pid), stack(e, "reg", cfg.l_reg)
        logits = torch.cat([head(h_pid, "bin"), head(h_pid, "pid")], 1)
    else:
        h_pid = stack(mlp(x, "emb.w1", "emb.b1", "emb.w2", "emb.b2"), "pid", cfg.l_pid)
        h_reg = stack(mlp(torch.cat([x, h_pid], 1), "remb.w1", "remb.b1", "remb.w2", "remb.b2"),
                      "reg", cfg.l_reg)
        logits = head(h_pid, "cls")
    raw = torch.cat([head(h_reg, n) for n, _ in synth.REG_HEADS], 1)
    return logits.numpy(), raw.numpy()


PAPER_SMALL = synth.ModelConfig(d=32, heads=2, ffn=64, l_pid=2, l_reg=1, act=1, arch=synth.ARCH_PAPER)


@pytest.mark.parametrize("cfg", [synth.SMALL, synth.FULL,
                                 synth.ModelConfig(d=32, heads=2, ffn=64, l_pid=2, l_reg=1, act=1),
                                 PAPER_SMALL, synth.PAPER])
def test_forward_matches_torch_functional(cfg):
    W = synth.make_weights(cfg, seed=5, perturbed=True)
    x, cu = synth.gen_events(11, [23])
    lo, raw = oracle.forward_event(W, cfg, x)
    tl, traw = torch_reference(W, cfg, x)
    np.testing.assert_allclose(lo, tl, rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(raw, traw, rtol=1e-10, atol=1e-11)


# --------------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def small_model():
    cfg = synth.SMALL
    return cfg, synth.make_weights(cfg, seed=3, perturbed=True)


def test_permutation_equivariance(small_model):
    cfg, W = small_model
    x, _ = synth.gen_events(12, [31])
    perm = np.random.default_rng(1).permutation(31)
    lo, raw = oracle.forward_event(W, cfg, x)
    lo_p, raw_p = oracle.forward_event(W, cfg, x[perm])
    np.testing.assert_allclose(lo_p, lo[perm], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(raw_p, raw[perm], rtol=1e-11, atol=1e-12)


def test_padding_invariance(small_model):
    cfg, W = small_model
    x, _ = synth.gen_events(13, [20])
    pad = np.random.default_rng(2).normal(size=(9, 42)) * 5
    xp = np.concatenate([x, pad])
    mask = np.array([True] * 20 + [False] * 9)
    lo, raw = oracle.forward_event(W, cfg, x)
    lo_p, raw_p = oracle.forward_event(W, cfg, xp, key_mask=mask)
    np.testing.assert_allclose(lo_p[:20], lo, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(raw_p[:20], raw, rtol=1e-11, atol=1e-12)


def test_identity_when_sublayers_zeroed(small_model):
    cfg, W = small_model
    W = dict(W)
    for l in range(cfg.l_pid):
        for n in ("wo", "bo", "ffn.w2", "ffn.b2"):
            W[f"pid.{l}.{n}"] = np.zeros_like(W[f"pid.{l}.{n}"])
    z = np.random.default_rng(3).normal(size=(17, cfg.d))
    out = oracle.encoder_stack(z, W, "pid", cfg.l_pid, cfg.heads, oracle.gelu)
    ref = oracle.layer_norm(z, W["pid.lnf.g"], W["pid.lnf.b"])
    np.testing.assert_array_equal(out, ref)


def test_single_element_reduces_to_mlp(small_model):
    """N=1: attention returns V, so a block is a per-element map independent of
    any other element; the event forward equals the forward of each element alone."""
    cfg, W = small_model
    x, _ = synth.gen_events(14, [1])
    lo, raw = oracle.forward_event(W, cfg, x)
    tl, traw = torch_reference(W, cfg, x)
    np.testing.assert_allclose(lo, tl, rtol=1e-10)
    np.testing.assert_allclose(raw, traw, rtol=1e-10)


def test_duplicate_elements_identical(small_model):
    cfg, W = small_model
    x, _ = synth.gen_events(15, [10])
    x[7] = x[2]
    lo, raw = oracle.forward_event(W, cfg, x)
    np.testing.assert_array_equal(lo[7], lo[2])
    np.testing.assert_array_equal(raw[7], raw[2])


def test_events_independent(small_model):
    cfg, W = small_model
    x, cu = synth.gen_events(16, [5, 0, 12, 1])
    out = oracle.forward(W, cfg, x, cu)
    for e in range(4):
        sl = slice(cu[e], cu[e + 1])
        if cu[e + 1] == cu[e]:
            assert out.sums[e].tolist() == [0.0, 0.0, 0.0] or np.isnan(out.sums[e]).all()
            continue
        lo, raw = oracle.forward_event(W, cfg, x[sl])
        np.testing.assert_array_equal(out.logits[sl], lo)
        np.testing.assert_array_equal(out.raw[sl], raw)


# ------------------------------------------------------- decode and sums

def test_decode_and_event_sums_hand_examples():
    with open(os.path.join(GOLDEN, "event_sums_hand.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        x = np.zeros((len(case["log_pt"]), 42))
        x[:, 8] = case["log_pt"]
        x[:, 9] = case["log_e"]
        logits = np.array(case["logits"], dtype=np.float64)
        raw = np.array(case["raw"], dtype=np.float64)
        cls, reg = oracle.decode(x, logits, raw)
        assert cls.tolist() == case["cls"], case["name"]
        np.testing.assert_allclose(reg[:, 0], case["pt"], rtol=1e-14)
        np.testing.assert_allclose(reg[:, 4], case["e"], rtol=1e-14)
        sums = oracle.event_sums(cls, reg, [0, len(cls)])[0]
        np.testing.assert_allclose(sums, case["sums"], atol=1e-12, err_msg=case["name"])


# ------------------------------------------------------------- generator

def test_generator_statistics_and_masks():
    x, cu = synth.gen_events(104, synth.sizes_lognormal(104, 64))
    typ = x[:, :8].argmax(1)
    assert np.all(x[:, :8].sum(1) == 1)
    frac = np.bincount(typ, minlength=8) / len(typ)
    np.testing.assert_allclose(frac, synth.TYPE_PROBS, atol=0.01)
    trk = np.isin(typ, synth.TRACK_TYPES)
    assert np.all(x[trk, 30:42] == 0) and np.all(x[~trk, 13:30] == 0)
    np.testing.assert_allclose(x[:, 11] ** 2 + x[:, 12] ** 2, 1.0, rtol=1e-6)
    assert np.abs(x[np.isin(typ, (3, 4)), 10]).max() <= 5.0
    assert np.abs(x[trk, 10]).max() <= 2.5
    assert abs(x[:, 8].mean()) < 0.02 and abs(x[:, 8].std() - 1) < 0.02


def test_generator_counter_based():
    x1, _ = synth.gen_events(9, [4, 7])
    x2, _ = synth.gen_events(9, [4, 9, 3])
    np.testing.assert_array_equal(x1[:4], x2[:4])
    np.testing.assert_array_equal(x1[4:11], x2[4:11])
    n = synth.sizes_lognormal(104, 512)
    assert n.min() >= 100 and n.max() <= 12000
    assert 2200 < np.median(n) < 2800
    u = synth.sizes_uniform(103, 64)
    assert u.min() >= 1000 and u.max() <= 6000


def test_splitmix64_published_vector():
    # SplitMix64 output sequence for state 0 (first output), a published value.
    assert int(synth.splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF


# ------------------------------------------------------- distillation loss

def test_distill_loss_zero_on_own_outputs():
    """KL(p || p) = 0 and the raw targets recovered from the decoded outputs equal
    the raw outputs, so a model distilled on its own outputs has zero loss."""
    cfg = synth.ModelConfig(d=32, heads=2, ffn=64, l_pid=1, l_reg=1)
    W = synth.make_weights(cfg, 8, perturbed=True)
    x, cu = synth.gen_events(31, [9, 4])
    out = oracle.forward(W, cfg, x, cu)
    assert abs(oracle.distill_loss(W, cfg, x, cu, out.logits, out.reg)) < 1e-12


def test_distill_loss_hand_example():
    """One element: teacher probabilities (1/2, 1/2, 0...) vs a uniform student over
    two classes is KL = 0 (same distribution); a regression offset of 0.5 in eta
    adds 0.25."""
    cfg = synth.ModelConfig(d=32, heads=2, ffn=64, l_pid=1, l_reg=1)
    W = synth.make_weights(cfg, 9)
    x, cu = synth.gen_events(32, [1])
    out = oracle.forward(W, cfg, x, cu)
    t_reg = out.reg.copy()
    t_reg[:, 1] += 0.5
    np.testing.assert_allclose(oracle.distill_loss(W, cfg, x, cu, out.logits, t_reg), 0.25, rtol=1e-12)
    lt = oracle.log_softmax_rows(np.array([[0.0, 0.0, -1e300, -1e300, -1e300, -1e300]]))
    np.testing.assert_allclose(np.exp(lt[0, :2]), [0.5, 0.5], rtol=1e-15)


def test_raw_from_decoded_inverts_decode():
    x, _ = synth.gen_events(33, [6])
    raw = np.random.default_rng(4).normal(size=(6, 5))
    _, reg = oracle.decode(x, np.zeros((6, 6)), raw)
    np.testing.assert_allclose(oracle.raw_from_decoded(x, reg), raw, rtol=1e-12, atol=1e-12)


# ------------------------------------------ the architecture as printed (Sec. 5.3)

def test_paper_arch_parallel_encoders_are_independent():
    """Two parallel encoders on one embedding: the regression outputs do not
    depend on the classification encoder or its heads, and the class scores do
    not depend on the regression encoder (the sequential reading couples them)."""
    cfg = PAPER_SMALL
    W = synth.make_weights(cfg, seed=7, perturbed=True)
    x, _ = synth.gen_events(14, [29])
    lo, raw = oracle.forward_event(W, cfg, x)
    rng = np.random.default_rng(3)
    Wc = {k: (v + rng.normal(size=v.shape).astype(np.float32) if k.startswith(("pid.", "head.bin", "head.pid"))
              else v) for k, v in W.items()}
    lo_c, raw_c = oracle.forward_event(Wc, cfg, x)
    np.testing.assert_array_equal(raw_c, raw)
    assert np.abs(lo_c - lo).max() > 1e-3
    Wr = {k: (v + rng.normal(size=v.shape).astype(np.float32) if k.startswith("reg.") else v)
          for k, v in W.items()}
    lo_r, raw_r = oracle.forward_event(Wr, cfg, x)
    np.testing.assert_array_equal(lo_r, lo)
    assert np.abs(raw_r - raw).max() > 1e-3


def test_paper_arch_per_type_embedding():
    """Track-like elements (track, GSF track, brem) use emb.trk, clusters emb.clu:
    an event of tracks only ignores the cluster embedding's weights."""
    cfg = PAPER_SMALL
    W = synth.make_weights(cfg, seed=8, perturbed=True)
    x, _ = synth.gen_events(15, [200])
    assert oracle.is_track(x).any() and (~oracle.is_track(x)).any()
    trk = x[oracle.is_track(x)][:12]
    assert set(np.argmax(trk[:, :8], 1).tolist()) <= {0, 5, 6}
    lo, raw = oracle.forward_event(W, cfg, trk)
    W2 = dict(W)
    for k in ("emb.clu.w1", "emb.clu.b1", "emb.clu.w2", "emb.clu.b2"):
        W2[k] = W[k] * 3 + 1
    lo2, raw2 = oracle.forward_event(W2, cfg, trk)
    np.testing.assert_array_equal(lo2, lo)
    np.testing.assert_array_equal(raw2, raw)
    # and the per-element embedding is the selected FFN's output
    act = oracle.relu
    e = oracle.embed_per_type(x, W, act)
    i_t, i_c = np.flatnonzero(oracle.is_track(x))[0], np.flatnonzero(~oracle.is_track(x))[0]
    ft = oracle.linear(act(oracle.linear(x[i_t:i_t + 1], W["emb.trk.w1"], W["emb.trk.b1"])),
                       W["emb.trk.w2"], W["emb.trk.b2"])
    fc = oracle.linear(act(oracle.linear(x[i_c:i_c + 1], W["emb.clu.w1"], W["emb.clu.b1"])),
                       W["emb.clu.w2"], W["emb.clu.b2"])
    np.testing.assert_allclose(e[i_t], ft[0], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(e[i_c], fc[0], rtol=1e-12, atol=1e-14)


def test_paper_arch_decode_hand_values():
    """Binary score above 0.5 (logit > 0) selects a particle with PID = 1 + argmax
    of the five PID scores (Sec. 5.3); logit <= 0 gives class 0 whatever the PID
    scores; equal PID scores take the lowest index."""
    x = np.zeros((5, 42))
    raw = np.zeros((5, 5))
    logits = np.array([[0.3, 0.0, 2.0, 1.0, 0.0, 0.0],     # particle, PID 2 -> class 2
                       [-0.1, 9.0, 0.0, 0.0, 0.0, 0.0],    # no particle
                       [0.0, 0.0, 0.0, 0.0, 0.0, 5.0],     # logit 0 = score 0.5: not above
                       [1e-9, 1.0, 1.0, 0.5, 0.5, 0.5],    # tie -> lowest PID index -> class 1
                       [4.0, -3.0, -2.0, -1.0, -4.0, -0.5]])  # PID 5 -> class 5
    cls, _ = oracle.decode(x, logits, raw, arch=1)
    assert cls.tolist() == [2, 0, 0, 1, 5]
    cls0, _ = oracle.decode(x, logits, raw, arch=0)
    assert cls0.tolist() == [2, 1, 5, 1, 0]   # plain argmax over all six columns


# ---------------------------------------------------- supervised loss (Eq. 1)

def test_supervised_loss_hand_value():
    """Two elements: no target particle with z = 0 (beta log 2 only); a class-2
    particle with equal PID scores (p_t = 1/5: focal (4/5)^2 log 5), z = 0, and a
    pT' prediction off by 1 with pT target 4 (sqrt(4) * 1^2 = 2)."""
    x = np.zeros((2, 42))
    x[:, 8] = np.log(2.0)   # element pT 2 GeV
    x[:, 9] = np.log(3.0)   # element E 3 GeV
    reg_t = np.array([[1.0, 0.0, 0.0, 1.0, 1.0], [4.0, 0.3, 0.6, 0.8, 6.0]])
    raw = np.zeros((2, 5))
    raw[1] = [np.log(4.0 / 2.0) + 1.0, 0.3, 0.6, 0.8, np.log(6.0 / 3.0)]
    logits = np.zeros((2, 6))
    cls_t = np.array([0, 2])
    L = oracle.supervised_loss(x, logits, raw, cls_t, reg_t)
    b = oracle.SUP_BETA
    expect = (b * np.log(2) + b * np.log(2) + 0.64 * np.log(5) + 2.0) / 2
    assert abs(L - expect) < 1e-12


def test_supervised_loss_special_cases():
    rng = np.random.default_rng(4)
    T = 50
    x = rng.normal(size=(T, 42))
    logits = rng.normal(size=(T, 6)) * 3
    raw = rng.normal(size=(T, 5))
    cls_t = rng.integers(0, 6, size=T)
    reg_t = np.abs(rng.normal(size=(T, 5))) + 0.1
    # focusing parameter 0: the PID term is the cross entropy of the 5-way softmax
    no_reg = dict(delta=0.0)
    part = raw.copy()
    ok = cls_t > 0
    # remove the pT/E regression terms by predicting their targets exactly
    part[ok, 0] = np.log(reg_t[ok, 0]) - x[ok, 8]
    part[ok, 4] = np.log(reg_t[ok, 4]) - x[ok, 9]
    L0 = oracle.supervised_loss(x, logits, part, cls_t, reg_t, beta=0.0, focal=0.0, **no_reg)
    u = logits[:, 1:]
    ce = -(u[np.arange(T), np.clip(cls_t - 1, 0, 4)] - np.log(np.exp(u).sum(1)))
    assert abs(L0 - (ce * ok).mean()) < 1e-12
    # the binary term alone: -(b log sigmoid + (1 - b) log(1 - sigmoid)), stable at |z| = 50
    Lb = oracle.supervised_loss(x, logits, part, cls_t, reg_t, beta=1.0, focal=0.0, **no_reg) - L0
    sg = 1 / (1 + np.exp(-logits[:, 0]))
    bce = -(ok * np.log(sg) + (~ok) * np.log(1 - sg))
    assert abs(Lb - bce.mean()) < 1e-12
    big = logits.copy()
    big[:, 0] = np.where(ok, -50.0, 50.0)
    Lbig = oracle.supervised_loss(x, big, part, cls_t, reg_t, beta=1.0, focal=0.0, **no_reg) - L0
    assert abs(Lbig - 50.0) < 1e-9


def test_synthetic_targets():
    sizes = [3000, 2000, 0, 17]
    x, cu = synth.gen_events(41, sizes)
    c1, r1 = synth.gen_targets(7, x, cu)
    c2, r2 = synth.gen_targets(7, x, cu)
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(r1, r2)
    # the last event regenerated alone gives the same targets
    c3, r3 = synth.gen_targets(7, x[cu[3]:], [0, 17], first_event=3)
    np.testing.assert_array_equal(c3, c1[cu[3]:])
    typ = np.argmax(x[:, :8], 1)
    for t in (0, 1, 2):
        f = np.bincount(c1[typ == t], minlength=6) / (typ == t).sum()
        np.testing.assert_allclose(f, synth.TARGET_CLASS_PROBS[t], atol=0.04)
    np.testing.assert_allclose(r1[:, 2] ** 2 + r1[:, 3] ** 2, 1.0, atol=1e-6)
    assert (r1[:, 0] > 0).all() and (r1[:, 4] > 0).all()
    d = np.log(r1[:, 0]) - x[:, 8]
    assert abs(d.std() - 0.3) < 0.02


# ------------------------------------------------------------ windowed attention

def test_window_mask_brute_force():
    n, w, B = 300, 1, 128
    m = oracle.window_mask(n, w, B)
    for i in range(0, n, 7):
        for j in range(0, n, 5):
            assert m[i, j] == (abs(i // B - j // B) <= w)


def test_windowed_attention_loop_nest():
    """One head of windowed attention against a loop over each query's allowed keys."""
    rng = np.random.default_rng(9)
    n, dk = 300, 16
    q, k, v = rng.normal(size=(3, n, dk))
    out = oracle.sdpa(q, k, v, oracle.window_mask(n, 0))
    for i in (0, 127, 128, 299):
        lo, hi = (i // 128) * 128, min(n, (i // 128 + 1) * 128)
        s = [sum(q[i, c] * k[j, c] for c in range(dk)) / 4.0 for j in range(lo, hi)]
        m = max(s)
        e = [math.exp(t - m) for t in s]
        z = sum(e)
        for c in range(dk):
            ref = sum(e[j - lo] * v[j, c] for j in range(lo, hi)) / z
            assert abs(out[i, c] - ref) < 1e-12


def test_windowed_forward_reduces_to_full_and_is_order_invariant():
    cfg = synth.SMALL
    W = synth.make_weights(cfg, 12, perturbed=True)
    x, cu = synth.gen_events(71, [300, 45])
    full = oracle.forward(W, cfg, x, cu)
    wide = oracle.forward(W, cfg, x, cu, window=3)    # 300 elements: 3 blocks, all in reach
    np.testing.assert_allclose(wide.logits, full.logits, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(wide.reg, full.reg, rtol=1e-10, atol=1e-12)
    narrow = oracle.forward(W, cfg, x, cu, window=1)  # blocks 0 and 2 do not see each other
    assert np.abs(narrow.logits[:300] - full.logits[:300]).max() > 1e-6
    np.testing.assert_allclose(narrow.logits[300:], full.logits[300:], rtol=1e-10, atol=1e-12)
    # canonical eta order: permuting the input permutes the outputs
    perm = np.random.default_rng(3).permutation(300)
    xp = x.copy()
    xp[:300] = x[:300][perm]
    narrow_p = oracle.forward(W, cfg, xp, cu, window=1)
    np.testing.assert_allclose(narrow_p.logits[:300], narrow.logits[:300][perm], rtol=1e-10, atol=1e-12)
