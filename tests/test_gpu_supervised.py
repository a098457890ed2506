"""Supervised training step (loss of Eq. 1) of the printed architecture on the
hand-written FP32 backward kernels.

The loss matches the FP64 oracle's supervised_loss of the oracle's forward;
gradients match central finite differences of that loss for two entries of every
parameter tensor (both embeddings, both encoders, the binary and PID heads and the
regression heads); training on synthetic targets lowers the loss.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TINY_P = synth.ModelConfig(d=32, heads=2, ffn=64, l_pid=1, l_reg=1, act=1, arch=synth.ARCH_PAPER)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def sup_loss(W, x, cu, cls_t, reg_t):
    out = oracle.forward(W, TINY_P, x, cu)
    return oracle.supervised_loss(x, out.logits, out.raw, cls_t, reg_t)


@pytest.fixture(scope="module")
def case():
    from paper_2601_17554_b300 import Trainer
    W = synth.make_weights(TINY_P, 9, perturbed=True)
    x, cu = synth.gen_events(61, [13, 29, 1])
    cls_t, reg_t = synth.gen_targets(62, x, cu)
    assert (cls_t == 0).any() and (cls_t > 0).any()
    tr = Trainer(synth.pack_blob(TINY_P, W))
    g = torch.zeros(tr.num_params, dtype=torch.float32, device="cuda")
    loss = tr.step_supervised(dev(x), dev(cu), 29, dev(cls_t), dev(reg_t), lr=0.0, update=False, grads=g)
    tr.close()
    G, off = {}, 0
    gv = g.cpu().numpy().astype(np.float64)
    for name, shape, _ in synth.tensor_specs(TINY_P):
        n = int(np.prod(shape))
        G[name] = gv[off:off + n].reshape(shape)
        off += n
    return W, x, cu, cls_t, reg_t, loss, G


def test_supervised_loss_matches_oracle(case):
    W, x, cu, cls_t, reg_t, loss, _ = case
    ref = sup_loss(W, x, cu, cls_t, reg_t)
    assert abs(loss - ref) <= 1e-5 * max(1.0, abs(ref)), (loss, ref)


def test_supervised_gradients_match_finite_differences(case):
    W, x, cu, cls_t, reg_t, loss, G = case
    rng = np.random.default_rng(1)
    Wd = {k: v.astype(np.float64) for k, v in W.items()}
    gmax = max(np.abs(v).max() for v in G.values())
    for name, shape, _ in synth.tensor_specs(TINY_P):
        for _ in range(2):
            idx = tuple(int(rng.integers(s)) for s in shape)
            w0 = Wd[name][idx]
            h = 1e-6 * max(1.0, abs(w0))
            Wd[name][idx] = w0 + h
            lp = sup_loss(Wd, x, cu, cls_t, reg_t)
            Wd[name][idx] = w0 - h
            lm = sup_loss(Wd, x, cu, cls_t, reg_t)
            Wd[name][idx] = w0
            fd = (lp - lm) / (2 * h)
            g = G[name][idx]
            assert abs(g - fd) <= 2e-3 * abs(fd) + 2e-5 * gmax, (name, idx, g, fd)
    # both embeddings and both heads receive gradient
    for name in ("emb.trk.w1", "emb.clu.w1", "head.bin.w2", "head.pid.w2", "pid.0.wq", "reg.0.wq"):
        assert np.abs(G[name]).max() > 0, name


def test_supervised_training_lowers_loss():
    from paper_2601_17554_b300 import Model, Trainer
    W = synth.make_weights(TINY_P, 10)
    tr = Trainer(synth.pack_blob(TINY_P, W))
    x, cu = synth.gen_events(63, [400, 300, 500, 200])
    cls_t, reg_t = synth.gen_targets(64, x, cu)
    X, CU, C, R = dev(x), dev(cu), dev(cls_t), dev(reg_t)
    first = tr.step_supervised(X, CU, 500, C, R, lr=0.0, update=False)
    for i in range(60):
        tr.step_supervised(X, CU, 500, C, R, lr=2e-3, update=True, want_loss=False)
    last = tr.step_supervised(X, CU, 500, C, R, lr=0.0, update=False)
    assert last < 0.6 * first, (first, last)
    # the exported blob loads as an arch-1 model whose forward gives that loss
    blob = tr.export()
    tr.close()
    m = Model(blob)
    assert m.config["arch"] == 1
    lo, rg, cl, su = m.forward(X, CU, 500, precision="fp32")
    m.sync()
    raw = oracle.raw_from_decoded(x, rg.cpu().numpy())
    ref = oracle.supervised_loss(x, lo.cpu().numpy(), raw, cls_t, reg_t)
    assert abs(ref - last) <= 1e-3 * last, (ref, last)


def test_supervised_step_rejects_arch0():
    from paper_2601_17554_b300 import MlpfError, Trainer
    cfg = synth.ModelConfig(d=32, heads=2, ffn=64, l_pid=1, l_reg=1)
    tr = Trainer(synth.pack_blob(cfg, synth.make_weights(cfg, 1)))
    x, cu = synth.gen_events(65, [10])
    cls_t, reg_t = synth.gen_targets(66, x, cu)
    with pytest.raises(MlpfError) as ei:
        tr.step_supervised(dev(x), dev(cu), 10, dev(cls_t), dev(reg_t), lr=0.0, update=False)
    assert ei.value.status == 7
    tr.close()
