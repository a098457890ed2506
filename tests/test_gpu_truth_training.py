"""Training the full pipeline on a learnable task (GPU).

The library's BF16 trainer (tcgen05 GEMMs, warp-level MMA attention, LAMB) fits
the deterministic synthetic truth of synth.gen_pf_truth: a d=64, 1 + 1 model
trained on it from random weights classifies held-out events far better than the
same model untrained, and better than its element type alone allows (the truth's
muon and cluster rules depend on the element's features and on its event).  This
is the task the distillation driver trains the full model on before distilling
its students from it.
"""
import math

import numpy as np
import pytest
import torch

import synth
from tests.util import run_gpu

pytestmark = pytest.mark.gpu

TRUTH_LOGIT = 6.0


def _type_only_accuracy(x, cls):
    """Accuracy of the best rule that looks at the element type alone (the most
    frequent true class of each type)."""
    typ = np.argmax(x[:, :8], axis=1)
    hit = 0
    for t in range(8):
        c = cls[typ == t]
        if len(c):
            hit += np.bincount(c, minlength=6).max()
    return hit / len(cls)


def test_trained_model_learns_the_synthetic_truth():
    from paper_2601_17554_b300 import Model, Trainer
    cfg = synth.SMALL
    init = synth.pack_blob(cfg, synth.make_weights(cfg, 0))
    # 16 training batches of 8 events (N ~ U{300..1500}), held-out evaluation events
    sizes = synth.sizes_uniform(71, 128, lo=300, hi=1500)
    batches = []
    for b in range(16):
        x, cu = synth.gen_events(71, sizes[8 * b:8 * b + 8], first_event=8 * b)
        cls, reg = synth.gen_pf_truth(x, cu)
        lg = np.zeros((len(cls), 6), np.float32)
        lg[np.arange(len(cls)), cls] = TRUTH_LOGIT
        batches.append(tuple(torch.from_numpy(a).cuda() for a in (x, cu, lg, reg)) + (int(np.diff(cu).max()),))
    xe, cue = synth.gen_events(72, synth.sizes_uniform(72, 8, lo=300, hi=1500))
    cls_e, _ = synth.gen_pf_truth(xe, cue)

    tr = Trainer(init, precision="bf16")
    steps = 600
    losses = []
    for s in range(steps):
        X, CU, TL, TR, mn = batches[s % len(batches)]
        lr = 2e-4 + 0.5 * (2e-3 - 2e-4) * (1 + math.cos(math.pi * s / steps))
        loss = tr.step(X, CU, mn, TL, TR, lr, want_loss=(s % 100 == 0 or s == steps - 1))
        if loss is not None:
            losses.append(loss)
    trained = Model(tr.export())
    tr.close()
    untrained = Model(init)
    acc_t = (run_gpu(trained, xe, cue, "bf16")[2] == cls_e).mean()
    acc_u = (run_gpu(untrained, xe, cue, "bf16")[2] == cls_e).mean()
    acc_type = _type_only_accuracy(xe, cls_e)
    print(f"truth accuracy: trained {acc_t:.4f}, untrained {acc_u:.4f}, type alone {acc_type:.4f}; "
          f"loss {losses[0]:.3f} -> {losses[-1]:.4f}")
    assert losses[-1] < 0.1 * losses[0]
    assert acc_u < 0.6
    assert acc_t > acc_type + 0.05
    assert acc_t >= 0.95
    trained.close()
    untrained.close()
