"""GPU training kernels and the gated student/teacher forward.

Gradients of the hand-written backward kernels are checked against central
finite differences of the FP64 oracle's distillation loss (N <= 32, small
model) and against torch float64 autograd of the same loss.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.util import f64_distill_reference, run_gpu

pytestmark = pytest.mark.gpu

TINY = synth.ModelConfig(d=32, heads=2, ffn=64, l_pid=1, l_reg=1)


def teacher_targets(cfg, seed, x, cu):
    W = synth.make_weights(cfg, seed, perturbed=True)
    out = oracle.forward(W, cfg, x, cu)
    return out.logits.astype(np.float32), out.reg.astype(np.float32)


def gpu_grads(blob, x, cu, tl, tr):
    from paper_2601_17554_b300 import Trainer
    tr_ = Trainer(blob)
    g = torch.zeros(tr_.num_params, dtype=torch.float32, device="cuda")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    loss = tr_.step(dev(x), dev(cu), int(np.diff(cu).max()), dev(tl), dev(tr), lr=0.0, update=False, grads=g)
    tr_.close()
    return loss, g.cpu().numpy().astype(np.float64)


def unflatten(cfg, vec):
    out, off = {}, 0
    for name, shape, _ in synth.tensor_specs(cfg):
        n = int(np.prod(shape))
        out[name] = vec[off:off + n].reshape(shape)
        off += n
    assert off == len(vec)
    return out


@pytest.fixture(scope="module")
def tiny_case():
    W = synth.make_weights(TINY, 5, perturbed=True)
    x, cu = synth.gen_events(51, [13, 29])
    tl, tr = teacher_targets(TINY, 6, x, cu)
    loss, g = gpu_grads(synth.pack_blob(TINY, W), x, cu, tl, tr)
    return W, x, cu, tl, tr, loss, unflatten(TINY, g)


def test_loss_matches_oracle(tiny_case):
    W, x, cu, tl, tr, loss, _ = tiny_case
    ref = oracle.distill_loss(W, TINY, x, cu, tl, tr)
    assert abs(loss - ref) <= 1e-5 * max(1.0, abs(ref)), (loss, ref)


def test_gradients_match_oracle_finite_differences(tiny_case):
    W, x, cu, tl, tr, loss, G = tiny_case
    rng = np.random.default_rng(0)
    Wd = {k: v.astype(np.float64) for k, v in W.items()}
    gmax = max(np.abs(v).max() for v in G.values())
    checked = 0
    for name, shape, _ in synth.tensor_specs(TINY):
        for _ in range(2):
            idx = tuple(int(rng.integers(s)) for s in shape)
            w0 = Wd[name][idx]
            h = 1e-6 * max(1.0, abs(w0))
            Wd[name][idx] = w0 + h
            lp = oracle.distill_loss(Wd, TINY, x, cu, tl, tr)
            Wd[name][idx] = w0 - h
            lm = oracle.distill_loss(Wd, TINY, x, cu, tl, tr)
            Wd[name][idx] = w0
            fd = (lp - lm) / (2 * h)
            g = G[name][idx]
            assert abs(g - fd) <= 2e-3 * abs(fd) + 2e-5 * gmax, (name, idx, g, fd)
            checked += 1
    assert checked == 2 * len(synth.tensor_specs(TINY))


def test_gradients_match_torch_autograd(tiny_case):
    W, x, cu, tl, tr, loss, G = tiny_case
    _, ref_g = f64_distill_reference(W, TINY, x, cu, tl, tr)
    # The key bias has an exactly zero gradient (the softmax of a row is invariant to
    # a constant added to all its scores), so errors are taken relative to
    # max(|grad of the tensor|, 1e-3 |whole gradient|).
    gnorm = np.sqrt(sum(np.linalg.norm(ref_g[n]) ** 2 for n in W))
    for name in W:
        ref = ref_g[name]
        err = np.linalg.norm(G[name] - ref) / max(np.linalg.norm(ref), 1e-3 * gnorm)
        assert err <= 1e-4, (name, err)


def test_training_reduces_loss():
    from paper_2601_17554_b300 import Model, Trainer
    cfg = synth.SMALL
    x, cu = synth.gen_events(52, [300, 180, 420])
    teacher = Model(synth.pack_blob(cfg, synth.make_weights(cfg, 7, cls_scale=4.0)))
    tl, trg, _, _ = run_gpu(teacher, x, cu, "fp32")
    tr_ = Trainer(synth.pack_blob(cfg, synth.make_weights(cfg, 0)))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    X, CU, TL, TR = dev(x), dev(cu), dev(tl), dev(trg)
    losses = [tr_.step(X, CU, 420, TL, TR, lr=2e-3) for _ in range(40)]
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.7 * losses[0], losses[::8]
    # the exported blob loads and runs
    student = Model(tr_.export())
    out = run_gpu(student, x, cu, "fp32")
    assert np.isfinite(out[0]).all()


def test_export_round_trip_without_update():
    from paper_2601_17554_b300 import Trainer
    blob = synth.pack_blob(TINY, synth.make_weights(TINY, 11, perturbed=True))
    tr_ = Trainer(blob)
    assert tr_.export() == blob


def test_gated_forward_extremes_and_flags():
    from paper_2601_17554_b300 import Model, forward_gated
    cfg = synth.SMALL
    student = Model(synth.pack_blob(cfg, synth.make_weights(cfg, 0)))
    teacher = Model(synth.pack_blob(cfg, synth.make_weights(cfg, 3, perturbed=True)))
    sizes = [500, 40, 1200, 7, 260]
    x, cu = synth.gen_events(53, sizes)
    X, CU = torch.from_numpy(x).cuda(), torch.from_numpy(cu).cuda()
    s_out = run_gpu(student, x, cu, "bf16")
    t_out = run_gpu(teacher, x, cu, "fp32")
    lo, rg, cl, su, used, nfb = forward_gated(student, teacher, 2.0, X, CU, 1200)  # every event falls back
    assert nfb == 5 and used.cpu().numpy().tolist() == [1] * 5
    np.testing.assert_array_equal(lo.cpu().numpy(), t_out[0])
    np.testing.assert_array_equal(rg.cpu().numpy(), t_out[1])
    np.testing.assert_array_equal(su.cpu().numpy(), t_out[3])
    lo, rg, cl, su, used, nfb = forward_gated(student, teacher, -1.0, X, CU, 1200)  # none does
    assert nfb == 0
    np.testing.assert_array_equal(lo.cpu().numpy(), s_out[0])
    np.testing.assert_array_equal(cl.cpu().numpy(), s_out[2])
    # a threshold in between: flags follow the student's mean max-softmax per event
    p = np.exp(s_out[0] - s_out[0].max(1, keepdims=True))
    conf = np.array([(1.0 / p[cu[e]:cu[e + 1]].sum(1)).mean() for e in range(5)])
    c = np.sort(conf)
    thr = float((c[1] + c[2]) / 2)  # between two events' confidences, away from either
    lo, rg, cl, su, used, nfb = forward_gated(student, teacher, thr, X, CU, 1200)
    flags = used.cpu().numpy()
    assert flags.tolist() == (conf < thr).astype(int).tolist()
    lo = lo.cpu().numpy()
    for e in range(5):
        src = t_out if flags[e] else s_out
        np.testing.assert_array_equal(lo[cu[e]:cu[e + 1]], src[0][cu[e]:cu[e + 1]])
    # event confidence = minimum over the event's elements (MLPF_OPT_GATE_CONFIDENCE = 1)
    cmin = np.array([(1.0 / p[cu[e]:cu[e + 1]].sum(1)).min() for e in range(5)])
    c = np.sort(cmin)
    thr = float((c[2] + c[3]) / 2)
    student.set_option(11, 1)
    try:
        lo, rg, cl, su, used, nfb = forward_gated(student, teacher, thr, X, CU, 1200)
    finally:
        student.set_option(11, 0)
    assert used.cpu().numpy().tolist() == (cmin < thr).astype(int).tolist()
    assert nfb == int((cmin < thr).sum())
