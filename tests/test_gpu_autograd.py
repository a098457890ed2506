"""The training kernels behind torch.autograd.Function (GPU).

The gradient that torch autograd obtains through StudentFunction (loss in torch,
backward in the library's hand-written kernels) equals the fused training step's
gradient and an independent float64 torch model's; a student trained through the
Function with a torch optimizer gains over the untrained student and stands in
for the teacher on most events at a fraction of its cost.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.util import f64_distill_reference, make_model, run_gpu

pytestmark = pytest.mark.gpu

TINY = synth.ModelConfig(d=32, heads=2, ffn=64, l_pid=1, l_reg=1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_function_gradient_matches_fused_step_and_float64_autograd():
    from paper_2601_17554_b300 import Trainer
    from paper_2601_17554_b300.autograd import StudentMLPF, distill_loss
    W = synth.make_weights(TINY, 5, perturbed=True)
    blob = synth.pack_blob(TINY, W)
    x, cu = synth.gen_events(61, [13, 29, 1])
    Wt = synth.make_weights(TINY, 6, perturbed=True)
    ref_out = oracle.forward(Wt, TINY, x, cu)
    tl, tr = ref_out.logits.astype(np.float32), ref_out.reg.astype(np.float32)
    X, CU, TL, TR = dev(x), dev(cu), dev(tl), dev(tr)
    m = StudentMLPF(blob)
    logits, raw = m(X, CU, 29)
    loss = distill_loss(logits, raw, X, TL, TR)
    loss.backward()
    g_fn = m.params.grad.detach().cpu().numpy().astype(np.float64)
    # the fused step (loss and gradient in the library's kernels)
    tr_ = Trainer(blob)
    g_step = torch.zeros(tr_.num_params, device="cuda")
    l_step = tr_.step(X, CU, 29, TL, TR, lr=0.0, update=False, grads=g_step)
    assert abs(float(loss.detach()) - l_step) <= 1e-5 * max(1.0, abs(l_step))
    g_step = g_step.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g_fn - g_step) <= 1e-5 * np.linalg.norm(g_step)
    # an independent float64 model
    l64, G64 = f64_distill_reference(W, TINY, x, cu, tl, tr)
    assert abs(float(loss.detach()) - l64) <= 1e-5 * max(1.0, abs(l64))
    off, gnorm = 0, np.sqrt(sum(np.linalg.norm(v) ** 2 for v in G64.values()))
    for name, shape, _ in synth.tensor_specs(TINY):
        n = int(np.prod(shape))
        ref = G64[name].reshape(-1)
        err = np.linalg.norm(g_fn[off:off + n] - ref) / max(np.linalg.norm(ref), 1e-3 * gnorm)
        assert err <= 1e-4, (name, err)
        off += n
    m.close()
    tr_.close()


def test_backward_needs_its_forward():
    from paper_2601_17554_b300 import MlpfError, check
    from paper_2601_17554_b300.autograd import StudentMLPF
    m = StudentMLPF(synth.pack_blob(TINY, synth.make_weights(TINY, 5)))
    x, cu = synth.gen_events(62, [20, 7])
    X, CU = dev(x), dev(cu)
    g = torch.empty(m.trainer.num_params, device="cuda")
    d6, d5 = torch.zeros((27, 6), device="cuda"), torch.zeros((27, 5), device="cuda")
    p = lambda t: __import__("ctypes").c_void_p(t.data_ptr())
    with pytest.raises(MlpfError):   # no forward yet
        check(m.trainer.L.mlpf_trainer_backward(m.trainer.h, p(X), p(CU), 2, 27, 20, p(d6), p(d5), p(g), None))
    m.close()


def test_trained_student_gains_over_untrained():
    """Distillation through the autograd Function with torch's Adam: a d=32, 1 + 1
    student of a d=64, 2 + 2 teacher (BF16 forward for the targets) agrees with
    the teacher on held-out events far more often than the same student before
    training, and its regressions are closer."""
    import dataclasses
    from paper_2601_17554_b300 import Model
    from paper_2601_17554_b300.autograd import StudentMLPF, distill_loss
    tcfg = dataclasses.replace(synth.SMALL, l_pid=2, l_reg=2)
    teacher, _ = make_model(tcfg, 7, cls_scale=8.0)
    blob0 = synth.pack_blob(TINY, synth.make_weights(TINY, 0))
    # held-out evaluation events
    xe, cue = synth.gen_events(3000, synth.sizes_uniform(3000, 8, 200, 600))
    t_lo, t_rg, t_cl, _ = run_gpu(teacher, xe, cue, "bf16")

    def agreement(blob):
        s = Model(blob)
        lo, rg, cl, _ = run_gpu(s, xe, cue, "fp32")
        s.close()
        err = np.sqrt(((rg - t_rg) ** 2).sum(0)) / np.sqrt((t_rg ** 2).sum(0))
        return float((cl == t_cl).mean()), float(err.max())

    a0, e0 = agreement(blob0)
    m = StudentMLPF(blob0)
    opt = torch.optim.Adam(m.parameters(), lr=3e-3)
    for step in range(300):
        x, cu = synth.gen_events(2000 + step, synth.sizes_uniform(2000 + step, 6, 100, 500))
        X, CU = dev(x), dev(cu)
        tlo, trg, _, _ = teacher.forward(X, CU, int(np.diff(cu).max()), precision="bf16")
        lo, raw = m(X, CU, int(np.diff(cu).max()))
        loss = distill_loss(lo, raw, X, tlo, trg)
        opt.zero_grad()
        loss.backward()
        opt.step()
    a1, e1 = agreement(m.export())
    print(f"untrained: agreement {a0:.3f}, max column error {e0:.3f}; trained: {a1:.3f}, {e1:.3f}")
    assert a1 >= a0 + 0.2 and a1 >= 0.6, (a0, a1)
    assert e1 <= 0.5 * e0, (e0, e1)
    m.close()
    teacher.close()
