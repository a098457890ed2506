"""Training with 16-bit tensor-core GEMMs (GPU): mlpf_trainer_set_precision(BF16 / FP16).

In that mode every linear layer's GEMM (forward, input gradient, weight gradient) takes
its operands rounded to the 16-bit format and accumulates in FP32 on tcgen05, and the
attention forward and backward multiply 16-bit Q, K, V, probabilities, output and score
gradients on warp-level tensor-core MMAs; the rest of the step is FP32.  Its gradient therefore differs from the float64 gradient by the
effect of that rounding, whose size a float64 model that rounds the same operands at the
same places measures (tests.util.f64_distill_reference with operand_format).  The GPU
does not reproduce that model's rounding errors one by one beyond the first layer: an
FP32 activation that rounds to the other neighbour of a 16-bit value changes the next
layer's activations by part of an ulp, which moves further roundings, and the two runs
decorrelate with depth (measured: per element, the GPU's BF16 logits of the d=128
2 + 2 student differ from the model's by 30 % of the rounding effect, the FP16 ones by
46 %, while both lie as far from the exact logits as the model does).  So the tests bound the
GPU's error by the size of the modelled rounding effect: per tensor at most three times
the model's relative error (plus 1e-4 of the whole gradient), and in total between half
and twice it.  A dropped term or a wrong index would exceed that by far; the GEMM
itself is pinned elementwise in tests/test_gpu_gemm_tc.py.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.util import f64_distill_reference, run_gpu

pytestmark = pytest.mark.gpu

TINY = synth.ModelConfig(d=32, heads=2, ffn=64, l_pid=1, l_reg=1)
# the distillation configuration's student: d=128, 4 heads of 32, FFN 512, 2 + 2 blocks
STUDENT = dataclasses.replace(synth.SMALL, d=128, heads=4, ffn=512, l_pid=2, l_reg=2)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def teacher_targets(cfg, seed, x, cu):
    out = oracle.forward(synth.make_weights(cfg, seed, perturbed=True), cfg, x, cu)
    return out.logits.astype(np.float32), out.reg.astype(np.float32)


def rel_errors(cfg, G, ref):
    gnorm = np.sqrt(sum(np.linalg.norm(v) ** 2 for v in ref.values()))
    out, off = {}, 0
    for name, shape, _ in synth.tensor_specs(cfg):
        n = int(np.prod(shape))
        r = ref[name].reshape(-1)
        out[name] = np.linalg.norm(G[off:off + n] - r) / max(np.linalg.norm(r), 1e-3 * gnorm)
        off += n
    return out


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
@pytest.mark.parametrize("cfg,sizes", [(TINY, [13, 29, 150]), (STUDENT, [40, 1, 97, 130])])
def test_gradient_error_is_the_operand_rounding(fmt, cfg, sizes):
    from paper_2601_17554_b300 import Trainer
    W = synth.make_weights(cfg, 5, perturbed=True)
    x, cu = synth.gen_events(71, sizes)
    tl, tr = teacher_targets(cfg, 6, x, cu)
    t = Trainer(synth.pack_blob(cfg, W), precision=fmt)
    g = torch.zeros(t.num_params, device="cuda")
    loss = t.step(dev(x), dev(cu), max(sizes), dev(tl), dev(tr), lr=0.0, update=False, grads=g)
    t.close()
    g = g.cpu().numpy().astype(np.float64)
    l_r, G_r = f64_distill_reference(W, cfg, x, cu, tl, tr, operand_format=fmt)
    l_x, G_x = f64_distill_reference(W, cfg, x, cu, tl, tr)
    flat = lambda G: np.concatenate([G[n].reshape(-1) for n, _, _ in synth.tensor_specs(cfg)])
    e_gpu, e_model = rel_errors(cfg, g, G_x), rel_errors(cfg, flat(G_r), G_x)
    ratio = np.linalg.norm(g - flat(G_x)) / np.linalg.norm(flat(G_r) - flat(G_x))
    print(f"{fmt} d={cfg.d}: loss {loss:.7f} (rounded model {l_r:.7f}, exact {l_x:.7f}); "
          f"worst tensor error {max(e_gpu.values()):.2e} (model {max(e_model.values()):.2e}); "
          f"gradient error / model's {ratio:.3f}")
    assert abs(loss - l_x) <= 2 * abs(l_r - l_x) + 1e-6 * abs(l_x)
    for name in e_gpu:
        assert e_gpu[name] <= 3 * e_model[name] + 1e-4, (name, e_gpu[name], e_model[name])
    assert 0.5 <= ratio <= 2.0


def test_bf16_training_tracks_fp32_training():
    """40 LAMB steps on the same batch: the BF16-GEMM trainer reduces the loss like the
    FP32 trainer and its loss curve stays within a few per cent of it; the exported
    student runs."""
    from paper_2601_17554_b300 import Model, Trainer
    cfg = synth.SMALL
    x, cu = synth.gen_events(52, [300, 180, 420])
    teacher = Model(synth.pack_blob(cfg, synth.make_weights(cfg, 7, cls_scale=4.0)))
    tl, trg, _, _ = run_gpu(teacher, x, cu, "fp32")
    teacher.close()
    X, CU, TL, TR = dev(x), dev(cu), dev(tl), dev(trg)
    curves = {}
    for prec in ("fp32", "bf16"):
        t = Trainer(synth.pack_blob(cfg, synth.make_weights(cfg, 0)), precision=prec)
        curves[prec] = np.array([t.step(X, CU, 420, TL, TR, lr=2e-3) for _ in range(40)])
        if prec == "bf16":
            student = Model(t.export())
            assert np.isfinite(run_gpu(student, x, cu, "fp32")[0]).all()
            student.close()
        t.close()
    f, b = curves["fp32"], curves["bf16"]
    assert np.isfinite(b).all()
    assert b[-1] < 0.7 * b[0], b[::8]
    assert np.abs(b - f).max() <= 0.05 * f[0], np.abs(b - f).max() / f[0]


def test_autograd_function_in_bf16_matches_the_fused_step():
    from paper_2601_17554_b300 import Trainer
    from paper_2601_17554_b300.autograd import StudentMLPF, distill_loss
    W = synth.make_weights(TINY, 5, perturbed=True)
    blob = synth.pack_blob(TINY, W)
    x, cu = synth.gen_events(61, [13, 29, 140])
    tl, tr = teacher_targets(TINY, 6, x, cu)
    X, CU, TL, TR = dev(x), dev(cu), dev(tl), dev(tr)
    m = StudentMLPF(blob, precision="bf16")
    logits, raw = m(X, CU, 140)
    loss = distill_loss(logits, raw, X, TL, TR)
    loss.backward()
    g_fn = m.params.grad.detach().cpu().numpy().astype(np.float64)
    t = Trainer(blob, precision="bf16")
    g_step = torch.zeros(t.num_params, device="cuda")
    l_step = t.step(X, CU, 140, TL, TR, lr=0.0, update=False, grads=g_step)
    g_step = g_step.cpu().numpy().astype(np.float64)
    assert abs(float(loss.detach()) - l_step) <= 1e-5 * max(1.0, abs(l_step))
    assert np.linalg.norm(g_fn - g_step) <= 1e-5 * np.linalg.norm(g_step)
    m.close()
    t.close()


def test_rejects_other_precisions():
    from paper_2601_17554_b300 import MlpfError, Trainer
    t = Trainer(synth.pack_blob(TINY, synth.make_weights(TINY, 0)))
    with pytest.raises(MlpfError):
        t.set_precision("fp8")
    t.close()
