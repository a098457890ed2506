"""GPU parity of the architecture as Sec. 5.3 prints it (per-type embedding,
two parallel encoders on one embedding, binary + 5-class PID heads, ReLU,
d=256 with 16 heads of 16, 3+3 blocks) against the FP64 oracle.

It runs on the plain FP32 path (within 1e-4 relative per output column); the
tensor-core precisions refuse it with MLPF_E_UNSUPPORTED.  The class decision
(binary logit > 0, then 1 + argmax of the PID scores) must match the oracle on
every element whose binary logit and top-2 PID margin are not within 1e-3 of
a tie.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.util import make_model, max_scaled_err, rel_err_cols, run_gpu

pytestmark = pytest.mark.gpu


def _decisive(logits):
    top2 = np.sort(logits[:, 1:], axis=1)[:, -2:]
    return (np.abs(logits[:, 0]) > 1e-3) & (top2[:, 1] - top2[:, 0] > 1e-3)


@pytest.fixture(scope="module")
def paper_model():
    return make_model(synth.PAPER, 4, perturbed=True)   # weight seed with both decisions common


def test_paper_arch_fp32_parity(paper_model):
    model, w = paper_model
    assert model.config["arch"] == 1 and model.config["heads"] == 16
    x, cu = synth.gen_events(31, [300, 1, 129, 700, 0, 64])
    lo, rg, cl, su = run_gpu(model, x, cu, "fp32")
    ref = oracle.forward(w, synth.PAPER, x, cu)
    assert rel_err_cols(lo, ref.logits).max() <= 1e-4
    assert rel_err_cols(rg, ref.reg).max() <= 1e-4
    assert max_scaled_err(rg, ref.reg) <= 5e-3
    keep = _decisive(ref.logits)
    assert keep.mean() > 0.95
    np.testing.assert_array_equal(cl[keep], ref.cls[keep])
    # both decision branches occur: particles and non-particles
    assert (ref.cls == 0).any() and (ref.cls != 0).any()
    assert su[4].tolist() == [0.0, 0.0, 0.0]
    ok = np.all(cl == ref.cls)
    if ok:
        np.testing.assert_allclose(su, ref.sums, rtol=1e-4, atol=1e-4 * np.abs(ref.sums).max())


def test_paper_arch_sampled_full_workload(paper_model):
    """Two events of the 8-event U{1000..6000} workload of this architecture."""
    model, w = paper_model
    cfg, _, seed, sizes = synth.workload("paper8")
    x, cu = synth.gen_events(seed, sizes)
    lo, rg, cl, su = run_gpu(model, x, cu, "fp32")
    ref = oracle.forward(w, cfg, x, cu, events=[0, 5])
    for e in (0, 5):
        sl = slice(cu[e], cu[e + 1])
        assert rel_err_cols(lo[sl], ref.logits[sl]).max() <= 1e-4
        assert rel_err_cols(rg[sl], ref.reg[sl]).max() <= 1e-4
        keep = _decisive(ref.logits[sl])
        np.testing.assert_array_equal(cl[sl][keep], ref.cls[sl][keep])


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_paper_arch_tensor_core_refused(paper_model, prec):
    from paper_2601_17554_b300 import MlpfError
    model, _ = paper_model
    x, cu = synth.gen_events(32, [10])
    with pytest.raises(MlpfError) as ei:
        run_gpu(model, x, cu, prec)
    assert ei.value.status == 7   # MLPF_E_UNSUPPORTED
