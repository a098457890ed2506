"""Windowed attention (MLPF_OPT_ATTN_WINDOW): each event's elements in eta order,
query block b of 128 elements attends to key blocks b - w .. b + w.

Parity with the FP64 oracle's windowed forward on the FP32 path (1e-4) and the
16-bit paths (their usual bounds); a window wider than the event equals full
attention; the variants of each kernel family agree bit for bit, and the two
families agree within the 16-bit bounds; argument checks.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.util import make_model, rel_err_cols, run_gpu

pytestmark = pytest.mark.gpu

SIZES = [300, 700, 1, 129, 0, 1000, 64, 385]
OPT_WINDOW = 10


@pytest.fixture(scope="module")
def model():
    return make_model(synth.SMALL, 13, perturbed=True)


def _with_window(m, w, fn):
    m.set_option(OPT_WINDOW, w)
    try:
        return fn()
    finally:
        m.set_option(OPT_WINDOW, 0)


def test_window_fp32_parity(model):
    m, W = model
    x, cu = synth.gen_events(81, SIZES)
    for w in (1, 2):
        out = _with_window(m, w, lambda: run_gpu(m, x, cu, "fp32"))
        ref = oracle.forward(W, synth.SMALL, x, cu, window=w)
        assert rel_err_cols(out[0], ref.logits).max() <= 1e-4
        assert rel_err_cols(out[1], ref.reg).max() <= 1e-4
        np.testing.assert_allclose(out[3], ref.sums, rtol=1e-4, atol=1e-4 * np.abs(ref.sums).max())
        # the window changes the result of the events longer than its reach
        full = oracle.forward(W, synth.SMALL, x, cu)
        assert np.abs(ref.logits[cu[1]:cu[2]] - full.logits[cu[1]:cu[2]]).max() > 1e-6


@pytest.mark.parametrize("prec,argmax_min,reg_tol", [("bf16", 0.999, 1e-2), ("fp16", 0.999, 1e-2)])
def test_window_16bit_parity(model, prec, argmax_min, reg_tol):
    m, W = model
    # about 9700 elements, so that the 0.1 % of the argmax bound is several elements
    x, cu = synth.gen_events(82, SIZES + [3000, 4096])
    lo, rg, cl, su = _with_window(m, 1, lambda: run_gpu(m, x, cu, prec))
    ref = oracle.forward(W, synth.SMALL, x, cu, window=1)
    assert (cl == ref.cls).mean() >= argmax_min
    assert rel_err_cols(rg, ref.reg).max() <= reg_tol


def test_wide_window_equals_full_attention(model):
    m, _ = model
    x, cu = synth.gen_events(83, SIZES)
    full = run_gpu(m, x, cu, "fp32")
    wide = _with_window(m, 8, lambda: run_gpu(m, x, cu, "fp32"))   # 1000 elements: 8 blocks
    assert rel_err_cols(wide[0], full[0]).max() <= 1e-5
    assert rel_err_cols(wide[1], full[1]).max() <= 1e-5


def test_window_variants_agree(model):
    m, _ = model
    x, cu = synth.gen_events(84, SIZES)
    outs = []
    try:
        # warp-level MMAs (4, 3, 5), tensor-memory kernel (2, 0), QK^T on tcgen05 (7, 6),
        # PV on tcgen05 (9, 8)
        for v in (4, 3, 5, 2, 0, 7, 6, 9, 8):
            m.set_option(7, v)
            outs.append(_with_window(m, 1, lambda: run_gpu(m, x, cu, "bf16")))
    finally:
        m.set_option(7, 4)
    for grp in ((0, 1, 2), (3, 4), (5, 6), (7, 8)):
        for i in grp[1:]:
            for a, b in zip(outs[grp[0]], outs[i]):
                np.testing.assert_array_equal(a, b)
    for o in (outs[3], outs[5], outs[7]):
        assert (outs[0][2] == o[2]).mean() >= 0.999
        assert rel_err_cols(o[1], outs[0][1]).max() <= 1e-2


def test_window_argument_checks(model):
    from paper_2601_17554_b300 import MlpfError
    m, _ = model
    with pytest.raises(MlpfError):
        m.set_option(OPT_WINDOW, -1)
    x, cu = synth.gen_events(85, [16385])
    with pytest.raises(MlpfError) as ei:
        _with_window(m, 1, lambda: run_gpu(m, x, cu, "bf16"))
    assert ei.value.status == 7
