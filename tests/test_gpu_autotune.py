"""Attention kernel variants and the autotuner (through the C ABI).

The four variants (one or two heads per warpgroup, two or four K/V stages)
run the same per-head arithmetic in the same order, so their outputs must be
bit-identical; each must also meet the oracle bounds of its precision.  The
autotuner must pick a valid variant, write its cache line and reuse it.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.util import make_model, rel_err_cols, run_gpu

pytestmark = pytest.mark.gpu

SIZES = [1, 17, 64, 65, 129, 300, 0, 511, 1024, 2]


@pytest.fixture(scope="module")
def model():
    return make_model(synth.SMALL, 5, perturbed=True)


@pytest.mark.parametrize("precision,opt,argmax_min,reg_tol", [
    ("bf16", 7, 0.99, 3e-2), ("fp16", 8, 0.995, 1.5e-2)])
def test_variants_identical(model, precision, opt, argmax_min, reg_tol):
    m, w = model
    x, cu = synth.gen_events(77, SIZES)
    ref = oracle.forward(w, synth.SMALL, x, cu)
    outs = []
    try:
        for v in range(4):
            m.set_option(opt, v)
            assert m.get_option(opt) == v
            outs.append(run_gpu(m, x, cu, precision))
    finally:
        m.set_option(opt, 0)
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            np.testing.assert_array_equal(a, b)
    lo, rg, cl, _ = outs[0]
    assert (cl == ref.cls).mean() >= argmax_min
    assert rel_err_cols(rg, ref.reg).max() <= reg_tol


def test_variant_option_range(model):
    from paper_2601_17554_b300 import MlpfError
    m, _ = model
    with pytest.raises(MlpfError):
        m.set_option(7, 4)
    with pytest.raises(MlpfError):
        m.set_option(9, -1)


def test_autotune_cache(model, tmp_path):
    import torch
    m, _ = model
    x, cu = synth.gen_events(78, [300, 1000, 64, 5])
    xt = torch.from_numpy(x).cuda()
    ct = torch.from_numpy(cu).cuda()
    path = str(tmp_path / "tune.txt")
    try:
        v = m.autotune(xt, ct, 1000, precision="bf16", cache_path=path)
        assert v in range(4)
        lines = open(path).read().split("\n")
        lines = [ln for ln in lines if ln]
        assert len(lines) == 1
        key, var, ms = lines[0].split()
        assert int(var) == v and float(ms) > 0 and "_prec1_T2048" in key
        # a cached key is applied without timing and without a new line
        m.set_option(7, (v + 1) % 4)
        assert m.autotune(xt, ct, 1000, precision="bf16", cache_path=path) == v
        assert len([ln for ln in open(path).read().split("\n") if ln]) == 1
        assert m.autotune(xt, ct, 1000, precision="fp32", cache_path=path) is None
    finally:
        m.set_option(7, 0)
