"""Attention kernel variants and the autotuner (through the C ABI).

Variants in one group run the same per-head arithmetic in the same order and
must be bit-identical: the tcgen05 kernels with S and P in tensor memory (four,
six or eight K/V stages), the warp-level-MMA kernels (four or eight stages,
128- or 64-row items), the warp-level kernels with QK^T on tcgen05 (four or
eight stages) and the warp-level kernels with PV and the row sums on tcgen05
(four or eight stages).  Groups differ in
summation order and exponent references: each must meet the oracle bounds of
the precision and stay close to variant 0.  The autotuner must pick a valid
variant, write its cache line and reuse it.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.util import make_model, rel_err_cols, run_gpu

pytestmark = pytest.mark.gpu

SIZES = [1, 17, 64, 65, 129, 300, 0, 511, 1024, 2]
N_VARIANTS = 10
GROUPS = ((0, 1, 2), (3, 4, 5), (6, 7), (8, 9))


@pytest.fixture(scope="module")
def model():
    return make_model(synth.SMALL, 5, perturbed=True)


@pytest.mark.parametrize("precision,opt,argmax_min,reg_tol", [
    ("bf16", 7, 0.999, 1e-2), ("fp16", 8, 0.999, 1e-2)])
def test_variants_identical(model, precision, opt, argmax_min, reg_tol):
    m, w = model
    x, cu = synth.gen_events(77, SIZES)
    ref = oracle.forward(w, synth.SMALL, x, cu)
    outs = []
    default = m.get_option(opt)
    assert default == 4   # warp-level MMAs, 8 K/V stages
    try:
        for v in range(N_VARIANTS):
            m.set_option(opt, v)
            assert m.get_option(opt) == v
            outs.append(run_gpu(m, x, cu, precision))
    finally:
        m.set_option(opt, default)
    for grp in GROUPS:
        first = outs[grp[0]]
        for v in grp[1:]:
            for a, b in zip(first, outs[v]):
                np.testing.assert_array_equal(a, b)
        lo, rg, cl, _ = first
        assert (cl == ref.cls).mean() >= argmax_min
        assert rel_err_cols(rg, ref.reg).max() <= reg_tol
        assert (cl == outs[0][2]).mean() >= argmax_min
        assert rel_err_cols(rg, outs[0][1]).max() <= reg_tol


def test_variant_option_range(model):
    from paper_2601_17554_b300 import MlpfError
    m, _ = model
    with pytest.raises(MlpfError):
        m.set_option(7, N_VARIANTS)
    with pytest.raises(MlpfError):
        m.set_option(9, -1)


def test_autotune_cache(model, tmp_path):
    import torch
    m, _ = model
    x, cu = synth.gen_events(78, [300, 1000, 64, 5])
    xt = torch.from_numpy(x).cuda()
    ct = torch.from_numpy(cu).cuda()
    path = str(tmp_path / "tune.txt")
    default = m.get_option(7)
    try:
        v = m.autotune(xt, ct, 1000, precision="bf16", cache_path=path)
        assert v in range(N_VARIANTS)
        lines = open(path).read().split("\n")
        lines = [ln for ln in lines if ln]
        assert len(lines) == 1
        key, var, ms = lines[0].split()
        assert int(var) == v and float(ms) > 0 and "_prec1_T2048" in key
        # a cached key is applied without timing and without a new line
        m.set_option(7, (v + 1) % N_VARIANTS)
        assert m.autotune(xt, ct, 1000, precision="bf16", cache_path=path) == v
        assert len([ln for ln in open(path).read().split("\n") if ln]) == 1
        assert m.autotune(xt, ct, 1000, precision="fp32", cache_path=path) is None
    finally:
        m.set_option(7, default)
