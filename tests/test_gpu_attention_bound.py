"""Both paths of the warp-MMA attention kernels against the oracle.

The kernel bounds a key tile's scores row by row, |q . k| <= |q| max|k|
(Cauchy-Schwarz, the per-block maxima of |k| written by the QKV epilogues).  A
full tile (after the first) whose bound stays within 2^15 of every row's
exponent reference runs without the maxima check; otherwise it takes the checked
path (row maxima, warp vote, lazy rescale).  With the random-weight test model
every full tile passes; scaling the Q and K projections sharpens the attention
and moves tiles to the checked path.  A float64 emulation of the check on the
first PID layer gives, for the events below: Q, K x 1.4 -> 79 % of the (warp,
tile) pairs on the bound path and 21 % checked (both, interleaved within an
item); x 2 -> 0.4 % on the bound path.

Bounds: sharper attention amplifies the 16-bit rounding of Q and K (the score
error grows with |S|, up to about 40 log2 units at x 2), so the floors are
looser than the parity tests' for the unscaled model.

Both warp-level kernels are checked: the default (variant 4: P V and the row sums
on warp-level MMAs, O rescaled in registers) and the one with P V and the row sums
on tcgen05 (variant 9: one reference per row and key tile, O and l rescaled in
tensor memory).
"""
import numpy as np
import pytest

import oracle
import synth
from tests.util import rel_err_cols, run_gpu

pytestmark = pytest.mark.gpu

SIZES = [1000, 4097, 300, 65, 129, 64, 1]
# The specified bounds (>= 99.9 % argmax agreement, <= 1e-2 regression error), except
# BF16 at Q and K x 2: scores four times larger than the model's make the BF16
# rounding of Q and K (an error proportional to the score) cost more; the float64
# emulation of the BF16 mode's roundings (tests/lowp_emul.py) gives 99.77 % and
# 6.5e-3 on exactly these inputs, and the floor allows four flips more (of 5656).
BOUNDS = {("fp16", 1.4): (0.999, 1e-2), ("bf16", 1.4): (0.999, 1e-2),
          ("fp16", 2.0): (0.999, 1e-2), ("bf16", 2.0): (0.997, 1e-2)}


def scaled_model(f):
    from paper_2601_17554_b300 import Model
    cfg = synth.SMALL
    w = synth.make_weights(cfg, 3, perturbed=True)
    for stack in ("pid", "reg"):
        for t in ("wq", "bq", "wk", "bk"):
            w[f"{stack}.0.{t}"] = w[f"{stack}.0.{t}"] * f
    return Model(synth.pack_blob(cfg, w)), w


@pytest.mark.parametrize("variant", [4, 9])
@pytest.mark.parametrize("f", [1.4, 2.0])
def test_bound_and_checked_paths_match_oracle(f, variant):
    from paper_2601_17554_b300 import _lib
    model, w = scaled_model(f)
    model.set_option(_lib.OPT_ATTN_VARIANT_BF16, variant)
    model.set_option(_lib.OPT_ATTN_VARIANT_FP16, variant)
    x, cu = synth.gen_events(22, SIZES)
    ref = oracle.forward(w, synth.SMALL, x, cu)
    for prec in ("fp16", "bf16"):
        lo, rg, cl, su = run_gpu(model, x, cu, prec)
        assert np.isfinite(lo).all() and np.isfinite(rg).all() and np.isfinite(su).all()
        agree = (cl == ref.cls).mean()
        err = rel_err_cols(rg, ref.reg)
        print(f"variant {variant} scale {f} {prec}: argmax agreement {agree:.5f}, max column rel err {err.max():.3e}")
        amin, etol = BOUNDS[(prec, f)]
        assert agree >= amin, (prec, f, agree)
        assert err.max() <= etol, (prec, f, err)
    model.close()
