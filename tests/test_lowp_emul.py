"""Pins of the float64 rounding emulation used for the 16-bit / E4M3 error budget.

With no stage rounded the emulation is the oracle's forward; its rounding
functions agree with torch's BF16, FP16 and E4M3 conversions; rounding one stage
changes the outputs by about that format's unit roundoff.
"""
import numpy as np
import torch

import oracle
import synth
from tests.lowp_emul import (STAGES, Emulation, gpu_formats, round_bf16, round_e4m3,
                             round_fp16)


def test_no_rounding_is_the_oracle():
    cfg = synth.SMALL
    W = synth.make_weights(cfg, 3, perturbed=True)
    x, cu = synth.gen_events(7, [40, 1, 77])
    lo, raw, reg, cls, rows = Emulation(W, cfg, {}).forward(x, cu)
    ref = oracle.forward(W, cfg, x, cu)
    assert np.allclose(lo, ref.logits, rtol=1e-12, atol=1e-12)
    assert np.allclose(raw, ref.raw, rtol=1e-12, atol=1e-12)
    assert (cls == ref.cls).all()


def test_roundings_match_torch_conversions():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 3, 4000),
                        [0.0, 1.0, -1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 448.0, -300.0]])
    t = torch.from_numpy(v.astype(np.float32))
    assert np.array_equal(round_bf16(v), t.to(torch.bfloat16).double().numpy())
    assert np.array_equal(round_fp16(v), t.to(torch.float16).double().numpy())
    inr = np.abs(v) <= 448.0
    e4 = torch.from_numpy(v[inr].astype(np.float32)).to(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(round_e4m3(v[inr]), e4)
    # ties to even: 1 + 2^-8 is halfway between BF16 neighbours 1 and 1 + 2^-7
    assert round_bf16(1 + 2 ** -8) == 1.0 and round_bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6
    assert round_e4m3(1000.0) == 448.0   # saturating


def test_one_stage_costs_about_its_unit_roundoff():
    cfg = synth.SMALL
    W = synth.make_weights(cfg, 0)
    x, cu = synth.gen_events(8, [300])
    ref = Emulation(W, cfg, {}).forward(x, cu)[0]
    for fmt, u in (("bf16", 2.0 ** -8), ("fp16", 2.0 ** -11)):   # unit roundoffs
        lo = Emulation(W, cfg, {"w_head2": fmt}).forward(x, cu)[0]
        rel = np.sqrt(((lo - ref) ** 2).mean()) / np.sqrt((ref ** 2).mean())
        assert 0.05 * u < rel < 2 * u, (fmt, rel)


def test_gpu_formats_cover_every_stage():
    for mode in ("bf16", "fp16", "fp8", "bf16_all"):
        f = gpu_formats(mode)
        assert set(f) == set(STAGES)
    # the BF16 mode: attention operands in BF16, GEMM operands in FP16
    f = gpu_formats("bf16")
    assert {s for s, v in f.items() if v == "bf16"} == {"qk", "v", "p_arg", "p"}
