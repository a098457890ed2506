"""GPU parity of the generic-width tensor-core path (models outside the fused d=64
kernels: the full-size d=256 model with 8 heads of 32, the distillation student d=128
with 4 heads of 32, the architecture as printed with 16 heads of 16) against the FP64
oracle, at the bounds of the 16-bit path: >= 99.9 % per-element argmax agreement and
<= 1e-2 relative regression error per output column.  Plus the properties the path
owes by construction: graph replay equals direct launches bitwise, an event alone
equals the same event inside a batch bitwise (every GEMM row and attention row is
computed independently of its neighbours), windowed attention matches the oracle's
windowed forward, and FP8 is refused.  Both attention kernels of the path run: the one
with the PV products on tcgen05 (MLPF_OPT_WIDE_ATTN_KERNEL = 1) and the warp-level
one (MLPF_OPT_WIDE_ATTN_KERNEL = 0, the default).
"""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from tests.util import make_model, rel_err_cols, run_gpu

pytestmark = pytest.mark.gpu

STUDENT = dataclasses.replace(synth.SMALL, d=128, heads=4, ffn=512, l_pid=2, l_reg=2)


def check_lowp(out, ref, argmax_min=0.999, reg_tol=1e-2):
    lo, rg, cl, _ = out
    assert np.isfinite(lo).all() and np.isfinite(rg).all()
    agree = float((cl == ref.cls).mean())
    e_rg = rel_err_cols(rg, ref.reg)
    print(f"agreement {agree:.5f} over {len(cl)} elements, regression errors {np.round(e_rg, 5)}")
    assert agree >= argmax_min, agree
    assert e_rg.max() <= reg_tol, e_rg
    return agree, e_rg


@pytest.fixture(scope="module")
def full_model():
    return make_model(synth.FULL, 1, perturbed=True)


def _with_kernel(model, kernel, fn):
    from paper_2601_17554_b300._lib import OPT_WIDE_ATTN_KERNEL
    model.set_option(OPT_WIDE_ATTN_KERNEL, kernel)
    assert model.get_option(OPT_WIDE_ATTN_KERNEL) == kernel
    try:
        return fn()
    finally:
        model.set_option(OPT_WIDE_ATTN_KERNEL, 0)


# attention kernels of the path: 0 = every product on warp-level MMAs (default), 1 = PV
# and row sums on tcgen05 (heads of 16 or 32 in groups of four)
@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_full_size_model(full_model, prec, kernel):
    model, w = full_model
    x, cu = synth.gen_events(102, [700, 1, 129, 2100, 64, 0, 300])
    out = _with_kernel(model, kernel, lambda: run_gpu(model, x, cu, prec))
    ref = oracle.forward(w, synth.FULL, x, cu)
    check_lowp(out, ref)
    assert out[3][5].tolist() == [0.0, 0.0, 0.0]


@pytest.mark.parametrize("kernel", [0, 1])
def test_sharpened_attention(kernel):
    """The full-size model with its Q and K projections scaled by 2 (scores four times
    the model's): the running references are raised within and between key tiles, which
    the tcgen05 kernel handles by rescaling the tile's stored P and the row's O and l in
    tensor memory.  Both kernels against the oracle."""
    from paper_2601_17554_b300 import Model
    w = synth.make_weights(synth.FULL, 1, perturbed=True)
    for stack, n in (("pid", synth.FULL.l_pid), ("reg", synth.FULL.l_reg)):
        for l in range(n):
            for t in ("wq", "bq", "wk", "bk"):
                w[f"{stack}.{l}.{t}"] = w[f"{stack}.{l}.{t}"] * 2.0
    model = Model(synth.pack_blob(synth.FULL, w))
    x, cu = synth.gen_events(107, [1500, 129, 700])
    ref = oracle.forward(w, synth.FULL, x, cu)
    for prec in ("bf16", "fp16"):
        out = _with_kernel(model, kernel, lambda: run_gpu(model, x, cu, prec))
        check_lowp(out, ref, argmax_min=0.995)
    model.close()


def test_full_size_workload_sampled(full_model):
    """The 16-event U{1000..6000} workload of the full-size model in BF16; the oracle
    on three of its events."""
    model, w = full_model
    cfg, _, seed, sizes = synth.workload("full16")
    x, cu = synth.gen_events(seed, sizes)
    lo, rg, cl, su = run_gpu(model, x, cu, "bf16")
    ev = [0, 7, 15]
    ref = oracle.forward(w, cfg, x, cu, events=ev)
    rows = np.concatenate([np.arange(cu[e], cu[e + 1]) for e in ev])
    sub = lambda a: a[rows]

    class R:
        cls, reg = sub(ref.cls), sub(ref.reg)
    check_lowp((sub(lo), sub(rg), sub(cl), None), R)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_student_model(prec, kernel):
    model, w = make_model(STUDENT, 2, perturbed=True)
    x, cu = synth.gen_events(103, [1500, 2, 640, 129])
    out = _with_kernel(model, kernel, lambda: run_gpu(model, x, cu, prec))
    check_lowp(out, oracle.forward(w, STUDENT, x, cu))
    model.close()


def test_graph_replay_and_batch_invariance(full_model):
    from paper_2601_17554_b300 import OPT_USE_GRAPHS
    model, _ = full_model
    sizes = [300, 17, 129, 64]
    x, cu = synth.gen_events(104, sizes)
    a = run_gpu(model, x, cu, "bf16")
    model.set_option(OPT_USE_GRAPHS, 0)   # direct launches
    try:
        b = run_gpu(model, x, cu, "bf16")
    finally:
        model.set_option(OPT_USE_GRAPHS, 1)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    # event 2 alone
    xe = x[cu[2]:cu[3]]
    c = run_gpu(model, xe, np.array([0, len(xe)], np.int32), "bf16")
    np.testing.assert_array_equal(c[0], a[0][cu[2]:cu[3]])
    np.testing.assert_array_equal(c[1], a[1][cu[2]:cu[3]])


@pytest.mark.parametrize("kernel", [0, 1])
def test_windowed_attention(full_model, kernel):
    from paper_2601_17554_b300 import OPT_ATTN_WINDOW
    model, w = full_model
    x, cu = synth.gen_events(105, [700, 129, 1000])
    model.set_option(OPT_ATTN_WINDOW, 2)   # 128-row blocks +- 2 in eta order
    try:
        out = _with_kernel(model, kernel, lambda: run_gpu(model, x, cu, "bf16"))
    finally:
        model.set_option(OPT_ATTN_WINDOW, 0)
    check_lowp(out, oracle.forward(w, synth.FULL, x, cu, window=2))


def test_fp8_refused(full_model):
    from paper_2601_17554_b300 import MlpfError
    model, _ = full_model
    x, cu = synth.gen_events(106, [10])
    with pytest.raises(MlpfError) as ei:
        run_gpu(model, x, cu, "fp8")
    assert ei.value.status == 7   # MLPF_E_UNSUPPORTED


def test_autotune_picks_a_wide_kernel(full_model, tmp_path):
    """mlpf_autotune on a generic-width model times its two attention kernels, keeps
    one in MLPF_OPT_WIDE_ATTN_KERNEL, writes a "_wide" cache line and reuses it."""
    import torch
    from paper_2601_17554_b300._lib import OPT_WIDE_ATTN_KERNEL
    model, w = full_model
    x, cu = synth.gen_events(108, [900, 300, 1200])
    xt, ct = torch.from_numpy(x).cuda(), torch.from_numpy(cu).cuda()
    path = str(tmp_path / "tune.txt")
    try:
        model.autotune(xt, ct, 1200, precision="bf16", cache_path=path)
        k = model.get_option(OPT_WIDE_ATTN_KERNEL)
        assert k in (0, 1)
        lines = [ln for ln in open(path).read().split("\n") if ln]
        assert len(lines) == 1 and lines[0].split()[0].endswith("_wide") and int(lines[0].split()[1]) == k
        model.set_option(OPT_WIDE_ATTN_KERNEL, 1 - k)
        model.autotune(xt, ct, 1200, precision="bf16", cache_path=path)   # cached: no timing
        assert model.get_option(OPT_WIDE_ATTN_KERNEL) == k
        assert len([ln for ln in open(path).read().split("\n") if ln]) == 1
        check_lowp(run_gpu(model, x, cu, "bf16"), oracle.forward(w, synth.FULL, x, cu))
    finally:
        model.set_option(OPT_WIDE_ATTN_KERNEL, 0)
