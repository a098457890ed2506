"""GPU parity of the library against the FP64 oracle (through the C ABI).

FP32 path: within 1e-4 relative (normwise per output column) on logits and the
decoded regressions.  16-bit tensor-core path (FP16, and BF16 attention with FP16 GEMM operands): >= 99.9 %
per-element argmax agreement and <= 1e-2 relative regression error (normwise
per column), the bounds the path is specified to, in every test.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.util import make_model, max_scaled_err, rel_err_cols, run_gpu

pytestmark = pytest.mark.gpu

EDGE_SIZES = [1, 2, 15, 16, 17, 63, 64, 65, 127, 128, 129, 255, 0, 300]


@pytest.fixture(scope="module")
def small_plain():
    return make_model(synth.SMALL, 0)


@pytest.fixture(scope="module")
def small_perturbed():
    return make_model(synth.SMALL, 3, perturbed=True)


def oracle_out(w, cfg, x, cu):
    return oracle.forward(w, cfg, x, cu)


def check_fp32(out, ref, tol=1e-4):
    lo, rg, cl, su = out
    assert np.isfinite(lo).all() and np.isfinite(rg).all()
    e_lo = rel_err_cols(lo, ref.logits)
    e_rg = rel_err_cols(rg, ref.reg)
    assert e_lo.max() <= tol, e_lo
    assert e_rg.max() <= tol, e_rg
    assert max_scaled_err(lo, ref.logits) <= 50 * tol
    assert max_scaled_err(rg, ref.reg) <= 50 * tol


def check_lowp(out, ref, argmax_min=0.999, reg_tol=1e-2):
    lo, rg, cl, su = out
    assert np.isfinite(lo).all() and np.isfinite(rg).all()
    agree = (cl == ref.cls).mean()
    assert agree >= argmax_min, agree
    e_rg = rel_err_cols(rg, ref.reg)
    assert e_rg.max() <= reg_tol, e_rg
    return agree, e_rg


def test_fp32_one_event_256(small_plain):
    model, w = small_plain
    cfg, _, seed, sizes = synth.workload("event256")
    x, cu = synth.gen_events(seed, sizes)
    out = run_gpu(model, x, cu, "fp32")
    ref = oracle_out(w, cfg, x, cu)
    check_fp32(out, ref)
    assert (out[2] == ref.cls).all()
    np.testing.assert_allclose(out[3], ref.sums, rtol=1e-4, atol=1e-4 * np.abs(ref.sums).max())


def test_fp32_edge_sizes_perturbed(small_perturbed):
    model, w = small_perturbed
    x, cu = synth.gen_events(21, EDGE_SIZES)
    out = run_gpu(model, x, cu, "fp32")
    ref = oracle_out(w, synth.SMALL, x, cu)
    check_fp32(out, ref)
    assert out[3][EDGE_SIZES.index(0)].tolist() == [0.0, 0.0, 0.0]


def test_fp32_full_size_model():
    cfg = synth.FULL
    model, w = make_model(cfg, 1, perturbed=True)
    x, cu = synth.gen_events(102, [700, 1, 129])
    out = run_gpu(model, x, cu, "fp32")
    ref = oracle_out(w, cfg, x, cu)
    check_fp32(out, ref)


BOUNDS = {"fp16": (0.999, 1e-2), "bf16": (0.999, 1e-2)}


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_edge_sizes(small_perturbed, prec):
    model, w = small_perturbed
    x, cu = synth.gen_events(22, EDGE_SIZES + [1000, 4097])
    out = run_gpu(model, x, cu, prec)
    ref = oracle_out(w, synth.SMALL, x, cu)
    check_lowp(out, ref, *BOUNDS[prec])
    assert out[3][EDGE_SIZES.index(0)].tolist() == [0.0, 0.0, 0.0]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_prec64_subset(small_plain, prec):
    model, w = small_plain
    cfg, _, seed, sizes = synth.workload("prec64")
    x, cu = synth.gen_events(seed, sizes[:12])
    out = run_gpu(model, x, cu, prec)
    ref = oracle_out(w, cfg, x, cu)
    agree, _ = check_lowp(out, ref, *BOUNDS[prec])
    # event sums for events whose classes all agree
    for e in range(12):
        sl = slice(cu[e], cu[e + 1])
        if (out[2][sl] == ref.cls[sl]).all():
            np.testing.assert_allclose(out[3][e], ref.sums[e], rtol=0,
                                       atol=2e-2 * np.abs(ref.sums[e]).max())


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_two_blocks_per_stack(prec):
    """d=64 with 2 + 2 encoder blocks: the middle-layer kernel (out-projection, FFN,
    the next block's LayerNorm and QKV with the K-norm maxima of the attention's
    bound) runs between the two attention launches of each stack."""
    import dataclasses
    cfg = dataclasses.replace(synth.SMALL, l_pid=2, l_reg=2)
    model, w = make_model(cfg, 5, perturbed=True)
    x, cu = synth.gen_events(24, [700, 129, 1, 2000, 64])
    out = run_gpu(model, x, cu, prec)
    ref = oracle_out(w, cfg, x, cu)
    check_lowp(out, ref, *BOUNDS[prec])
    model.close()


def test_tc_full_batch_sampled(small_plain):
    """The 512-event workload in the benchmark's launch configuration; events
    sampled for the oracle (the largest, the smallest and a few in between)."""
    model, w = small_plain
    cfg, _, seed, sizes = synth.workload("batch512")
    x, cu = synth.gen_events(seed, sizes)
    order = np.argsort(sizes)
    sample = [int(order[-1]), int(order[0]), 5, 100, 300]
    ref = oracle.forward(w, cfg, x, cu, events=sample)
    for prec in ("fp16", "bf16"):
        lo, rg, cl, su = run_gpu(model, x, cu, prec)
        assert np.isfinite(lo).all() and np.isfinite(rg).all() and np.isfinite(su).all()
        rows = np.concatenate([np.arange(cu[e], cu[e + 1]) for e in sample])
        agree = (cl[rows] == ref.cls[rows]).mean()
        err = rel_err_cols(rg[rows], ref.reg[rows])
        assert agree >= BOUNDS[prec][0], (prec, agree)
        assert err.max() <= BOUNDS[prec][1], (prec, err)


def test_graphs_and_direct_launches_agree(small_perturbed):
    from paper_2601_17554_b300 import OPT_USE_GRAPHS
    model, w = small_perturbed
    x, cu = synth.gen_events(25, [333, 64, 1])
    for prec in ("fp16", "fp32"):
        a = run_gpu(model, x, cu, prec)
        model.set_option(OPT_USE_GRAPHS, 0)
        b = run_gpu(model, x, cu, prec)
        model.set_option(OPT_USE_GRAPHS, 1)
        for u, v in zip(a, b):
            np.testing.assert_array_equal(u, v)


def test_device_wait_timeout_is_reported_and_recoverable(small_perturbed):
    """A consumer waits on a barrier nothing arms: the bounded wait runs out, the
    kernel returns, mlpf_sync reports MLPF_E_TIMEOUT and the model still works."""
    from paper_2601_17554_b300 import MlpfError, OPT_DEBUG_STALL, OPT_WAIT_LIMIT_NS, _lib
    model, w = small_perturbed
    x, cu = synth.gen_events(26, [200, 50])
    model.set_option(OPT_WAIT_LIMIT_NS, 50_000_000)
    model.set_option(OPT_DEBUG_STALL, 1)
    with pytest.raises(MlpfError) as ei:
        run_gpu(model, x, cu, "fp16")
    assert ei.value.status == _lib.MLPF_E_TIMEOUT
    model.set_option(OPT_DEBUG_STALL, 0)
    model.set_option(OPT_WAIT_LIMIT_NS, 2_000_000_000)
    out = run_gpu(model, x, cu, "fp16")
    ref = oracle_out(w, synth.SMALL, x, cu)
    check_lowp(out, ref, *BOUNDS["fp16"])


def test_host_buffer_entry_point_matches_device(small_perturbed):
    import torch
    model, w = small_perturbed
    x, cu = synth.gen_events(27, [400, 90])
    dev = run_gpu(model, x, cu, "fp16")
    lo = torch.empty((len(x), 6))
    rg = torch.empty((len(x), 5))
    cl = torch.empty((len(x),), dtype=torch.int32)
    su = torch.empty((2, 3), dtype=torch.float64)
    model.forward_host(torch.from_numpy(x), torch.from_numpy(cu), 400, precision="fp16",
                       logits=lo, reg=rg, cls=cl, event_sums=su)
    np.testing.assert_array_equal(lo.numpy(), dev[0])
    np.testing.assert_array_equal(rg.numpy(), dev[1])
    np.testing.assert_array_equal(cl.numpy(), dev[2])
    np.testing.assert_array_equal(su.numpy(), dev[3])


@pytest.mark.parametrize("streams", [1, 2])
@pytest.mark.parametrize("chunks", [1, 3, 4, 16])
def test_host_chunked_pipeline_matches_device(small_perturbed, chunks, streams):
    """mlpf_forward_host on a batch above the chunking threshold: chunks of
    consecutive events with their copies overlapped by the neighbours' compute (and,
    with two compute streams, alternate chunks on a second stream and workspace) give
    the device-buffer results bitwise (an event's outputs do not depend on the
    other events)."""
    import torch
    from paper_2601_17554_b300._lib import OPT_HOST_CHUNKS, OPT_HOST_STREAMS
    model, w = small_perturbed
    sizes = synth.sizes_lognormal(31, 40)
    x, cu = synth.gen_events(31, sizes)
    assert len(x) >= 65536
    T, E = len(x), len(sizes)
    model.set_option(OPT_HOST_CHUNKS, chunks)
    model.set_option(OPT_HOST_STREAMS, streams)
    assert model.get_option(OPT_HOST_STREAMS) == streams
    try:
        for prec in ("bf16", "fp16", "fp32"):
            dev = run_gpu(model, x, cu, prec)
            xh, cuh = torch.from_numpy(x).pin_memory(), torch.from_numpy(cu).pin_memory()
            lo = torch.full((T, 6), float("nan")).pin_memory()
            rg = torch.full((T, 5), float("nan")).pin_memory()
            cl = torch.full((T,), -1, dtype=torch.int32).pin_memory()
            su = torch.full((E, 3), float("nan"), dtype=torch.float64).pin_memory()
            model.forward_host(xh, cuh, int(sizes.max()), precision=prec, logits=lo, reg=rg, cls=cl,
                               event_sums=su)
            np.testing.assert_array_equal(lo.numpy(), dev[0])
            np.testing.assert_array_equal(rg.numpy(), dev[1])
            np.testing.assert_array_equal(cl.numpy(), dev[2])
            np.testing.assert_array_equal(su.numpy(), dev[3])
    finally:
        model.set_option(OPT_HOST_CHUNKS, 8)
        model.set_option(OPT_HOST_STREAMS, 2)


def test_host_chunked_pipeline_windowed_attention(small_perturbed):
    """The chunked host pipeline with windowed attention: every chunk's forward
    reuses the eta-order, gather and scatter buffers on the same stream; the results
    equal the device-buffer forward's bitwise."""
    import torch
    from paper_2601_17554_b300._lib import OPT_ATTN_WINDOW, OPT_HOST_CHUNKS
    model, w = small_perturbed
    sizes = synth.sizes_lognormal(33, 40)
    x, cu = synth.gen_events(33, sizes)
    assert len(x) >= 65536
    T, E = len(x), len(sizes)
    model.set_option(OPT_ATTN_WINDOW, 2)
    model.set_option(OPT_HOST_CHUNKS, 5)
    try:
        dev = run_gpu(model, x, cu, "bf16")
        lo = torch.full((T, 6), float("nan")).pin_memory()
        rg = torch.full((T, 5), float("nan")).pin_memory()
        cl = torch.full((T,), -1, dtype=torch.int32).pin_memory()
        su = torch.full((E, 3), float("nan"), dtype=torch.float64).pin_memory()
        model.forward_host(torch.from_numpy(x).pin_memory(), torch.from_numpy(cu).pin_memory(), int(sizes.max()),
                           precision="bf16", logits=lo, reg=rg, cls=cl, event_sums=su)
        np.testing.assert_array_equal(lo.numpy(), dev[0])
        np.testing.assert_array_equal(rg.numpy(), dev[1])
        np.testing.assert_array_equal(cl.numpy(), dev[2])
        np.testing.assert_array_equal(su.numpy(), dev[3])
    finally:
        model.set_option(OPT_ATTN_WINDOW, 0)
        model.set_option(OPT_HOST_CHUNKS, 8)


def calibrate(model, n=32, seed=999):
    import torch
    sizes = synth.sizes_lognormal(seed, n)
    x, cu = synth.gen_events(seed, sizes)
    model.calibrate_fp8(torch.from_numpy(x).cuda(), torch.from_numpy(cu).cuda(), int(sizes.max()))


def test_fp8_needs_calibration():
    from paper_2601_17554_b300 import MlpfError, _lib
    model, w = make_model(synth.SMALL, 0)
    x, cu = synth.gen_events(28, [100])
    with pytest.raises(MlpfError) as ei:
        run_gpu(model, x, cu, "fp8")
    assert ei.value.status == _lib.MLPF_E_INVALID
    calibrate(model)
    scales = model.fp8_scales()
    assert len(scales) >= 16 and all(v > 0 for v in scales.values())
    assert np.isfinite(run_gpu(model, x, cu, "fp8")[1]).all()


# E4M3 (3 mantissa bits, unit roundoff 2^-4) in the projection and FFN GEMMs cannot meet the
# 16-bit bounds on this model: in the float64 emulation of the E4M3 roundings
# (tests/lowp_emul.py) every single E4M3 GEMM stage alone already costs 0.4-1.5 % of argmax
# agreement and 1.5-5 % regression error.  The bounds here are the emulation's prediction on
# exactly these inputs (static scales from the same 32 calibration events: 97.46 % agreement,
# 9.97 % largest column error) with 0.5 % and 10 % relative margin for the GPU's summation
# order.
FP8_BOUNDS = (0.970, 0.11)


def test_fp8_prec64_subset(small_plain):
    model, w = small_plain
    calibrate(model)
    cfg, _, seed, sizes = synth.workload("prec64")
    x, cu = synth.gen_events(seed, sizes[:12])
    out = run_gpu(model, x, cu, "fp8")
    ref = oracle_out(w, cfg, x, cu)
    agree = (out[2] == ref.cls).mean()
    err = rel_err_cols(out[1], ref.reg)
    print(f"FP8 argmax agreement {agree:.5f}, reg rel err {err}")
    assert agree >= FP8_BOUNDS[0] and err.max() <= FP8_BOUNDS[1], (agree, err)
    # deterministic
    out2 = run_gpu(model, x, cu, "fp8")
    np.testing.assert_array_equal(out[0], out2[0])


def test_fp8_two_blocks_per_stack():
    """FP8 (E4M3 projections and FFN, calibrated scales) through the middle-layer
    kernel of a d=64, 2 + 2 block model.  The float64 emulation of the E4M3 roundings
    on exactly these inputs predicts 94.64 % argmax agreement and 7.64 % largest
    column regression error (two more E4M3-quantised blocks than the 1 + 1 model);
    bounds: that prediction with 1.1 % (of 2894 elements) and 10 % relative margin."""
    import dataclasses
    cfg = dataclasses.replace(synth.SMALL, l_pid=2, l_reg=2)
    model, w = make_model(cfg, 0)
    calibrate(model)
    x, cu = synth.gen_events(25, [700, 129, 1, 2000, 64])
    out = run_gpu(model, x, cu, "fp8")
    ref = oracle_out(w, cfg, x, cu)
    agree = (out[2] == ref.cls).mean()
    err = rel_err_cols(out[1], ref.reg)
    print(f"FP8 2+2 blocks: argmax agreement {agree:.5f}, reg rel err {err}")
    assert np.isfinite(out[0]).all() and np.isfinite(out[1]).all()
    assert agree >= 0.935 and err.max() <= 0.085, (agree, err)
    model.close()


def test_bf16_deterministic_and_batch_invariant(small_perturbed):
    model, w = small_perturbed
    sizes = [500, 77, 1300, 64, 3]
    x, cu = synth.gen_events(23, sizes)
    a = run_gpu(model, x, cu, "bf16")
    b = run_gpu(model, x, cu, "bf16")
    c = run_gpu(model, x, cu, "fp16")
    assert not np.array_equal(a[0], c[0])  # the two operand formats really differ
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    # the same event alone gives bitwise the same rows
    e = 2
    xs = x[cu[e]:cu[e + 1]]
    s = run_gpu(model, xs, np.array([0, len(xs)], np.int32), "bf16")
    np.testing.assert_array_equal(s[0], a[0][cu[e]:cu[e + 1]])
    np.testing.assert_array_equal(s[1], a[1][cu[e]:cu[e + 1]])
    np.testing.assert_array_equal(s[3][0], a[3][e])


def test_fp32_deterministic(small_perturbed):
    model, w = small_perturbed
    x, cu = synth.gen_events(24, [300, 40])
    a = run_gpu(model, x, cu, "fp32")
    b = run_gpu(model, x, cu, "fp32")
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_x_alignment(precision):
    """x may start at any 8-byte boundary: a view one row (168 bytes) into a buffer gives the
    same outputs, bit for bit, as an aligned copy; an x that is not 8-byte aligned is
    rejected before anything is launched."""
    import torch
    from paper_2601_17554_b300 import MlpfError, _lib
    model, _ = make_model(synth.SMALL, 0)
    sizes = [1, 63, 64, 65, 130, 700, 0, 257]
    x, cu = synth.gen_events(45, sizes)
    ct = torch.from_numpy(cu).cuda()
    ref = run_gpu(model, x, cu, precision)
    buf = torch.zeros((len(x) + 1, 42), dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(x).cuda()
    xv = buf[1:]
    assert xv.data_ptr() % 16 == 8
    got = model.forward(xv, ct, max(sizes), precision=precision)
    model.sync()
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a.cpu().numpy(), b)
    flat = torch.zeros(len(x) * 42 + 1, dtype=torch.float32, device="cuda")
    xm = flat[1:].view(len(x), 42)
    assert xm.data_ptr() % 8 == 4
    with pytest.raises(MlpfError) as ei:
        model.forward(xm, ct, max(sizes), precision=precision)
    assert ei.value.status == _lib.MLPF_E_INVALID
    model.close()
