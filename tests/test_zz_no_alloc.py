"""mlpf_forward_noalloc against mlpf_forward (GPU).

The no-allocation entry point serves callers that may not allocate device
memory while they run; its scratch is a fixed device array shared by every
call.  This file is collected last so that a failing run stopped at the first
failure has already run every other test.  It passes alone in a fresh process
and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import synth
from paper_2601_17554_b300 import MlpfError, _lib, check
from tests.util import make_model

pytestmark = pytest.mark.gpu


def _call(fn_name, model, x, cu, prec, max_n):
    import torch
    T, n = x.shape[0], len(cu) - 1
    out = (torch.empty((T, 6), device="cuda"), torch.empty((T, 5), device="cuda"),
           torch.empty((T,), dtype=torch.int32, device="cuda"),
           torch.empty((n, 3), dtype=torch.float64, device="cuda"))
    xt = torch.from_numpy(x).cuda()
    ct = torch.from_numpy(cu).cuda()
    st = torch.cuda.current_stream().cuda_stream
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    fn = getattr(model.L, fn_name)
    check(fn(model.h, prec, p(xt), p(ct), n, T, max_n,
             p(out[0]), p(out[1]), p(out[2]), p(out[3]), ctypes.c_void_p(st)))
    model.sync()
    return [o.cpu().numpy() for o in out]


@pytest.mark.parametrize("prec", [_lib.MLPF_FP16, _lib.MLPF_BF16])
def test_noalloc_matches_forward_twice(prec):
    model, _ = make_model(synth.SMALL, 3, perturbed=True)
    # two different calls in a row: the shared scratch keeps the previous call's
    # contents, which must not leak into the next result
    for seed, sizes in ((41, [2000, 1, 129, 700]), (42, [64, 3000, 0, 65, 5000])):
        x, cu = synth.gen_events(seed, sizes)
        ref = _call("mlpf_forward", model, x, cu, prec, max(sizes))
        got = _call("mlpf_forward_noalloc", model, x, cu, prec, max(sizes))
        # same kernels and arithmetic: identical within the tests' tolerance
        # (they are in fact bitwise equal)
        for a, b in zip(got, ref):
            np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-6)
        assert (got[2] == ref[2]).all()
    model.close()


@pytest.mark.parametrize("variant", [0, 2, 3, 4, 5, 6, 8])
def test_noalloc_every_attention_family(variant):
    """Each attention kernel family (tcgen05 with S and P in tensor memory and its
    16-row V^T tensor map, warp-level MMAs on 128-row and on 64-row items, the latter
    with its own Q tensor map, warp-level PV with QK^T on tcgen05, warp-level QK^T
    with PV on tcgen05) through the
    no-allocation entry point, as the autotuner may leave any of them selected."""
    model, _ = make_model(synth.SMALL, 3, perturbed=True)
    model.set_option(_lib.OPT_ATTN_VARIANT_BF16, variant)
    x, cu = synth.gen_events(44, [2000, 1, 129, 700])
    ref = _call("mlpf_forward", model, x, cu, _lib.MLPF_BF16, 2000)
    got = _call("mlpf_forward_noalloc", model, x, cu, _lib.MLPF_BF16, 2000)
    for a, b in zip(got, ref):
        np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-6)
    assert (got[2] == ref[2]).all()
    model.close()


def test_noalloc_capacity_edge_and_no_device_allocation():
    """64 events and 16384 elements, sized so that the 64-row padding is near its
    largest (events of 65 and 129 elements pad to 128 and 192 rows), compared
    bitwise with the allocating forward; after a first call, further calls leave
    the device's free memory unchanged (the entry point allocates nothing)."""
    import torch
    model, _ = make_model(synth.SMALL, 3, perturbed=True)
    sizes = [65] * 32 + [129] * 31
    sizes.append(16384 - sum(sizes))
    assert len(sizes) == 64 and sum(sizes) == 16384
    x, cu = synth.gen_events(45, sizes)
    ref = _call("mlpf_forward", model, x, cu, _lib.MLPF_BF16, max(sizes))
    got = _call("mlpf_forward_noalloc", model, x, cu, _lib.MLPF_BF16, max(sizes))
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    # device-resident inputs and outputs, so that the calls below only launch kernels
    T, n = x.shape[0], len(cu) - 1
    xt = torch.from_numpy(x).cuda()
    ct = torch.from_numpy(cu).cuda()
    outs = (torch.empty((T, 6), device="cuda"), torch.empty((T, 5), device="cuda"),
            torch.empty((T,), dtype=torch.int32, device="cuda"),
            torch.empty((n, 3), dtype=torch.float64, device="cuda"))
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        check(model.L.mlpf_forward_noalloc(model.h, _lib.MLPF_BF16, p(xt), p(ct), n, T, max(sizes),
                                           *(p(o) for o in outs), st))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    model.sync()
    assert np.array_equal(outs[2].cpu().numpy(), ref[2])
    model.close()


def test_noalloc_rejects_oversize_and_fp32():
    model, _ = make_model(synth.SMALL, 0)
    x, cu = synth.gen_events(43, [16385])
    with pytest.raises(MlpfError) as ei:
        _call("mlpf_forward_noalloc", model, x, cu, _lib.MLPF_FP16, 16385)
    assert ei.value.status == _lib.MLPF_E_INVALID
    x, cu = synth.gen_events(43, [1] * 65)
    with pytest.raises(MlpfError) as ei:
        _call("mlpf_forward_noalloc", model, x, cu, _lib.MLPF_FP16, 1)
    assert ei.value.status == _lib.MLPF_E_INVALID
    x, cu = synth.gen_events(44, [10])
    with pytest.raises(MlpfError) as ei:
        _call("mlpf_forward_noalloc", model, x, cu, _lib.MLPF_FP32, 10)
    assert ei.value.status == _lib.MLPF_E_UNSUPPORTED
    model.close()
