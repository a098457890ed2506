"""Guard bands around every output buffer, and non-finite inputs.

compute-sanitizer is not available, so out-of-bounds writes are looked for the
other way: each output is a view into a larger buffer whose leading and trailing
rows hold a canary; after the call the canaries must be unchanged (a write past
either end of an output lands in them).  Events of awkward sizes (0, 1, 63, 64,
65, 129, a long one) put tile and block edges next to the guards.

Non-finite inputs: a NaN feature in one element of one event makes that event's
outputs NaN (attention mixes it into every element of the event), leaves every
other event's outputs bitwise unchanged (events are independent), and is
reported by the status word (MLPF_E_NONFINITE from mlpf_sync).
"""
import ctypes

import numpy as np
import pytest

import synth
from tests.util import make_model

pytestmark = pytest.mark.gpu

G = 256          # guard rows on each side
SIZES = [1, 63, 0, 64, 65, 129, 700, 2048]
F_CANARY, I_CANARY, D_CANARY = 12345.678, -7, 9.87e300


def guarded(rows, cols, dtype, canary, device="cuda", pin=False):
    """(full buffer, the view of `rows` rows in its middle)."""
    import torch
    shape = (rows + 2 * G,) + ((cols,) if cols else ())
    full = torch.full(shape, canary, dtype=dtype, device=device if not pin else "cpu")
    if pin:
        full = full.pin_memory()
    return full, full[G:G + rows]


def assert_guards(full, canary, rows):
    a = full.cpu().numpy()
    assert (a[:G] == canary).all(), "write before the output"
    assert (a[G + rows:] == canary).all(), "write after the output"


def outputs(T, E, pin=False):
    import torch
    dev = "cpu" if pin else "cuda"
    bufs = [guarded(T, 6, torch.float32, F_CANARY, dev, pin), guarded(T, 5, torch.float32, F_CANARY, dev, pin),
            guarded(T, 0, torch.int32, I_CANARY, dev, pin), guarded(E, 3, torch.float64, D_CANARY, dev, pin)]
    return bufs


def check_all(bufs, T, E):
    for (full, _), canary, rows in zip(bufs, (F_CANARY, F_CANARY, I_CANARY, D_CANARY), (T, T, T, E)):
        assert_guards(full, canary, rows)


@pytest.fixture(scope="module")
def case():
    import torch
    model, _ = make_model(synth.SMALL, 3, perturbed=True)
    x, cu = synth.gen_events(46, SIZES)
    yield model, x, cu, torch.from_numpy(x).cuda(), torch.from_numpy(cu).cuda()
    model.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_forward_writes_stay_inside_outputs(case, prec):
    model, x, cu, xt, ct = case
    T, E = len(x), len(SIZES)
    bufs = outputs(T, E)
    model.forward(xt, ct, max(SIZES), precision=prec, logits=bufs[0][1], reg=bufs[1][1], cls=bufs[2][1],
                  event_sums=bufs[3][1])
    model.sync()
    check_all(bufs, T, E)
    assert np.isfinite(bufs[1][1].cpu().numpy()).all()


def test_host_and_noalloc_writes_stay_inside_outputs(case):
    import torch
    from paper_2601_17554_b300 import _lib
    model, x, cu, xt, ct = case
    T, E = len(x), len(SIZES)
    bufs = outputs(T, E, pin=True)
    xh, cuh = torch.from_numpy(x).pin_memory(), torch.from_numpy(cu).pin_memory()
    model.forward_host(xh, cuh, max(SIZES), precision="bf16", logits=bufs[0][1], reg=bufs[1][1],
                       cls=bufs[2][1], event_sums=bufs[3][1])
    check_all(bufs, T, E)
    bufs = outputs(T, E)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    _lib.check(model.L.mlpf_forward_noalloc(model.h, _lib.MLPF_BF16, p(xt), p(ct), E, T, max(SIZES),
                                            p(bufs[0][1]), p(bufs[1][1]), p(bufs[2][1]), p(bufs[3][1]),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    model.sync()
    check_all(bufs, T, E)


def test_jet_writes_stay_inside_outputs(case):
    import torch
    from paper_2601_17554_b300 import _lib
    model, x, cu, xt, ct = case
    T, E = len(x), len(SIZES)
    _, rg, cl, _ = model.forward(xt, ct, max(SIZES), precision="bf16")
    model.sync()
    jets = guarded(T, 4, torch.float32, F_CANARY)
    nj = guarded(E, 0, torch.int32, I_CANARY)
    jof = guarded(T, 0, torch.int32, I_CANARY)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    _lib.check(model.L.mlpf_cluster_jets(model.h, p(rg), p(cl), p(ct), E, T, 0.4, p(jets[1]), p(nj[1]),
                                         p(jof[1]), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    assert_guards(jets[0], F_CANARY, T)
    assert_guards(nj[0], I_CANARY, E)
    assert_guards(jof[0], I_CANARY, T)
    # the rows past each event's jets are not written either
    n = nj[1].cpu().numpy()
    j = jets[1].cpu().numpy()
    for e in range(E):
        assert (j[cu[e] + n[e]:cu[e + 1]] == np.float32(F_CANARY)).all()


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_nan_input_is_confined_to_its_event_and_reported(case, prec):
    import torch
    from paper_2601_17554_b300 import MlpfError, _lib
    model, x, cu, xt, ct = case
    ref = [t.cpu().numpy() for t in model.forward(xt, ct, max(SIZES), precision=prec)]
    model.sync()
    bad_e = 5                                  # the 129-element event
    xb = x.copy()
    xb[cu[bad_e] + 17, 20] = np.nan
    out = model.forward(torch.from_numpy(xb).cuda(), ct, max(SIZES), precision=prec)
    with pytest.raises(MlpfError) as ei:
        model.sync()
    assert ei.value.status == _lib.MLPF_E_NONFINITE
    model.sync()                               # the status word was cleared
    lo, rg = out[0].cpu().numpy(), out[1].cpu().numpy()
    sl = slice(cu[bad_e], cu[bad_e + 1])
    assert np.isnan(lo[sl]).all() and np.isnan(rg[sl]).all()
    keep = np.ones(len(x), bool)
    keep[sl] = False
    np.testing.assert_array_equal(lo[keep], ref[0][keep])
    np.testing.assert_array_equal(rg[keep], ref[1][keep])
    np.testing.assert_array_equal(out[2].cpu().numpy()[keep], ref[2][keep])
    ev = np.arange(len(SIZES)) != bad_e
    np.testing.assert_array_equal(out[3].cpu().numpy()[ev], ref[3][ev])
