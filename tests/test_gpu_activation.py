"""The tensor-core epilogues' GELU (erf of Abramowitz & Stegun 7.1.26, |error| <=
1.5e-7, evaluated two values at a time with packed FP32x2 arithmetic and MUFU
reciprocal and exponential) against the FP32 path's GELU from CUDA erff, on device
arrays through mlpf_eval_activation (odd lengths exercise the unpaired last value).

Bound: the erf error 1.5e-7 plus about 2 ulp from the approximate reciprocal and
exponential gives |GELU_tc - GELU_f32| <= 4e-7 |x| (Phi errs by half the erf
error and GELU = x Phi); ReLU is exact in both.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _eval(impl, act, x):
    import torch
    from paper_2601_17554_b300 import _lib
    L = _lib.load()
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    _lib.check(L.mlpf_eval_activation(impl, act, ctypes.c_void_p(xd.data_ptr()),
                                      ctypes.c_void_p(yd.data_ptr()), x.size,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def test_gelu_tensor_core_form_matches_erff():
    x = np.concatenate([np.linspace(-12, 12, 2_000_001, dtype=np.float32),
                        np.array([0.0, -0.0, 1e-30, -1e-30, 1e-7, -1e-7, 3.0e38, -3.0e38], np.float32)])
    y_tc = _eval(1, 0, x).astype(np.float64)
    y_ref = _eval(0, 0, x).astype(np.float64)
    fin = np.isfinite(y_ref)
    assert np.isfinite(y_tc[fin]).all()
    err = np.abs(y_tc - y_ref)[fin]
    assert (err <= 4e-7 * np.abs(x[fin].astype(np.float64)) + 1e-37).all(), err.max()
    # closed forms: GELU(0) = 0; GELU(x) = x for large x, 0 for very negative x
    assert y_tc[x.size - 8] == 0.0
    assert y_tc[x.size - 2] == np.float32(3.0e38) and y_tc[x.size - 1] == 0.0
    # and against float64 erf (the method's own bound)
    from scipy.special import erf
    xs = x[:2_000_001].astype(np.float64)
    exact = 0.5 * xs * (1 + erf(xs / np.sqrt(2)))
    assert np.max(np.abs(y_tc[:2_000_001] - exact) - 4e-7 * np.abs(xs)) <= 1e-7


def test_odd_length_tail():
    x = np.linspace(-3, 3, 1001, dtype=np.float32)
    y = _eval(1, 0, x).astype(np.float64)
    from scipy.special import erf
    xs = x.astype(np.float64)
    exact = 0.5 * xs * (1 + erf(xs / np.sqrt(2)))
    assert np.max(np.abs(y - exact) - 4e-7 * np.abs(xs)) <= 1e-7


def test_relu_identical():
    x = np.linspace(-5, 5, 10_001, dtype=np.float32)
    np.testing.assert_array_equal(_eval(1, 1, x), np.maximum(x, 0))
    np.testing.assert_array_equal(_eval(0, 1, x), np.maximum(x, 0))


def test_bad_arguments_rejected():
    from paper_2601_17554_b300 import _lib
    L = _lib.load()
    assert L.mlpf_eval_activation(2, 0, None, None, 0, None) == _lib.MLPF_E_INVALID
    assert L.mlpf_eval_activation(0, 0, None, None, 5, None) == _lib.MLPF_E_INVALID
