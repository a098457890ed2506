"""The training step's tensor-core GEMM (mlpf_gemm_tc) against a float64 torch product
of the same 16-bit operands (GPU).

The operands are exactly representable in the 16-bit format, so the only differences
are the FP32 accumulation and the epilogue: each element must lie within
2^-14 sum_k |a_k b_k| (plus a few FP32 ulps of the bias and residual) of the float64
value.  A wrong row, column, K offset or swizzle gives errors of the order of the
element itself.  Shapes cover ragged M and N tails, several N tiles, N below the
MMA's minimum, one and many K stages, split-K with atomics, and every epilogue
option; the columns beyond N and the rows beyond M are never written.
"""
import math

import pytest
import torch

pytestmark = pytest.mark.gpu


def operands(seed, M, N, K, dtype, lda=None, ldb=None):
    g = torch.Generator().manual_seed(seed)
    lda, ldb = lda or K, ldb or K
    A = (torch.randn((M, lda), generator=g) * 2.0).to(dtype)
    B = (torch.randn((N, ldb), generator=g) / math.sqrt(K)).to(dtype)
    return A, B


def check(A, B, K, C, *, bias=None, R=None, act=-1, C0=None, mode=0, ldc_pad=0):
    a = A[:, :K].double().cpu()
    b = B[:, :K].double().cpu()
    ref = a @ b.T
    scale = (a.abs() @ b.abs().T)
    if bias is not None:
        ref = ref + bias.double().cpu()
    pre = ref.abs()
    if act == 1:
        ref = ref.clamp_min(0.0)
    elif act == 0:
        ref = 0.5 * ref * (1.0 + torch.special.erf(ref / math.sqrt(2.0)))
    if R is not None:
        ref = ref + R.double().cpu()
    if mode in (1, 2) and C0 is not None:
        ref = ref + C0.double().cpu()
    N = B.shape[0]
    got = C[:, :N].double().cpu()
    tol = 2.0 ** -14 * scale + 4e-7 * ref.abs() + 1e-30
    if act == 0:
        # GELU with the Abramowitz & Stegun 7.1.26 erf (|error| <= 1.5e-7): at most
        # 0.75e-7 |x|, plus the FP32 reciprocal and exponential approximations inside it
        tol = tol + 2e-7 + 2e-7 * pre
    err = (got - ref).abs()
    assert bool((err <= tol).all()), (float((err / tol).max()), err.argmax())
    if ldc_pad:
        assert bool(torch.isnan(C[:, N:]).all())


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("M,N,K", [(1, 1, 64), (130, 6, 64), (300, 64, 128), (257, 100, 320),
                                   (128, 128, 64), (500, 200, 256), (77, 256, 192), (1000, 300, 512),
                                   (3, 1024, 128)])
def test_plain_product(dtype, M, N, K):
    from paper_2601_17554_b300 import gemm_tc
    A, B = operands(M * 7 + N, M, N, K, dtype)
    A, B = A.cuda(), B.cuda()
    C = torch.full((M, N + 8), float("nan"), device="cuda")
    st = gemm_tc(A, B, C)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    check(A, B, K, C, ldc_pad=8)


@pytest.mark.parametrize("act", [-1, 0, 1])
def test_epilogue_bias_activation_residual(act):
    from paper_2601_17554_b300 import gemm_tc
    M, N, K = 333, 160, 192
    A, B = operands(11 + act, M, N, K, torch.bfloat16, lda=200, ldb=256)   # padded row strides
    A, B = A.cuda(), B.cuda()
    g = torch.Generator().manual_seed(5)
    bias = torch.randn(N, generator=g).cuda()
    R = torch.randn((M, N + 3), generator=g).cuda()
    C = torch.full((M, N), float("nan"), device="cuda")
    st = gemm_tc(A[:, :K], B[:, :K], C, bias=bias, R=R[:, :N], act=act)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    check(A, B, K, C, bias=bias, R=R[:, :N], act=act)


@pytest.mark.parametrize("kchunk", [0, 64, 128, 448])
def test_accumulate_and_split_k(kchunk):
    from paper_2601_17554_b300 import gemm_tc
    # the shape of a weight gradient: few output rows, a long reduction over elements
    M, N, K = 64, 96, 2944
    A, B = operands(3, M, N, K, torch.bfloat16)
    A, B = A.cuda(), B.cuda()
    C0 = torch.randn((M, N), generator=torch.Generator().manual_seed(9)).cuda()
    C = C0.clone()
    st = gemm_tc(A, B, C, mode=2 if kchunk else 1, kchunk=kchunk)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    check(A, B, K, C, C0=C0, mode=2)


def test_rejects_bad_arguments():
    from paper_2601_17554_b300 import MlpfError, gemm_tc
    A = torch.zeros((8, 72), dtype=torch.bfloat16, device="cuda")
    B = torch.zeros((8, 64), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((8, 8), device="cuda")
    with pytest.raises(MlpfError):      # K not a multiple of 64
        gemm_tc(A, B, C)
    with pytest.raises(MlpfError):      # A's row stride not a multiple of 8 elements
        gemm_tc(torch.zeros((8, 68), dtype=torch.bfloat16, device="cuda")[:, :64], B, C)
    with pytest.raises(MlpfError):      # kchunk not a multiple of 64
        gemm_tc(A[:, :64], B, C, mode=2, kchunk=32)
