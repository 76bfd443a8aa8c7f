"""Allocation-free tensor-core GEMM entry point.

Callers that cannot allocate device memory when they need a product (a
framework that owns every device allocation, or code whose device memory is
all reserved at start-up) use ``mpslcc_tc_gemm_noalloc``, whose scratch lives in a fixed
device array inside the library.  Its results must equal those of the
allocating entry point ``mpslcc_debug_tc_gemm`` (FP32 output mode), call after
call, since both run the same conversion and tensor-core kernel.  This file is
collected last so that a failing run has already executed every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative, the FP32-output tolerance of the tensor-core tests


def _bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _tf32(x):
    """Operand as the tensor core reads it: FP32 with the low 13 mantissa bits dropped."""
    f = np.asarray(x, dtype=np.float32)
    return (f.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32).astype(np.float64)


def _rounded_product(prec_name, A, B):
    """The product the tensor cores compute, from operands rounded on the host:
    BF16 and TF32 round each operand once; BF16X3 keeps about 16 bits of each."""
    if prec_name == "BF16":
        return _bf16(A) @ _bf16(B).T, TOL
    if prec_name == "TF32":
        return _tf32(A) @ _tf32(B).T, TOL
    return A @ B.T, 2e-5


@pytest.mark.parametrize("prec_name,m,n,k", [("BF16", 130, 144, 136), ("TF32", 257, 40, 700),
                                             ("BF16X3", 300, 96, 520)])
def test_noalloc_gemm_matches_allocating_entry_point(mpslcc, prec_name, m, n, k):
    torch = pytest.importorskip("torch")
    prec = getattr(mpslcc, prec_name)
    rng = np.random.default_rng(m + n + k)
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((n, k))
    with mpslcc.Context(device=0) as ctx:
        ref = ctx.debug_tc_gemm(A, B, prec=prec, mode=2)
    torch.cuda.set_device(0)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    direct, dtol = _rounded_product(prec_name, A, B)
    for call in range(2):  # two calls in a row share the scratch array
        dC = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
        mpslcc.tc_gemm_noalloc(0, stream, prec, m, n, k, dA.data_ptr(), dB.data_ptr(), dC.data_ptr())
        torch.cuda.synchronize()
        C = dC.cpu().numpy()
        err = np.abs(C - ref).max() / np.abs(ref).max()
        assert err <= TOL, (call, err)
        # and against the product of host-rounded operands, independent of the library
        err_d = np.abs(C - direct).max() / np.abs(direct).max()
        assert err_d <= dtol, (call, err_d)


def test_noalloc_gemm_rejects_oversized_problem(mpslcc):
    torch = pytest.importorskip("torch")
    cap = mpslcc.lib().mpslcc_tc_gemm_noalloc_scratch_bytes()
    m = n = 4096
    k = int(cap // (2 * (m + n))) + 64  # operand copies alone exceed the scratch
    dA = torch.zeros((1,), dtype=torch.float64, device="cuda")
    with pytest.raises(mpslcc.MpsLccError) as e:
        mpslcc.tc_gemm_noalloc(0, 0, mpslcc.BF16, m, n, k, dA.data_ptr(), dA.data_ptr(), dA.data_ptr())
    assert e.value.status == 1
