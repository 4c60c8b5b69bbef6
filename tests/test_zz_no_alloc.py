"""The no-allocation GEMM entry point, through the C ABI.

hotrg_gemm_split_noalloc serves callers that cannot allocate device memory (their memory is
reserved by another framework, or they must not call cudaMalloc in a latency-critical loop):
it keeps its operand planes in a fixed device array inside the library. These tests check that
it returns the same product as hotrg_gemm_split (which takes scratch from its caller) and as
an FP64 product of the same inputs, on two calls in a row with different shapes, so that the
second call runs on an array that still holds the first call's contents; that a request exactly
at the documented size limit (odd M and N, so the plane starts need padding) is served; and
that larger or too small requests are refused. The file is collected last.
"""
from ctypes import c_void_p

import numpy as np
import pytest

from tests.inputs import random_matrix

pytestmark = pytest.mark.gpu

LIMIT = 2 ** 21  # HOTRG_GEMM_NOALLOC_MAX_ELEMS: (M + N) * round_up(K, 64)


def _noalloc(lib, A, Bt, C, npass, stream):
    M, K = A.shape
    N = Bt.shape[0]
    return lib.hotrg_gemm_split_noalloc(c_void_p(A.data_ptr()), A.stride(0), c_void_p(Bt.data_ptr()),
                                        Bt.stride(0), c_void_p(C.data_ptr()), C.stride(0), M, N, K, npass,
                                        c_void_p(stream.cuda_stream))


def _bound(a64, b64, K, npass):
    """Elementwise bound of the split GEMM against the exact product (as in test_gpu_gemm):
    split residuals and dropped plane products per product (bf16 u = 2^-8) plus FP32
    accumulation, on |A| |Bt|^T."""
    u = 2.0 ** -8
    rel = {1: 2 * u, 3: 3 * u ** 2, 4: 2 * u ** 2, 6: 3 * u ** 3}[npass]
    return (rel + K * 2.0 ** -24) * (np.abs(a64) @ np.abs(b64).T) + 1e-30


def _check_rows(C, A, Bt, npass, rows):
    """FP64 product of the FP32 inputs on the sampled rows, within the GEMM bound."""
    a64 = A[rows].double().cpu().numpy()
    b64 = Bt.double().cpu().numpy()
    got = C[rows].double().cpu().numpy()
    ref = a64 @ b64.T
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= _bound(a64, b64, A.shape[1], npass))


def test_noalloc_gemm_matches_allocating_entry_point_and_fp64():
    import torch
    from paper_1906_06060_gb300 import build, gemm_split, _lib
    build.build()
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    for call, (M, N, K, npass) in enumerate([(384, 512, 300, 3), (257, 700, 129, 6)]):
        A = torch.from_numpy(random_matrix(M, K, seed=40 + call).astype(np.float32)).cuda()
        Bt = torch.from_numpy(random_matrix(N, K, seed=50 + call).astype(np.float32)).cuda()
        ref = gemm_split(A, Bt, npass=npass)
        C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
        assert _noalloc(lib, A, Bt, C, npass, stream) == 0
        got, want = C.cpu().numpy(), ref.cpu().numpy()
        a64, b64 = A.double().cpu().numpy(), Bt.double().cpu().numpy()
        bound = _bound(a64, b64, K, npass)
        # the same kernel on the same operands as the allocating entry point (in practice bit for
        # bit), and the exact product within the GEMM's error bound
        assert np.all(np.abs(got - want) <= bound)
        assert np.all(np.abs(got - a64 @ b64.T) <= bound)
        assert np.all(np.isfinite(got))


def test_noalloc_gemm_serves_a_request_at_the_limit():
    """(M + N) * round_up(K, 64) == 2^21 with odd M and N: each bf16 plane's start is padded to
    256 bytes, and the request must still fit the array."""
    import torch
    from paper_1906_06060_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    K = 64
    M, N = 16383, 16385
    assert (M + N) * K == LIMIT
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn((M, K), device="cuda", generator=g, dtype=torch.float32)
    Bt = torch.randn((N, K), device="cuda", generator=g, dtype=torch.float32)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for npass in (6, 3):
        assert _noalloc(lib, A, Bt, C, npass, stream) == 0
        _check_rows(C, A, Bt, npass, [0, 1, 127, 128, 8191, M - 2, M - 1])


def test_noalloc_gemm_rejects_sizes_beyond_its_array_or_below_one_tile():
    import torch
    from paper_1906_06060_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    K = 4096
    M = N = 300  # (M + N) * round_up(K, 64) = 600 * 4096 > 2^21
    A = torch.zeros((M, K), dtype=torch.float32, device="cuda")
    C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    assert _noalloc(lib, A, A, C, 3, stream) == _lib.HOTRG_EINVAL
    # one past the limit: (M + N) * 64 = 2^21 + 64
    A = torch.zeros((16384, 64), dtype=torch.float32, device="cuda")
    C = torch.zeros((16384, 16385), dtype=torch.float32, device="cuda")
    assert _noalloc(lib, A, A[:1].expand(16385, 64).contiguous(), C, 3, stream) == _lib.HOTRG_EINVAL
    # below one 128 x 256 output tile
    A = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    C = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    assert _noalloc(lib, A, A, C, 3, stream) == _lib.HOTRG_EINVAL
