"""The no-allocation GEMM entry point against the allocating one, through the C ABI.

hotrg_gemm_split_noalloc serves callers that cannot allocate device memory (their memory is
reserved by another framework, or they must not call cudaMalloc in a latency-critical loop):
it keeps its operand planes in a fixed device array inside the library. This test checks that
it returns the same product as hotrg_gemm_split (which takes scratch from its caller) on two
calls in a row, with different shapes, so the second call runs on an array that still holds
the first call's contents. It lives in a file of its own that pytest collects last.
"""
from ctypes import c_void_p

import numpy as np
import pytest

from tests.inputs import random_matrix

pytestmark = pytest.mark.gpu


def _noalloc(lib, A, Bt, C, npass, stream):
    M, K = A.shape
    N = Bt.shape[0]
    return lib.hotrg_gemm_split_noalloc(c_void_p(A.data_ptr()), A.stride(0), c_void_p(Bt.data_ptr()),
                                        Bt.stride(0), c_void_p(C.data_ptr()), C.stride(0), M, N, K, npass,
                                        c_void_p(stream.cuda_stream))


def test_noalloc_gemm_matches_allocating_entry_point():
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
        # same kernel and operands: equal within the GEMM tolerance of the other tests (in
        # practice bit for bit)
        a64, b64 = A.double().cpu().numpy(), Bt.double().cpu().numpy()
        bound = (3 * 2.0 ** -16 + K * 2.0 ** -24) * (np.abs(a64) @ np.abs(b64).T)
        assert np.all(np.abs(got - want) <= bound)
        assert np.all(np.isfinite(got))


def test_noalloc_gemm_rejects_sizes_beyond_its_array():
    import torch
    from paper_1906_06060_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    K = 4096
    M = N = 300  # (M + N) * round_up(K, 64) = 600 * 4096 > 2^21
    A = torch.zeros((M, K), dtype=torch.float32, device="cuda")
    C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    assert _noalloc(lib, A, A, C, 3, torch.cuda.current_stream()) == _lib.HOTRG_EINVAL
