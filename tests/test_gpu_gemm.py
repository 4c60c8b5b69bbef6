"""Parity of the tcgen05 squeeze GEMM (BF16X3 split operands, FP32 accumulation) against an FP64
product of the same FP32 inputs, through the C ABI (hotrg_gemm_split)."""
import numpy as np
import pytest

from tests.inputs import random_matrix

pytestmark = pytest.mark.gpu


def _bound(A, Bt, K, npass):
    """Elementwise error bound on |A| |Bt|^T: per product the split residuals and dropped plane
    products (bf16 unit roundoff u = 2^-8: 2u for hi*hi only, 3u^2 for 3 passes, 3u^3 for 6
    passes), plus FP32 accumulation (K * 2^-24)."""
    u = 2.0 ** -8
    rel = {1: 2 * u, 3: 3 * u ** 2, 4: 2 * u ** 2, 6: 3 * u ** 3}[npass]
    return (rel + K * 2.0 ** -24) * (np.abs(A) @ np.abs(Bt).T) + 1e-30


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 700, 200), (257, 513, 129), (1000, 2560, 1000),
                                   (2048, 1024, 4096)])
@pytest.mark.parametrize("npass", [3, 1, 4, 6])
@pytest.mark.parametrize("kblock,fold_group", [(64, 0), (32, 1), (32, 2), (32, 3)])
def test_gemm_split_matches_fp64(M, N, K, npass, kblock, fold_group):
    import torch
    from paper_1906_06060_gb300 import gemm_split
    A = random_matrix(M, K, seed=M + K, scale_spread=2.0).astype(np.float32)
    Bt = random_matrix(N, K, seed=N + 7 * K).astype(np.float32)
    C = gemm_split(torch.from_numpy(A).cuda(), torch.from_numpy(Bt).cuda(), npass=npass, kblock=kblock,
                   fold_group=fold_group)
    torch.cuda.synchronize()
    got = C.cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ Bt.astype(np.float64).T
    err = np.abs(got - ref)
    bound = _bound(A.astype(np.float64), Bt.astype(np.float64), K, npass)
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3g}"
    scale = np.abs(A.astype(np.float64)) @ np.abs(Bt.astype(np.float64)).T
    if npass == 3:
        # the split must really win precision back: far better than a single bf16 pass
        assert np.max(err / scale) < 2.0 ** -14
    if npass == 6:
        # three planes: FP32-level products; accumulation restarts every k-block, so no
        # systematic drift with K
        assert np.max(err / scale) < 2.0 ** -20


@pytest.mark.parametrize("npass", [3, 6])
@pytest.mark.parametrize("kblock,fold_group", [(64, 1), (32, 1), (32, 2)])
def test_gemm_accumulation_has_no_drift_with_k(npass, kblock, fold_group):
    """All-positive operands: every partial sum has the same sign, so an accumulator that
    rounds toward zero would lose ~ (number of MMAs) x 2^-25 relative. The promoted
    accumulation keeps the mean relative error at rounding level even for K = 8192."""
    import torch
    from paper_1906_06060_gb300 import gemm_split
    M, N, K = 256, 512, 8192
    rng = np.random.default_rng(11)
    A = rng.uniform(0.5, 1.5, (M, K)).astype(np.float32)
    Bt = rng.uniform(0.5, 1.5, (N, K)).astype(np.float32)
    C = gemm_split(torch.from_numpy(A).cuda(), torch.from_numpy(Bt).cuda(), npass=npass,
                   kblock=kblock, fold_group=fold_group).cpu().numpy()
    ref = A.astype(np.float64) @ Bt.astype(np.float64).T
    rel = (C.astype(np.float64) - ref) / ref
    bias = abs(float(np.mean(rel)))
    limit = 2e-7 if npass == 6 else 1e-6
    assert bias < limit, bias


def test_gemm_strided_inputs_and_output():
    """lda/ldb/ldc larger than the logical sizes (views into bigger buffers)."""
    import torch
    from paper_1906_06060_gb300 import gemm_split
    M, N, K = 384, 512, 320
    Abig = torch.from_numpy(random_matrix(M, K + 13, seed=3).astype(np.float32)).cuda()
    Bbig = torch.from_numpy(random_matrix(N, K + 5, seed=4).astype(np.float32)).cuda()
    A, Bt = Abig[:, :K], Bbig[:, :K]
    Cbig = torch.full((M, N + 9), 7.0, dtype=torch.float32, device="cuda")
    gemm_split(A, Bt, C=Cbig[:, :N])
    torch.cuda.synchronize()
    ref = A.double().cpu().numpy() @ Bt.double().cpu().numpy().T
    got = Cbig.cpu().numpy()
    bound = _bound(A.cpu().numpy().astype(np.float64), Bt.cpu().numpy().astype(np.float64), K, 3)
    assert np.all(np.abs(got[:, :N] - ref) <= bound)
    assert np.all(got[:, N:] == 7.0)  # nothing written beyond N


def _f16_exponent(amax):
    """Scale exponent the library derives from an operand's largest magnitude: the largest e with
    amax 2^e < 2^15 (frexp convention), clamped to [-60, 60]."""
    import math
    if not amax > 0:
        return 0
    return max(-60, min(60, 15 - math.frexp(amax)[1]))


def _bound_f16(A, Bt, K, npass):
    """Elementwise bound of the fp16-plane GEMM. Each operand is scaled by 2^e (exact), split into
    fp16 hi + lo (u = 2^-11; subnormal spacing 2^-24 in scaled units). Per product: dropped plane
    products and split residuals (2u hi*hi only, 3u^2 for 3 passes, 2u^2 for 4), an absolute
    floor of 2^-24 scaled units per operand entry (2^-24-eA in A's own units), and FP32
    accumulation (K * 2^-24)."""
    u = 2.0 ** -11
    rel = {1: 2 * u, 3: 3 * u ** 2, 4: 2 * u ** 2}[npass]
    eA = _f16_exponent(float(np.abs(A).max()))
    eB = _f16_exponent(float(np.abs(Bt).max()))
    absA, absB = np.abs(A), np.abs(Bt)
    floor = (2.0 ** (-24 - eB) * absA.sum(axis=1)[:, None] + 2.0 ** (-24 - eA) * absB.sum(axis=1)[None, :])
    return (rel + K * 2.0 ** -24) * (absA @ absB.T) + floor + 1e-30


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 700, 200), (257, 513, 129), (1000, 2560, 1000)])
@pytest.mark.parametrize("npass", [3, 4, 1])
@pytest.mark.parametrize("spread,scale", [(0.0, 1.0), (2.0, 1e-4), (3.0, 3e3)])
def test_gemm_split_f16_matches_fp64(M, N, K, npass, spread, scale):
    """fp16 planes with power-of-two operand scales (FP16X3 / FP16X4): operands spanning several
    decades, far below 1 or above fp16's range before scaling."""
    import torch
    from paper_1906_06060_gb300 import gemm_split
    A = (scale * random_matrix(M, K, seed=M + 3 * K, scale_spread=spread)).astype(np.float32)
    Bt = random_matrix(N, K, seed=N + 5 * K, scale_spread=spread).astype(np.float32)
    C = gemm_split(torch.from_numpy(A).cuda(), torch.from_numpy(Bt).cuda(), npass=npass, fp16=True)
    torch.cuda.synchronize()
    got = C.cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ Bt.astype(np.float64).T
    err = np.abs(got - ref)
    bound = _bound_f16(A.astype(np.float64), Bt.astype(np.float64), K, npass)
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3g}"
    if npass >= 3 and spread == 0.0:
        # 22-bit products: far better than BF16X3's 2^-16
        rel = np.max(err / (np.abs(A.astype(np.float64)) @ np.abs(Bt.astype(np.float64)).T))
        assert rel < 2.0 ** -19, rel


def test_gemm_rejects_too_small_problem():
    import torch
    from paper_1906_06060_gb300 import gemm_split, HotrgError
    A = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(HotrgError):
        gemm_split(A, A)
