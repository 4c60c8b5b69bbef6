"""Full-size parity: one steady-state Dcut = 10 step (bond dimensions 10^4, P = 10^4, the squeeze
GEMM shapes and kernel variants the benchmark times) against the FP64 oracle on sampled slices.

The library squeezes chunk by chunk: a chunk fixes the new indices (k_1, k_2) of the first two
transverse axes, and its GEMM (M = P = 10^4 rows, N = 10 x P columns (k_3, n), K = P) computes
all 10 slices k_3 of that chunk. The samples cover the first and the last chunk, two chunks in
between, the last slice k_3 = 9 (the ragged last N-tile of the GEMM: N = 10^5 is not a multiple of
256), and, for the block-sparse squeeze, chunks of both parities (their GEMM blocks start at
rows and columns that are not tile multiples). The oracle computes the isometries of the same
input tensor and only the sampled slices (one slice = 10^5 of the 10^8 output entries) with its
slice-by-slice squeeze. The inputs are seeded Gaussian tensors: their Gram spectra are generic,
so the isometries are unique up to the sign convention both sides apply, and the comparison is
element by element (relative to the largest entry of the sampled slice).
"""
import math

import numpy as np
import pytest

from oracle import hotrg_ref as R
from tests.inputs import random_site_tensor, random_z2_site_tensor

pytestmark = pytest.mark.gpu

D = 10
A_AXIS = 0
TRANS = [1, 2, 3]
# (k_1, k_2, k_3) in the oracle's indices: first and last chunk (with the ragged last N-tile), two
# chunks in between
DENSE_SLICES = [(0, 0, 0), (D - 1, D - 1, D - 1), (3, 7, 5), (7, 2, D - 1)]
# (precision, GEMM k-block, tolerance relative to the largest sampled entry): BF16X3 with
# k-block 64 is the benchmark's steady-state step, BF16X6 with k-block 32 its six-product steps,
# FP16X3 the fp16-plane product set.
VARIANTS = [("bf16x3", 64, 2e-4), ("bf16x6", 32, 2e-6), ("fp16x3", 64, 1e-5)]


def _isometries(T):
    return {b: R.isometry_from_gram(R.gram(T, A_AXIS, b), D, D).U for b in TRANS}


@pytest.fixture(scope="module")
def dense_case():
    T = random_site_tensor((D,) * 4, seed=1010)
    ref = R.squeeze(T, T, A_AXIS, _isometries(T), slices=set(DENSE_SLICES))
    return T, ref


@pytest.mark.parametrize("precision,kblock,tol", VARIANTS)
def test_steady_dcut10_step_matches_oracle_on_sampled_chunks(dense_case, precision, kblock, tol):
    from paper_1906_06060_gb300 import HOTRG
    T, ref = dense_case
    with HOTRG(4, 0.1497, 0.0, D, precision=precision, fp64_steps=0, x6_steps=0, kblock=kblock,
               max_steps=8) as f:
        f.set_tensor(T)
        f.step(A_AXIS)
        got = f.get_tensor()
        c = math.exp(f.ln_norms()[-1])
    for k1, k2, k3 in DENSE_SLICES:
        want = ref[:, k1, k2, k3] / c          # [u_0 | p_0, p_1, p_2, p_3]
        have = got[:, k1, k2, k3]
        scale = np.abs(want).max()
        assert scale > 0
        np.testing.assert_allclose(have, want, rtol=0, atol=tol * scale, err_msg=str((k1, k2, k3)))
    # the GPU's norm is the norm of the whole output: the sampled slices carry part of it
    assert 0 < sum(np.sum((ref[:, k1, k2, k3] / c) ** 2) for k1, k2, k3 in DENSE_SLICES) < 1.0


# ------------------------------------------------------------------ the benchmark's default path
def _kept_parities(U, par):
    """Spin-flip parity of each kept vector of U (D x D x chi, fused index (x1, x2)) given the
    parities of the old bond's values: the parity of its largest component."""
    out = []
    for k in range(U.shape[2]):
        x1, x2 = np.unravel_index(np.argmax(np.abs(U[:, :, k])), U.shape[:2])
        out.append(par[x1] ^ par[x2])
    return np.array(out, dtype=int)


EVENS = (5, 4, 6, 5)   # uneven parity classes of the input bonds


@pytest.fixture(scope="module")
def z2_case():
    """The library writes every new bond even-parity first (stable in the eigenvalue order), so
    its indices are the oracle's permuted per new bond. The permutation comes from the parities of
    the oracle's kept vectors. Samples are chosen in the library's indices (chunks of both
    parities, first and last), then mapped to the oracle's."""
    T = random_z2_site_tensor((D,) * 4, EVENS, seed=2020)
    U = _isometries(T)
    par = [(np.arange(D) >= EVENS[b]).astype(int) for b in range(4)]
    sig = [np.arange(D)] + [None] * 3   # oracle index -> library index, per axis
    inv = [np.arange(D)] + [None] * 3   # library index -> oracle index
    ev = [0] * 4
    for b in TRANS:
        p = _kept_parities(U[b], par[b])
        inv[b] = np.argsort(p, kind="stable")
        sig[b] = np.argsort(inv[b], kind="stable")
        ev[b] = int(np.sum(p == 0))
    assert 0 < ev[1] < D and 0 < ev[2] < D
    # library chunks (K_1, K_2) and slices K_3: even x even, even x odd (odd chunk), odd x odd
    # (the last chunk), odd x even (odd chunk)
    lib = [(0, 0, 0), (0, ev[2], D - 1), (D - 1, D - 1, ev[3]), (ev[1], ev[2] - 1, ev[3] - 1)]
    parity = [int(K1 >= ev[1]) ^ int(K2 >= ev[2]) for K1, K2, _ in lib]
    assert parity == [0, 1, 0, 1]
    ora = [(int(inv[1][K1]), int(inv[2][K2]), int(inv[3][K3])) for K1, K2, K3 in lib]
    ref = R.squeeze(T, T, A_AXIS, U, slices=set(ora))
    return T, ref, sig, lib, ora


@pytest.mark.parametrize("precision,kblock,tol", VARIANTS)
def test_steady_dcut10_block_sparse_step_matches_oracle_on_sampled_chunks(z2_case, precision, kblock, tol):
    """The block-sparse squeeze (the benchmark's default at h = 0) at the benchmark's shapes, on a
    seeded Gaussian tensor with the zero-field block structure (bond dimensions 10^4, uneven
    parity classes), element by element on chunks of both parities."""
    from paper_1906_06060_gb300 import HOTRG
    T, ref, sig, lib, ora = z2_case
    with HOTRG(4, 0.1497, 0.0, D, precision=precision, fp64_steps=0, x6_steps=0, kblock=kblock, z2=True,
               max_steps=8) as f:
        f.set_tensor(T, evens=EVENS)
        f.step(A_AXIS)
        got = f.get_tensor()
        c = math.exp(f.ln_norms()[-1])
        # a second step runs the block-sparse path on its own output
        f.timing_start()
        f.step(3)
        t = f.timing_stop()
        assert 0.2 < t["step_flops"] / t["dense_step_flops"] < 0.3
    for (K1, K2, K3), (k1, k2, k3) in zip(lib, ora):
        want = ref[:, k1, k2, k3] / c                      # [u0 | p0, p1, p2, p3], oracle indices
        have = got[np.ix_(sig[0], [K1], [K2], [K3], sig[0], sig[1], sig[2], sig[3])].reshape(want.shape)
        scale = np.abs(want).max()
        assert scale > 0
        np.testing.assert_allclose(have, want, rtol=0, atol=tol * scale, err_msg=str((K1, K2, K3)))
