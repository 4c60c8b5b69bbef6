"""Full-size parity: one steady-state Dcut = 10 step (bond dimensions 10^4, P = 10^4, the squeeze
GEMM shape and kernel variants the benchmark times) against the FP64 oracle on sampled slices.

The oracle computes the isometries of the same input tensor and a few output slices (one slice
= one tuple of new transverse indices, 10^5 of the 10^8 output entries) with its slice-by-slice
squeeze. The input is a seeded Gaussian tensor: its Gram spectra are generic, so the isometries
are unique up to the sign convention both sides apply, and the comparison is element by
element (relative to the largest entry of the sampled slices).
"""
import math

import numpy as np
import pytest

from oracle import hotrg_ref as R
from tests.inputs import random_site_tensor

pytestmark = pytest.mark.gpu

D = 10
SLICES = 2


@pytest.fixture(scope="module")
def case():
    T = random_site_tensor((D,) * 4, seed=1010)
    a = 0
    trans = [b for b in range(4) if b != a]
    U = {b: R.isometry_from_gram(R.gram(T, a, b), D, D).U for b in trans}
    ref = R.squeeze(T, T, a, U, max_slices=SLICES)
    return T, a, ref


# (precision, GEMM k-block, tolerance relative to the largest sampled entry):
# BF16X3 with k-block 64 is the benchmark's steady-state step; BF16X6 with k-block 32 its x6 steps.
@pytest.mark.parametrize("precision,kblock,tol", [("bf16x3", 64, 2e-4), ("bf16x6", 32, 2e-6)])
def test_steady_dcut10_step_matches_oracle_on_sampled_slices(case, precision, kblock, tol):
    from paper_1906_06060_gb300 import HOTRG
    T, a, ref = case
    with HOTRG(4, 0.1497, 0.0, D, precision=precision, fp64_steps=0, x6_steps=0, kblock=kblock,
               max_steps=8) as f:
        f.set_tensor(T)
        f.step(a)
        got = f.get_tensor()
        c = math.exp(f.ln_norms()[-1])
    # the first SLICES slices in the oracle's order: (k_1, k_2, k_3) = (0, 0, 0), (0, 0, 1), ...
    for s in range(SLICES):
        k3 = s % D
        want = ref[:, 0, 0, k3] / c
        have = got[:, 0, 0, k3]
        scale = np.abs(want).max()
        assert scale > 0
        np.testing.assert_allclose(have, want, rtol=0, atol=tol * scale)
    # the GPU's norm is the norm of the whole output: sampled slices carry part of it
    assert 0 < np.sum((ref[:, 0, 0, :SLICES] / c) ** 2) < 1.0
