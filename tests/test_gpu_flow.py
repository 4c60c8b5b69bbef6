"""Parity of the CUDA HOTRG flow (through the C ABI) against the FP64 CPU oracle.

Element by element where the result is unique (a single step on generic random tensors: the
isometries are fixed up to the sign convention both sides apply), and on gauge-invariant
results (ln Z/N per step, ln c_n, Gram spectra) for the Ising flows. Expected values come from
oracle/ directly or from tests/golden/*.json (written by tests/golden/make_golden.py).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import exact as E
from oracle import hotrg_ref as R
from tests.inputs import random_site_tensor

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# FP64 path: agreement up to reassociation of sums (relative to the largest entry / value)
TOL_FP64 = 1e-12
# BF16X3 path: the squeeze products carry O(2^-16) relative error before FP32 accumulation
TOL_MIXED_TENSOR = 2e-4
# FP16X3 path: O(2^-22) per product (fp16 planes of power-of-two scaled operands)
TOL_F16_TENSOR = 1e-5


def golden(name):
    with open(os.path.join(GOLDEN, name + ".json")) as fh:
        return json.load(fh)


def flow(d, beta, h, Dcut, **kw):
    from paper_1906_06060_gb300 import HOTRG
    return HOTRG(d, beta, h, Dcut, **kw)


# ------------------------------------------------------------------------- initial tensor
@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("beta,h", [(0.1497, 0.0), (0.44, 0.3), (1.0, -1e-6)])
def test_initial_tensor_and_norm(d, beta, h):
    with flow(d, beta, h, 4) as f:
        T = f.get_tensor()
        ref = R.initial_tensor(d, beta, h)
        c0 = R.frobenius(ref)
        np.testing.assert_allclose(T, ref / c0, rtol=0, atol=1e-15)
        assert abs(f.ln_norms()[0] - math.log(c0)) < 1e-14
        lnz, _ = f.free_energy()
        assert abs(lnz[0] - (math.log(c0) + math.log(R.trace(ref / c0)))) < 1e-14


# ------------------------------------------------------------------------- one step, element-wise
STEP_CASES = [
    (2, (3, 2), 1, 4), (2, (5, 4), 0, 6), (3, (2, 3, 2), 0, 3), (3, (3, 3, 2), 2, 5),
    (4, (2, 2, 2, 2), 3, 4), (4, (2, 3, 2, 2), 1, 4), (4, (3, 2, 2, 3), 0, 9), (4, (3, 3, 3, 3), 2, 5),
    (4, (4, 3, 2, 3), 3, 7),
]


def _eigvec_tolerance(info, Dcut):
    """FP64 tolerance for entries of the coarse-grained tensor, relative to its largest entry.
    Eigenvectors computed in FP64 carry an error ~ ||dG|| / gap (first-order perturbation
    theory), where ||dG|| / lambda_1 is the Gram's rounding: a few eps for each of its summation
    levels (split-K partial sums, their reduction, the Q1 Q2 combination), taken as 8 eps; the
    tolerance scales with the smallest gap among the kept eigenvalues and at the cut."""
    worst = 1.0
    for iso in info.isometries.values():
        lam = iso.eigenvalues
        k = min(iso.chi + 1, lam.size)
        gaps = -np.diff(lam[:k]) / lam[0]
        if gaps.size:
            worst = min(worst, float(gaps.min()))
    return max(TOL_FP64, 8 * 2.2e-16 / max(worst, 1e-300))


@pytest.mark.parametrize("d,dims,a,Dcut", STEP_CASES)
def test_single_step_fp64_elementwise(d, dims, a, Dcut):
    T = random_site_tensor(dims, seed=sum(dims) * 10 + a)
    ref, info = R.coarse_grain(T, a, Dcut)
    c = R.frobenius(ref)
    with flow(d, 0.3, 0.0, Dcut) as f:
        f.set_tensor(T)
        f.step(a)
        got = f.get_tensor()
        assert got.shape == ref.shape
        tol = _eigvec_tolerance(info, Dcut)
        np.testing.assert_allclose(got, ref / c, rtol=0, atol=tol * np.abs(ref / c).max())
        assert abs(f.ln_norms()[1] - math.log(c)) < 1e-12
        for b, iso in info.isometries.items():
            lam = f.spectra(1, b)
            np.testing.assert_allclose(lam, iso.eigenvalues, rtol=0, atol=1e-12 * iso.eigenvalues[0])


@pytest.mark.parametrize("d,dims,a,Dcut", [(4, (4, 4, 4, 4), 3, 8), (4, (4, 4, 4, 4), 0, 5),
                                           (2, (16, 16), 1, 16), (3, (8, 8, 5), 2, 8), (4, (5, 4, 4, 4), 1, 6)])
@pytest.mark.parametrize("precision,tol", [("bf16x3", TOL_MIXED_TENSOR), ("fp16x3", TOL_F16_TENSOR)])
def test_single_step_split_elementwise(d, dims, a, Dcut, precision, tol):
    """Tensor-core path (P >= 256, including P not a multiple of 64 and ragged tiles)."""
    T = random_site_tensor(dims, seed=sum(dims) + a)
    ref, _ = R.coarse_grain(T, a, Dcut)
    ref /= R.frobenius(ref)
    with flow(d, 0.3, 0.0, Dcut, precision=precision, fp64_steps=0) as f:
        f.set_tensor(T)
        f.step(a)
        got = f.get_tensor()
        np.testing.assert_allclose(got, ref, rtol=0, atol=tol * np.abs(ref).max())


# ------------------------------------------------------------------------- exact pins through the GPU
@pytest.mark.parametrize("beta,h", [(0.1497, 0.0), (0.3, 0.01)])
def test_gpu_4d_lossless_steps_match_enumeration(beta, h):
    with flow(4, beta, h, 16, max_steps=2) as f:
        f.step()
        lnz1 = f.free_energy()[0][0]
        f.step()
        lnz2 = f.free_energy()[0][0]
    assert abs(2 * lnz1 - E.lnz_bruteforce(beta, h, (1, 1, 1, 2))) < 1e-12
    assert abs(4 * lnz2 - E.lnz_bruteforce(beta, h, (1, 1, 2, 2))) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "bf16x3", "bf16x6", "fp16x3"])
def test_gpu_2d_4x4_matches_enumeration(precision):
    beta, h = 0.4407, 0.05
    with flow(2, beta, h, 16, precision=precision, fp64_steps=0) as f:
        for _ in range(4):
            f.step()
        lnz = f.free_energy()[0][0]
    tol = {"fp64": 1e-12, "bf16x3": 1e-6, "bf16x6": 1e-9, "fp16x3": 1e-8}[precision]
    assert abs(16 * lnz - E.lnz_bruteforce(beta, h, (4, 4))) < tol * 16


# ------------------------------------------------------------------------- Ising flows vs golden
def _compare_flow(f, g, upto, tol_lnz, tol_spec, precision_note=""):
    lnc = f.ln_norms()
    assert abs(lnc[0] - g["ln_c0"]) < 1e-13
    for st in g["steps"][:upto]:
        n = st["step"]
        assert abs(lnc[n] - st["ln_c"]) < tol_lnz * max(1.0, abs(st["ln_c"])), (n, precision_note)
        for b, spec in st["spectra"].items():
            lam = f.spectra(n, int(b))
            lam = lam[: len(spec)] / lam[0]
            keep = np.array(spec) > 1e-10
            np.testing.assert_allclose(lam[keep], np.array(spec)[keep], rtol=tol_spec, atol=tol_spec * 1e-3)


def test_fp64_flow_dcut5_16_steps_matches_oracle():
    g = golden("flow_d4_b0.1497_h0_D5_n16")
    with flow(4, 0.1497, 0.0, 5) as f:
        for st in g["steps"]:
            f.step()
            lnz = f.free_energy()[0][0]
            assert abs(lnz - st["lnz"]) < TOL_FP64 * abs(st["lnz"]), st["step"]
            assert abs(f.observables()["x_indicator"] - st["x"]) < 1e-9
        _compare_flow(f, g, 16, 1e-12, 1e-9)


def test_fp64_flow_dcut10_first_steps_match_oracle():
    """The benchmark's configuration (Dcut = 10) through the FP64 steps of its schedule (steps 1-3,
    block-sparse as the benchmark runs them, and dense): ln Z/N, ln c_n, X^(n) and the Gram
    spectra against the oracle's golden to FP64 reassociation. No cut of these steps splits a
    degenerate multiplet (the golden records the gaps)."""
    g = golden("flow_d4_b0.1497_h0_D10_n4")
    assert g["first_ambiguous_step"] is None
    for z2 in (True, False):
        with flow(4, 0.1497, 0.0, 10, precision="fp64", z2=z2, max_steps=3) as f:
            for st in g["steps"][:3]:
                f.step()
                n = st["step"]
                assert abs(f.free_energy()[0][0] - st["lnz"]) < TOL_FP64 * abs(st["lnz"]), (z2, n)
                assert abs(f.observables()["x_indicator"] - st["x"]) < 1e-9, (z2, n)
            _compare_flow(f, g, 3, 1e-12, 1e-9)


@pytest.mark.parametrize("precision,x6_steps", [("fp16x3", 6), ("bf16x3", 12), ("fp16x3", 0)])
def test_mixed_flow_dcut10_step4_within_1e7_of_oracle(precision, x6_steps):
    """The benchmark's mixed path at its own Dcut = 10 through the first steady-state step (bond
    dimensions 10^4, the benchmark's GEMM shapes, block-sparse): |delta f / f| <= 1e-7 against the
    oracle after every step, ln c_n of the split step to the accuracy its products allow."""
    g = golden("flow_d4_b0.1497_h0_D10_n4")
    with flow(4, 0.1497, 0.0, 10, precision=precision, fp64_steps=3, x6_steps=x6_steps, z2=True,
              max_steps=4) as f:
        for st in g["steps"]:
            f.step()
            lnz = f.free_energy()[0][0]
            assert abs(lnz - st["lnz"]) < 1e-7 * abs(st["lnz"]), st["step"]
        lnc = f.ln_norms()
    assert abs(lnc[4] - g["steps"][3]["ln_c"]) < 1e-6


def test_fp64_flow_dcut4_until_cut_ambiguity():
    """Dcut = 4 splits an exactly degenerate multiplet at step 3 (gap ~1e-16): the kept subspace
    is not unique from there on, so only the steps before the split are compared."""
    g = golden("flow_d4_b0.1497_h0_D4_n16")
    upto = g["first_ambiguous_step"] - 1
    assert upto == 2
    with flow(4, 0.1497, 0.0, 4) as f:
        for _ in range(16):
            f.step()
        _compare_flow(f, g, upto, 1e-12, 1e-9)
        lnz = f.free_energy()[0][0]
        # past the split both sides still land on a valid truncation of the same flow
        assert abs(lnz - g["lnz_final"]) < 1e-3


def test_fp64_flow_with_field():
    g = golden("flow_d4_b0.1497_h1e-6_D4_n8")
    with flow(4, 0.1497, 1e-6, 4) as f:
        for _ in range(2):
            f.step()
        _compare_flow(f, g, 2, 1e-12, 1e-9)


def test_fp64_2d_flow_40_steps_matches_oracle_and_onsager():
    g = golden("flow_d2_b0.3_h0_D8_n40")
    with flow(2, 0.3, 0.0, 8) as f:
        for _ in range(40):
            f.step()
        lnz = f.free_energy()[0][0]
        _compare_flow(f, g, 40, 1e-11, 1e-8)
    assert abs(lnz - g["lnz_final"]) < 1e-12 * abs(lnz)
    assert abs(lnz - E.lnz_onsager(0.3)) < 1e-6


@pytest.mark.parametrize("precision,fp64_steps,x6_steps,bound", [
    ("fp16x3", 3, 6, 1e-7),    # the mixed path: the benchmark's schedule, the 1e-7 target
    ("bf16x3", 3, 12, 1e-7),   # the same with BF16X3 after the six-product steps
    ("bf16x6", 3, 0, 1e-7),    # six-product GEMM after the FP64 steps
    ("fp16x3", 3, 0, 1e-7),    # fp16 planes (22-bit products) after the FP64 steps
    ("fp16x4", 3, 0, 1e-7),
    ("bf16x3", 2, 0, 3e-7),    # BF16X3 products alone from step 3: not the mixed path (see below)
    ("fp16x3", 2, 0, 3e-7),    # fp16 planes from step 3: not the mixed path (step 3 split)
])
def test_split_flow_dcut5_relative_free_energy(precision, fp64_steps, x6_steps, bound):
    """Split-precision flows: |delta f / f| against the FP64 oracle after every step.

    The mixed path (FP64 for steps 1-3, where the flow's early steps weigh most, six-product
    GEMMs for a few steps, three-product fp16 or bf16 GEMMs after) must meet 1e-7. BF16X3 alone
    drops the lo*lo product, which is systematic when both GEMM operands come from the same
    tensor, and a split step 3 costs about 1e-7 by itself at Dcut = 5 (measured: 1.55e-7 with
    FP16X3 from step 3); those are checked with their own bound and are not what the benchmark
    runs."""
    g = golden("flow_d4_b0.1497_h0_D5_n16")
    worst = 0.0
    with flow(4, 0.1497, 0.0, 5, precision=precision, fp64_steps=fp64_steps, x6_steps=x6_steps) as f:
        for st in g["steps"]:
            f.step()
            lnz = f.free_energy()[0][0]
            worst = max(worst, abs(lnz - st["lnz"]) / abs(st["lnz"]))
    assert worst < bound, worst


# ------------------------------------------------------------------------- batching, state, errors
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("bf16x3", 1e-8)])
def test_batched_instances_match_separate_runs(precision, tol):
    """A temperature/field scan in one context (batched Gram, eigensolver and trace launches)
    gives each instance the flow it would have alone. The split-K factor of the Gram sums
    depends on the batch size, so agreement is to rounding, not bit for bit."""
    betas = [0.14, 0.1497, 0.16]
    hs = [0.0, 1e-5, -1e-5]
    with flow(4, betas, hs, 5, precision=precision) as fb:
        for _ in range(8):
            fb.step()
        lnz_b = fb.free_energy()[0]
        x_b = [fb.observables(i)["x_indicator"] for i in range(3)]
    for i, (b, h) in enumerate(zip(betas, hs)):
        with flow(4, b, h, 5, precision=precision) as f:
            for _ in range(8):
                f.step()
            assert abs(f.free_energy()[0][0] - lnz_b[i]) < tol * abs(lnz_b[i])
            assert abs(f.observables()["x_indicator"] - x_b[i]) < 1e-6


@pytest.mark.parametrize("precision,fp64_steps,x6_steps", [("fp64", 0, 0), ("bf16x3", 2, 5), ("fp16x3", 2, 0)])
def test_grouped_squeeze_is_bitwise_the_instance_by_instance_squeeze(precision, fp64_steps, x6_steps):
    """A temperature/field scan whose squeeze GEMM runs as one launch per chunk over a group of
    instances (the tile list spans the instances, each with its own operand planes and output)
    against the same context squeezing instance by instance: every tile sums the same products in
    the same order, so the flows agree bit for bit (the batched Gram and eigensolver launches are
    the same in both)."""
    betas = [0.14, 0.1497, 0.16, 0.152, 0.145]
    hs = [0.0, 1e-5, -1e-5, 0.0, 2e-5]
    res = []
    for group in (1, 5, 2):   # 2: groups of two and a group of one
        with flow(4, betas, hs, 5, precision=precision, fp64_steps=fp64_steps, x6_steps=x6_steps,
                  group=group) as f:
            for _ in range(7):
                f.step()
            res.append((f.free_energy()[0], [f.ln_norms(i) for i in range(5)], f.get_tensor(4),
                        [f.observables(i)["x_indicator"] for i in range(5)]))
    for other in res[1:]:
        assert np.array_equal(res[0][0], other[0])
        for a, b in zip(res[0][1], other[1]):
            assert np.array_equal(a, b)
        assert np.array_equal(res[0][2], other[2])
        assert res[0][3] == other[3]


@pytest.mark.parametrize("precision,fp64_steps,x6_steps,kblock,fold_group,batch", [
    ("fp16x3", 2, 4, 64, 1, 3),   # six-product steps 3-4, then FP16X3; a group of three instances
    ("bf16x4", 2, 0, 32, 2, 1),   # four products, 32-wide stages, two per fold
    ("bf16x3", 1, 0, 32, 1, 2),
])
def test_cta_pairs_and_single_ctas_give_bitwise_identical_flows(precision, fp64_steps, x6_steps, kblock, fold_group,
                                                               batch):
    """The squeeze GEMM on CTA pairs (256 x 256 output tiles, cta_group::2 MMAs reading A rows from
    both CTAs and half of the B rows from each) against one CTA per 128 x 256 tile: every output
    element is the same sequence of K = 16 MMA steps and register folds, so the flows agree bit for
    bit, ragged tiles (P = 625 rows: the last pair tile has 113 rows, the last single tile 113)
    included."""
    betas = [0.1497, 0.16, 0.14][:batch]
    hs = [0.0, 1e-5, -2e-5][:batch]
    res = []
    for cg in (2, 1):
        with flow(4, betas, hs, 5, precision=precision, fp64_steps=fp64_steps, x6_steps=x6_steps, kblock=kblock,
                  fold_group=fold_group, cta_group=cg, group=batch) as f:
            for _ in range(6):
                f.step()
            res.append((f.free_energy()[0], [f.ln_norms(i) for i in range(batch)], f.get_tensor(batch - 1)))
    assert np.array_equal(res[0][0], res[1][0])
    for a, b in zip(res[0][1], res[1][1]):
        assert np.array_equal(a, b)
    assert np.array_equal(res[0][2], res[1][2])


def test_invalid_cta_group_is_refused():
    from paper_1906_06060_gb300 import HotrgError, _lib
    with pytest.raises(HotrgError) as e:
        flow(4, 0.15, 0.0, 4, precision="bf16x3", cta_group=3)
    assert e.value.code == _lib.HOTRG_EINVAL


def test_group_larger_than_batch_and_invalid_group():
    from paper_1906_06060_gb300 import HotrgError, _lib
    with flow(4, [0.15, 0.16], 0.0, 4, group=64) as f:  # capped at the batch
        f.step()
        assert np.all(np.isfinite(f.free_energy()[0]))
    with pytest.raises(HotrgError) as e:
        flow(4, [0.15, 0.16], 0.0, 4, group=-1)
    assert e.value.code == _lib.HOTRG_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "bf16x3"])
def test_graph_replay_matches_direct_launches(precision):
    """Steady-state steps replayed from a captured CUDA graph give bit-identical results."""
    import torch
    stream = torch.cuda.Stream()  # the legacy default stream cannot be captured
    res = []
    for graphs in (False, True):
        with flow(4, [0.1497, 0.15], 0.0, 5, precision=precision, graphs=graphs, stream=stream) as f:
            for _ in range(12):
                f.step()
            res.append((f.free_energy()[0], f.ln_norms(1), f.spectra(12, 1, 1), f.get_tensor(1)))
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


def test_checkpoint_roundtrip_is_bitwise():
    with flow(4, 0.1497, 0.0, 5) as f:
        for _ in range(5):
            f.step()
        blob = f.state_save()
        for _ in range(3):
            f.step()
        a = f.free_energy()[0][0]
        f.state_load(blob)
        assert f.observables()["steps"] == 5
        for _ in range(3):
            f.step()
        b = f.free_energy()[0][0]
    assert a == b


def test_fp64_path_is_deterministic():
    out = []
    for _ in range(2):
        with flow(4, 0.1497, 0.0, 5) as f:
            for _ in range(6):
                f.step()
            out.append(f.get_tensor())
    assert np.array_equal(out[0], out[1])


def test_error_codes():
    from paper_1906_06060_gb300 import HotrgError
    from paper_1906_06060_gb300 import _lib
    with flow(4, 0.1497, 0.0, 4, max_steps=2) as f:
        with pytest.raises(HotrgError) as e:
            f.step(4)
        assert e.value.code == _lib.HOTRG_EINVAL
        f.step()
        f.step()
        with pytest.raises(HotrgError) as e:
            f.step()
        assert e.value.code == _lib.HOTRG_ESTATE
        # the context stays usable after argument errors
        assert f.observables()["steps"] == 2
    with pytest.raises(HotrgError):
        flow(4, -0.1, 0.0, 4)
    # a tensor larger than the workspace plan's largest state is refused, not copied
    with flow(4, 0.1497, 0.0, 4, max_steps=1) as f:
        with pytest.raises(HotrgError) as e:
            f.set_tensor(np.zeros((4,) * 8))
        assert e.value.code == _lib.HOTRG_EINVAL
        f.step()


def test_gpu_x_indicator_1d_matches_transfer_matrix():
    """X^(n) on the device against the exact d = 1 value (transfer-matrix eigenvalues)."""
    beta, h = 0.5, 0.1
    with flow(1, beta, h, 4) as f:
        for n in range(1, 9):
            f.step()
            assert abs(f.observables()["x_indicator"] - E.x_1d(beta, h, 2 ** n)) < 1e-13, n


def test_autotune_picks_a_candidate_and_keeps_accuracy():
    g = golden("flow_d4_b0.1497_h0_D5_n16")
    with flow(4, 0.1497, 0.0, 5, precision="bf16x3", fp64_steps=2) as f:
        with pytest.raises(Exception):
            f.autotune()  # no split-precision step yet
        for _ in range(4):
            f.step()
        t = f.autotune()
        assert t["kblock"] in (32, 64) and t["group_m"] in (4, 8, 16, 32, 64) and t["ms"] > 0
        assert t["fold_group"] in (1, 2) and t["cta_group"] in (1, 2)
        for _ in range(4):
            f.step()
        lnz = f.free_energy()[0][0]
    # BF16X3 products alone from step 3 (the bound of that case above): tuning must not cost accuracy
    assert abs(lnz - g["steps"][7]["lnz"]) < 3e-7 * abs(lnz)
