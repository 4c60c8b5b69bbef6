"""The zero-field block-sparse squeeze (opts.z2) against the dense path and the FP64 oracle.

z2 relabels every bond index (even parity first), so tensors differ from the dense path by a
permutation of each bond; the comparisons use gauge-invariant results (ln Z/N, ln c_n, Gram
spectra, X^(n)). The blocked GEMM sums the same nonzero products as the dense one in another
order, so agreement is to FP32 rounding of the split-precision path.
"""
import json
import os

import numpy as np
import pytest

from oracle import hotrg_ref as R

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name + ".json")) as fh:
        return json.load(fh)


def hotrg(*a, **kw):
    from paper_1906_06060_gb300 import HOTRG
    return HOTRG(*a, **kw)


def run(d, beta, Dcut, nsteps, **kw):
    with hotrg(d, beta, 0.0, Dcut, max_steps=nsteps, **kw) as f:
        lnz = []
        for _ in range(nsteps):
            f.step()
            lnz.append(f.free_energy()[0][0])
        spec = [f.spectra(n, ax) for n in range(1, nsteps + 1) for ax in range(d)
                if len(f.spectra(n, ax))]
        return np.array(lnz), f.ln_norms(), spec, f.observables()


@pytest.mark.parametrize("precision,x6", [("bf16x3", 0), ("bf16x3", 8), ("bf16x6", 0), ("fp16x3", 0)])
def test_z2_matches_dense_path_dcut5(precision, x6):
    kw = dict(precision=precision, fp64_steps=2, x6_steps=x6)
    lz, cz, sz, oz = run(4, 0.1497, 5, 12, z2=True, **kw)
    ld, cd, sd, od = run(4, 0.1497, 5, 12, **kw)
    np.testing.assert_allclose(lz, ld, rtol=5e-8, atol=0)
    np.testing.assert_allclose(cz, cd, rtol=0, atol=2e-6)
    for a, b in zip(sz, sd):
        np.testing.assert_allclose(a / a[0], b / b[0], rtol=0, atol=2e-6)
    assert abs(oz["x_indicator"] - od["x_indicator"]) < 1e-5


def test_z2_flow_matches_oracle_golden_dcut5():
    """The benchmark's form of the mixed path (block-sparse, FP64 steps 1-3, BF16X6 to step 6,
    FP16X3 after) against the oracle at every step: the 1e-7 target."""
    g = golden("flow_d4_b0.1497_h0_D5_n16")
    lz, _, _, _ = run(4, 0.1497, 5, 16, z2=True, precision="fp16x3", fp64_steps=3, x6_steps=6)
    for st in g["steps"]:
        n = st["step"]
        assert abs(lz[n - 1] - st["lnz"]) < 1e-7 * abs(st["lnz"]), n


@pytest.mark.parametrize("precision", ["fp16x3", "fp16x4"])
def test_z2_fp16_flow_matches_oracle_golden_dcut5(precision):
    """fp16 planes after the FP64 steps, block-sparse: 1e-7 against the oracle at every step."""
    g = golden("flow_d4_b0.1497_h0_D5_n16")
    lz, _, _, _ = run(4, 0.1497, 5, 16, z2=True, precision=precision, fp64_steps=3, x6_steps=0)
    for st in g["steps"]:
        n = st["step"]
        assert abs(lz[n - 1] - st["lnz"]) < 1e-7 * abs(st["lnz"]), n


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3"])
def test_z2_autotune_replays_the_block_gemm_and_keeps_accuracy(precision):
    """The autotuner on the block-sparse path: it times the last chunk's two-block GEMM (its
    device descriptor) for every candidate, and the flow continues on the chosen configuration
    within the mixed path's bound against the oracle."""
    g = golden("flow_d4_b0.1497_h0_D5_n16")
    with hotrg(4, 0.1497, 0.0, 5, precision=precision, fp64_steps=3, z2=True, max_steps=16) as f:
        with pytest.raises(Exception):
            f.autotune()  # no split-precision step yet
        for _ in range(4):
            f.step()
        t = f.autotune()
        assert t["kblock"] in (32, 64) and t["group_m"] in (4, 8, 16, 32, 64) and t["fold_group"] in (1, 2)
        assert t["ms"] > 0
        for _ in range(8):
            f.step()
        lnz = f.free_energy()[0][0]
    bound = 1e-7 if precision == "fp16x3" else 3e-7   # BF16X3 alone from step 4: its own bound
    assert abs(lnz - g["steps"][11]["lnz"]) < bound * abs(lnz)


def test_z2_fp64_flow_matches_oracle_golden_dcut5():
    """Every step in FP64 through the blocked FP64 GEMM: the oracle's ln Z/N, ln c_n and Gram
    spectra to reassociation of FP64 sums."""
    g = golden("flow_d4_b0.1497_h0_D5_n16")
    with hotrg(4, 0.1497, 0.0, 5, precision="fp64", z2=True, max_steps=16) as f:
        for st in g["steps"]:
            f.step()
            n = st["step"]
            assert abs(f.free_energy()[0][0] - st["lnz"]) < 1e-12 * abs(st["lnz"]), n
            assert abs(f.observables()["x_indicator"] - st["x"]) < 1e-9, n
            lnc = f.ln_norms()
            assert abs(lnc[n] - st["ln_c"]) < 1e-12 * max(1.0, abs(st["ln_c"])), n
            for b, spec in st["spectra"].items():
                lam = f.spectra(n, int(b))
                lam = lam[: len(spec)] / lam[0]
                keep = np.array(spec) > 1e-10
                np.testing.assert_allclose(lam[keep], np.array(spec)[keep], rtol=1e-9, atol=1e-12)


def test_z2_fp64_dcut10_steps_match_dense_fp64():
    """The FP64 steps of the benchmark's flow, blocked against dense: the same products summed
    in another order. Step 3 takes bond dimensions (4, 4, 10, 10) to 10^4, the largest FP64
    squeeze of the flow (a fourth step at P = 10^4 would cost ~2e15 FP64 flops)."""
    lz, cz, sz, _ = run(4, 0.1497, 10, 3, z2=True, precision="fp64")
    ld, cd, sd, _ = run(4, 0.1497, 10, 3, precision="fp64")
    np.testing.assert_allclose(lz, ld, rtol=1e-13, atol=0)
    np.testing.assert_allclose(cz, cd, rtol=0, atol=1e-12)
    for a, b in zip(sz, sd):
        n = min(10, len(a))
        np.testing.assert_allclose(a[:n] / a[0], b[:n] / b[0], rtol=0, atol=1e-11)


def test_z2_2d_flow_matches_oracle_golden():
    """2D at Dcut = 8 (P = 64 < 256: every step takes the FP64 path, blocked): FP64 parity."""
    g = golden("flow_d2_b0.3_h0_D8_n40")
    lz, _, _, _ = run(2, 0.3, 8, 40, z2=True, precision="bf16x3", fp64_steps=3, x6_steps=12)
    for st in g["steps"]:
        assert abs(lz[st["step"] - 1] - st["lnz"]) < 1e-12 * abs(st["lnz"]), st["step"]


def test_z2_3d_flow_matches_oracle():
    # Dcut = 10: every cut of this flow is clear of degenerate multiplets (smallest gap 0.12)
    # the mixed path with the benchmark's schedule (P = 1000 from step 3: tensor cores): 1e-7
    ref = R.run(3, 0.22, 0.0, 10, 9)
    lz, _, _, _ = run(3, 0.22, 10, 9, z2=True, precision="fp16x3", fp64_steps=3, x6_steps=6)
    np.testing.assert_allclose(lz, np.array(ref.lnz[1:]), rtol=1e-7, atol=0)


@pytest.mark.parametrize("x6", [0, 12])
def test_z2_dcut10_steady_steps_match_dense(x6):
    """The benchmark's shapes: bond dimensions 10^4 from step 3 on (BF16X3 k-block 64 or BF16X6)."""
    kw = dict(precision="bf16x3", fp64_steps=2, x6_steps=x6)
    lz, cz, sz, _ = run(4, 0.1497, 10, 5, z2=True, **kw)
    ld, cd, sd, _ = run(4, 0.1497, 10, 5, **kw)
    np.testing.assert_allclose(lz, ld, rtol=5e-8, atol=0)
    np.testing.assert_allclose(cz, cd, rtol=0, atol=5e-6)
    for a, b in zip(sz, sd):
        n = min(10, len(a))
        np.testing.assert_allclose(a[:n] / a[0], b[:n] / b[0], rtol=0, atol=5e-6)


@pytest.mark.parametrize("precision,fp64_steps,x6_steps", [("fp64", 0, 0), ("bf16x3", 3, 12), ("fp16x3", 2, 0)])
def test_z2_grouped_squeeze_is_bitwise_the_instance_by_instance_squeeze(precision, fp64_steps, x6_steps):
    """Block-sparse: one GEMM launch per chunk over the group, each instance with its own parity
    counts and block descriptor (the tile list's prefix over the instances), against squeezing
    instance by instance in the same context: bit for bit."""
    betas = [0.14, 0.1497, 0.16, 0.151]
    res = []
    for group in (1, 4, 3):
        with hotrg(4, betas, 0.0, 5, precision=precision, fp64_steps=fp64_steps, x6_steps=x6_steps, z2=True,
                   group=group, max_steps=8) as f:
            for _ in range(8):
                f.step()
            res.append((f.free_energy()[0], [f.ln_norms(i) for i in range(4)], f.get_tensor(3)))
    for other in res[1:]:
        assert np.array_equal(res[0][0], other[0])
        for a, b in zip(res[0][1], other[1]):
            assert np.array_equal(a, b)
        assert np.array_equal(res[0][2], other[2])


@pytest.mark.parametrize("Dcut,precision,fp64_steps,x6_steps,batch", [(5, "fp16x3", 2, 4, 3), (8, "bf16x3", 2, 0, 1)])
def test_z2_cta_pairs_and_single_ctas_give_bitwise_identical_flows(Dcut, precision, fp64_steps, x6_steps, batch):
    """Block-sparse squeeze on CTA pairs (256-row tiles of each block, both CTAs reading their rows
    at the block's offsets) against one CTA per 128-row tile: bit for bit, over instances with their
    own block descriptors and (Dcut = 8) the benchmark's block shapes scaled down."""
    betas = [0.1497, 0.16, 0.14][:batch]
    res = []
    for cg in (2, 1):
        with hotrg(4, betas, 0.0, Dcut, precision=precision, fp64_steps=fp64_steps, x6_steps=x6_steps, z2=True,
                   group=batch, cta_group=cg, max_steps=7) as f:
            for _ in range(7 if Dcut == 5 else 5):
                f.step()
            res.append((f.free_energy()[0], [f.ln_norms(i) for i in range(batch)], f.get_tensor(batch - 1)))
    assert np.array_equal(res[0][0], res[1][0])
    for a, b in zip(res[0][1], res[1][1]):
        assert np.array_equal(a, b)
    assert np.array_equal(res[0][2], res[1][2])


def test_z2_batched_instances_match_separate_runs():
    """Each instance carries its own parity counts. Dcut = 5: no cut of these flows splits a
    degenerate multiplet (at Dcut = 6 one does, and the Gram's batch-dependent summation order
    then picks another kept subspace)."""
    betas = [0.14, 0.1497, 0.16]
    with hotrg(4, betas, 0.0, 5, precision="bf16x3", fp64_steps=2, z2=True, max_steps=8) as fb:
        for _ in range(8):
            fb.step()
        lb = fb.free_energy()[0]
    for i, b in enumerate(betas):
        with hotrg(4, b, 0.0, 5, precision="bf16x3", fp64_steps=2, z2=True, max_steps=8) as f:
            for _ in range(8):
                f.step()
            assert abs(f.free_energy()[0][0] - lb[i]) < 1e-8 * abs(lb[i])


def test_z2_graph_replay_is_bitwise_and_counts_a_quarter_of_the_flops():
    import torch
    st = torch.cuda.Stream()
    out = []
    for graphs in (False, True):
        with hotrg(4, [0.1497, 0.15], 0.0, 5, precision="bf16x3", fp64_steps=2, z2=True, graphs=graphs,
                   stream=st, max_steps=10) as f:
            for _ in range(10):
                f.step()
            out.append((f.free_energy()[0], f.ln_norms(1)))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    with hotrg(4, 0.1497, 0.0, 8, precision="bf16x3", fp64_steps=2, z2=True, max_steps=8) as f:
        for _ in range(4):
            f.step()
        f.timing_start()
        f.step()
        t = f.timing_stop()
    ratio = t["step_flops"] / t["dense_step_flops"]
    assert 0.2 < ratio < 0.3, ratio


def test_z2_argument_checks_and_set_tensor():
    from paper_1906_06060_gb300 import HotrgError
    from paper_1906_06060_gb300 import _lib
    for kw in (dict(h=1e-6), dict(derivatives="fixed"), dict(impurities=True)):
        h = kw.pop("h", 0.0)
        with pytest.raises(HotrgError) as e:
            hotrg(4, 0.1497, h, 4, z2=True, **kw)
        assert e.value.code == _lib.HOTRG_EINVAL
    # an arbitrary tensor switches the context to the dense squeeze
    from tests.inputs import random_site_tensor
    T = random_site_tensor((4, 4, 4, 4), seed=3)
    ref, _ = R.coarse_grain(T, 2, 5)
    with hotrg(4, 0.3, 0.0, 5, precision="bf16x3", fp64_steps=0, z2=True) as f:
        f.set_tensor(T)
        f.step(2)
        got = f.get_tensor()
    ref = ref / R.frobenius(ref)
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-4 * np.abs(ref).max())


def test_set_tensor_z2_checks_the_structure_and_checkpoints_keep_the_parity_counts():
    from paper_1906_06060_gb300 import HotrgError
    from paper_1906_06060_gb300 import _lib
    from tests.inputs import random_z2_site_tensor, random_site_tensor
    evens = (2, 3, 2, 2)
    T = random_z2_site_tensor((4, 5, 4, 4), evens, seed=7)
    with hotrg(4, 0.3, 0.0, 6, precision="bf16x3", fp64_steps=0, z2=True, max_steps=6) as f:
        bad = T.copy()
        bad[0, 0, 0, 3, 0, 0, 0, 0] = 1e-3          # one leg odd, all others even: odd total
        with pytest.raises(HotrgError) as e:
            f.set_tensor(bad, evens=evens)
        assert e.value.code == _lib.HOTRG_EINVAL
        f.set_tensor(T, evens=evens)
        f.step(0)
        blob = f.state_save()
        f.step(1)
        f.step(2)
        want = f.get_tensor()
        f.state_load(blob)
        f.step(1)
        f.step(2)
        assert np.array_equal(f.get_tensor(), want)
    # the dense path on the same tensor gives the same free-energy increments
    with hotrg(4, 0.3, 0.0, 6, precision="bf16x3", fp64_steps=0, max_steps=6) as g:
        g.set_tensor(T)
        for ax in (0, 1, 2):
            g.step(ax)
        with hotrg(4, 0.3, 0.0, 6, precision="bf16x3", fp64_steps=0, z2=True, max_steps=6) as f:
            f.set_tensor(T, evens=evens)
            for ax in (0, 1, 2):
                f.step(ax)
            np.testing.assert_allclose(f.ln_norms()[1:], g.ln_norms()[1:], rtol=0, atol=1e-6)
    with hotrg(4, 0.3, 0.0, 6, max_steps=6) as h:          # created without z2
        with pytest.raises(HotrgError) as e:
            h.set_tensor(T, evens=evens)
        assert e.value.code == _lib.HOTRG_ESTATE
