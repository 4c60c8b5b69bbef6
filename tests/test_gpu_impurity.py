"""Parity of the CUDA impure-tensor estimates (Sec. 2, Eqs. (impTN), (SS), (ST), (energy), (spin))
against enumeration (lossless steps) and the FP64 oracle (oracle.hotrg_ref.impurity_flow)."""
import json
import os

import numpy as np
import pytest

from oracle import exact as E
from oracle import hotrg_ref as R

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def flow(d, beta, h, Dcut, **kw):
    from paper_1906_06060_gb300 import HOTRG
    return HOTRG(d, beta, h, Dcut, impurities=True, **kw)


def est(f, i=0):
    o = f.observables(i)
    return o["nn_correlation"], o["spin"]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("bf16x6", 1e-9), ("bf16x3", 1e-6)])
def test_2d_4x4_lossless_matches_enumeration(precision, tol):
    beta, h = 0.4407, 0.05
    with flow(2, beta, h, 16, precision=precision, fp64_steps=0) as f:
        nn0, s0 = est(f)
        assert np.isnan(nn0)
        pe, ps = E.pair_and_spin_bruteforce(beta, h, (1, 1), 1)
        assert abs(s0 - ps) < 1e-14
        for n, L in ((1, (1, 2)), (2, (2, 2)), (3, (2, 4)), (4, (4, 4))):
            f.step()
            pe, ps = E.pair_and_spin_bruteforce(beta, h, L, 1)
            nn, sp = est(f)
            assert abs(nn - pe) < tol and abs(sp - ps) < tol, n


def test_4d_lossless_matches_enumeration():
    beta, h = 0.3, 0.01
    with flow(4, beta, h, 16, max_steps=2) as f:
        for n, L in ((1, (1, 1, 1, 2)), (2, (1, 1, 2, 2))):
            f.step()
            pe, ps = E.pair_and_spin_bruteforce(beta, h, L, 3)
            nn, sp = est(f)
            assert abs(nn - pe) < 1e-12 and abs(sp - ps) < 1e-12, n


@pytest.mark.parametrize("beta,h", [(0.1497, 0.0), (0.16, 0.01)])
def test_4d_dcut3_matches_oracle(beta, h):
    nsteps = 12
    ref = R.impurity_flow(4, beta, h, 3, nsteps)
    gaps = R.run(4, beta, h, 3, nsteps).gaps
    last = next((n for n, g in enumerate(gaps) if g and min(g.values()) < 1e-8), nsteps)
    with flow(4, beta, h, 3, max_steps=nsteps) as f:
        for n in range(1, last + 1):
            f.step()
            nn, sp = est(f)
            assert abs(nn - ref.nn[n - 1]) < 1e-10, n
            assert abs(sp - ref.spin[n]) < 1e-10, n


@pytest.mark.parametrize("precision,fp64_steps,x6_steps,tol", [("fp64", 0, 0, 1e-11), ("bf16x3", 3, 12, 1e-6)])
def test_4d_dcut5_matches_golden(precision, fp64_steps, x6_steps, tol):
    with open(os.path.join(GOLDEN, "impurity_d4_b0.16_h0.01_D5_n8.json")) as fh:
        g = json.load(fh)
    c = g["config"]
    with flow(4, c["beta"], c["h"], c["Dcut"], precision=precision, fp64_steps=fp64_steps, x6_steps=x6_steps,
              max_steps=c["nsteps"]) as f:
        for n in range(1, c["nsteps"] + 1):
            f.step()
            nn, sp = est(f)
            assert abs(nn - g["nn"][n - 1]) < tol and abs(sp - g["spin"][n]) < tol, n


def test_zero_field_spin_vanishes_and_flow_is_unchanged():
    from paper_1906_06060_gb300 import HOTRG
    with flow(4, 0.1497, 0.0, 5, max_steps=8) as f, HOTRG(4, 0.1497, 0.0, 5, max_steps=8) as g:
        for _ in range(8):
            f.step()
            g.step()
            assert abs(est(f)[1]) < 1e-14
            assert 0 < est(f)[0] < 1
        assert f.free_energy()[0][0] == g.free_energy()[0][0]
        assert np.isnan(g.observables()["spin"])


def test_batched_impurities_match_separate_runs():
    betas, hs = [0.14, 0.1497, 0.16], [0.0, 1e-5, -1e-5]
    with flow(4, betas, hs, 5, max_steps=6) as fb:
        for _ in range(6):
            fb.step()
        got = [est(fb, i) for i in range(3)]
    for i, (b, h) in enumerate(zip(betas, hs)):
        with flow(4, b, h, 5, max_steps=6) as f:
            for _ in range(6):
                f.step()
            want = est(f)
        assert abs(got[i][0] - want[0]) < 1e-11 and abs(got[i][1] - want[1]) < 1e-11


def test_graph_replay_and_checkpoint_with_impurities_and_derivatives():
    import torch
    st = torch.cuda.Stream()
    out = []
    for graphs in (False, True):
        with flow(4, [0.1497, 0.15], 1e-5, 5, precision="bf16x3", fp64_steps=1, max_steps=10, stream=st,
                  graphs=graphs, derivatives="eig") as f:
            for _ in range(6):
                f.step()
            blob = f.state_save()
            for _ in range(4):
                f.step()
            o = f.observables(1)
            out.append((est(f, 0), est(f, 1), o["dlnz_dbeta"], o["dlnz_dh"]))
            f.state_load(blob)
            for _ in range(4):
                f.step()
            o = f.observables(1)
            assert (est(f, 0), est(f, 1), o["dlnz_dbeta"], o["dlnz_dh"]) == out[-1]
    assert out[0] == out[1]
