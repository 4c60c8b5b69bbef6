"""Parity of the CUDA derivative flow (forward-mode tangents with the isometries held fixed)
against exact results and the FP64 oracle.

Exact pins: d = 1 (every step exact; the differentiated transfer matrix) and lossless steps in
2D and 4D (thermal averages by enumeration). Truncated flows: the oracle's frozen-isometry
difference quotients (oracle.hotrg_ref.fixed_isometry_derivatives, directly at Dcut = 3 and
from tests/golden/deriv_*.json at Dcut = 5).
"""
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
    return HOTRG(d, beta, h, Dcut, derivatives=True, **kw)


def derivs(f, instance=0):
    o = f.observables(instance)
    return o["dlnz_dbeta"], o["dlnz_dh"], o


@pytest.mark.parametrize("beta,h", [(0.7, 0.2), (0.44, 0.0), (1.1, -0.05)])
def test_d1_matches_transfer_matrix_every_step(beta, h):
    with flow(1, beta, h, 2, max_steps=24) as f:
        for n in range(0, 21):
            if n:
                f.step()
            db, dh, o = derivs(f)
            rb, rh = E.dlnz_1d(beta, h, 2 ** n)
            assert abs(db - rb) < 1e-13 * max(1.0, abs(rb)), n
            assert abs(dh - rh) < 1e-13 * max(1.0, abs(rh)), n
            assert o["internal_energy"] == -db
            assert abs(o["magnetization"] - dh / beta) < 1e-16


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("bf16x6", 1e-9), ("bf16x3", 1e-6)])
def test_2d_4x4_lossless_matches_enumeration(precision, tol):
    beta, h = 0.4407, 0.05
    with flow(2, beta, h, 16, precision=precision, fp64_steps=0) as f:
        for n in range(1, 5):
            f.step()
            if n in (2, 4):
                L = (2, 2) if n == 2 else (4, 4)
                e, m = E.moments_bruteforce(beta, h, L)
                db, dh, _ = derivs(f)
                assert abs(db - (e + h * m)) < tol, n
                assert abs(dh - beta * m) < tol, n


@pytest.mark.parametrize("beta,h", [(0.1497, 0.0), (0.3, 0.01)])
def test_4d_lossless_steps_match_enumeration(beta, h):
    with flow(4, beta, h, 16, max_steps=2) as f:
        for n, L in ((1, (1, 1, 1, 2)), (2, (1, 1, 2, 2))):
            f.step()
            e, m = E.moments_bruteforce(beta, h, L)
            db, dh, _ = derivs(f)
            assert abs(db - (e + h * m)) < 1e-12, n
            assert abs(dh - beta * m) < 1e-12, n


@pytest.mark.parametrize("beta,h", [(0.1497, 0.0), (0.16, 0.01)])
def test_4d_dcut3_matches_oracle_fixed_isometry_difference_quotients(beta, h):
    nsteps = 12
    db_ref, dh_ref = R.fixed_isometry_derivatives(4, beta, h, 3, nsteps)
    # steps whose cut splits an exactly degenerate pair leave the kept subspace (and with it the
    # frozen flow) implementation-dependent: compare the steps before the first such cut
    gaps = R.run(4, beta, h, 3, nsteps).gaps
    last = next((n for n, g in enumerate(gaps) if g and min(g.values()) < 1e-8), nsteps)
    assert last >= 8
    with flow(4, beta, h, 3, max_steps=nsteps) as f:
        for n in range(1, last + 1):
            f.step()
            db, dh, _ = derivs(f)
            # the difference quotients carry ~1e-11 (Richardson, eps = 1e-3)
            assert abs(db - db_ref[n]) < 1e-9 * max(1.0, abs(db_ref[n])), n
            assert abs(dh - dh_ref[n]) < 1e-9 * max(1.0, abs(dh_ref[n])), n


@pytest.mark.parametrize("name", ["deriv_d4_b0.1497_h0_D5_n8", "deriv_d4_b0.16_h0.01_D5_n8"])
@pytest.mark.parametrize("precision,fp64_steps,x6_steps,tol", [
    ("fp64", 0, 0, 1e-9),        # bounded by the difference quotients of the golden values
    ("bf16x6", 0, 0, 1e-6),      # every squeeze split, FP32 accumulation: ~2e-7 .. 9e-7 measured
    ("bf16x3", 3, 12, 1e-6),     # the mixed path with BF16X6 to step 12 (tangent squeezes use bf16 planes)
    ("bf16x3", 0, 0, 1e-5),      # every squeeze with three bf16 products: ~4e-6 measured
])
def test_4d_dcut5_matches_golden(name, precision, fp64_steps, x6_steps, tol):
    """Tolerances are absolute below |value| = 1 and relative above (the tangents go through
    the same split-precision squeeze as the flow, and d ln c = <T, D>/c^2 does not benefit from
    the insensitivity of ln c to errors orthogonal to T)."""
    with open(os.path.join(GOLDEN, name + ".json")) as fh:
        g = json.load(fh)
    c = g["config"]
    with flow(4, c["beta"], c["h"], c["Dcut"], precision=precision, fp64_steps=fp64_steps,
              x6_steps=x6_steps, max_steps=c["nsteps"]) as f:
        for n in range(1, c["nsteps"] + 1):
            f.step()
            db, dh, _ = derivs(f)
            assert abs(db - g["dlnz_dbeta"][n]) < tol * max(1.0, abs(g["dlnz_dbeta"][n])), n
            assert abs(dh - g["dlnz_dh"][n]) < tol * max(1.0, abs(g["dlnz_dh"][n])), n


def test_zero_field_magnetization_vanishes():
    """Z2 symmetry: at h = 0 the h-tangent is odd, the flow even, and <s> = 0 at every step."""
    with flow(4, 0.1497, 0.0, 5, max_steps=10) as f:
        for _ in range(10):
            f.step()
            _, dh, o = derivs(f)
            assert abs(dh) < 1e-13 and abs(o["magnetization"]) < 1e-12


def test_derivatives_off_report_nan_and_leave_the_flow_unchanged():
    from paper_1906_06060_gb300 import HOTRG
    with HOTRG(4, 0.1497, 0.0, 4, max_steps=6) as a, flow(4, 0.1497, 0.0, 4, max_steps=6) as b:
        for _ in range(6):
            a.step()
            b.step()
        oa, ob = a.observables(), b.observables()
        assert np.isnan(oa["dlnz_dbeta"]) and np.isnan(oa["magnetization"])
        assert oa["lnz_per_site"] == ob["lnz_per_site"]


def test_batched_derivatives_match_separate_runs():
    from paper_1906_06060_gb300 import HOTRG
    # Dcut = 5 keeps every cut of these flows clear of degenerate multiplets; the Gram split-K
    # factor depends on the batch size, so agreement is to rounding
    betas, hs = [0.14, 0.1497, 0.16], [0.0, 1e-5, -1e-5]
    with HOTRG(4, betas, hs, 5, max_steps=8, derivatives=True) as fb:
        for _ in range(8):
            fb.step()
        got = [derivs(fb, i)[:2] for i in range(3)]
    for i, (b, h) in enumerate(zip(betas, hs)):
        with flow(4, b, h, 5, max_steps=8) as f:
            for _ in range(8):
                f.step()
            want = derivs(f)[:2]
        assert abs(got[i][0] - want[0]) < 1e-10 and abs(got[i][1] - want[1]) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "bf16x3"])
def test_graph_replay_with_derivatives_is_bitwise(precision):
    import torch
    from paper_1906_06060_gb300 import HOTRG
    st = torch.cuda.Stream()
    out = []
    for graphs in (False, True):
        with HOTRG(4, [0.1497, 0.15], 1e-5, 5, precision=precision, fp64_steps=1, max_steps=10, stream=st,
                   graphs=graphs, derivatives=True) as f:
            for _ in range(10):
                f.step()
            out.append([derivs(f, i)[:2] for i in range(2)])
    assert out[0] == out[1]


def test_checkpoint_roundtrip_keeps_tangents():
    from paper_1906_06060_gb300 import HOTRG
    with flow(4, 0.1497, 0.01, 4, max_steps=8) as a:
        for _ in range(3):
            a.step()
        blob = a.state_save()
        for _ in range(3):
            a.step()
        want = derivs(a)[:2]
    with flow(4, 0.1497, 0.01, 4, max_steps=8) as b:
        b.state_load(blob)
        for _ in range(3):
            b.step()
        assert derivs(b)[:2] == want
    with HOTRG(4, 0.1497, 0.01, 4, max_steps=8) as c:
        with pytest.raises(RuntimeError):
            c.state_load(blob)          # saved with tangents, loaded without


# ------------------------------------------------------------------ derivatives through the isometries
def eig_flow(d, beta, h, Dcut, **kw):
    from paper_1906_06060_gb300 import HOTRG
    return HOTRG(d, beta, h, Dcut, derivatives="eig", **kw)


@pytest.mark.parametrize("beta,h", [(0.7, 0.2)])
def test_eig_mode_d1_matches_transfer_matrix(beta, h):
    with eig_flow(1, beta, h, 2, max_steps=16) as f:
        for n in range(1, 17):
            f.step()
            db, dh, _ = derivs(f)
            rb, rh = E.dlnz_1d(beta, h, 2 ** n)
            assert abs(db - rb) < 1e-13 * max(1.0, abs(rb)) and abs(dh - rh) < 1e-13 * max(1.0, abs(rh))


def test_eig_mode_2d_lossless_matches_enumeration():
    beta, h = 0.4407, 0.05
    with eig_flow(2, beta, h, 16) as f:
        for _ in range(4):
            f.step()
        e, m = E.moments_bruteforce(beta, h, (4, 4))
        db, dh, _ = derivs(f)
        assert abs(db - (e + h * m)) < 1e-12 and abs(dh - beta * m) < 1e-12


@pytest.mark.parametrize("beta,h,Dcut,nsteps", [(0.4407, 0.01, 8, 16), (0.3, 0.05, 4, 20)])
def test_eig_mode_2d_truncated_matches_oracle_flow_difference_quotients(beta, h, Dcut, nsteps):
    fb, fh = R.flow_derivatives(2, beta, h, Dcut, nsteps)
    gaps = R.run(2, beta, h, Dcut, nsteps).gaps
    last = next((n for n, g in enumerate(gaps) if g and min(g.values()) < 1e-8), nsteps)
    assert last >= 8
    with eig_flow(2, beta, h, Dcut, max_steps=nsteps) as f:
        for n in range(1, last + 1):
            f.step()
            db, dh, _ = derivs(f)
            assert abs(db - fb[n]) < 1e-8 * max(1.0, abs(fb[n])), n
            assert abs(dh - fh[n]) < 1e-8 * max(1.0, abs(fh[n])), n


@pytest.mark.parametrize("beta,h", [(0.1497, 0.0), (0.16, 0.01)])
def test_eig_mode_4d_dcut3_matches_oracle_flow_difference_quotients(beta, h):
    nsteps = 12
    fb, fh = R.flow_derivatives(4, beta, h, 3, nsteps)
    gaps = R.run(4, beta, h, 3, nsteps).gaps
    last = next((n for n, g in enumerate(gaps) if g and min(g.values()) < 1e-8), nsteps)
    with eig_flow(4, beta, h, 3, max_steps=nsteps) as f:
        for n in range(1, last + 1):
            f.step()
            db, dh, _ = derivs(f)
            assert abs(db - fb[n]) < 1e-8 * max(1.0, abs(fb[n])), n
            assert abs(dh - fh[n]) < 1e-8 * max(1.0, abs(fh[n])), n


@pytest.mark.parametrize("name", ["deriv_d4_b0.1497_h0_D5_n8", "deriv_d4_b0.16_h0.01_D5_n8"])
@pytest.mark.parametrize("precision,fp64_steps,x6_steps,tol", [
    ("fp64", 0, 0, 1e-8),        # bounded by the difference quotients of the golden values
    ("bf16x3", 3, 12, 1e-6),     # the mixed path with BF16X6 to step 12 (tangent squeezes use bf16 planes)
])
def test_eig_mode_4d_dcut5_matches_golden(name, precision, fp64_steps, x6_steps, tol):
    with open(os.path.join(GOLDEN, name + ".json")) as fh:
        g = json.load(fh)
    c = g["config"]
    with eig_flow(4, c["beta"], c["h"], c["Dcut"], precision=precision, fp64_steps=fp64_steps,
                  x6_steps=x6_steps, max_steps=c["nsteps"]) as f:
        for n in range(1, c["nsteps"] + 1):
            f.step()
            db, dh, _ = derivs(f)
            assert abs(db - g["flow_dlnz_dbeta"][n]) < tol * max(1.0, abs(g["flow_dlnz_dbeta"][n])), n
            assert abs(dh - g["flow_dlnz_dh"][n]) < tol * max(1.0, abs(g["flow_dlnz_dh"][n])), n


@pytest.mark.parametrize("mode,tol_fp64", [("fixed", 1e-9), ("eig", 1e-8)])
@pytest.mark.parametrize("precision,fp64_steps,x6_steps,tol_split", [
    ("fp64", 0, 0, None),
    ("bf16x3", 2, 12, 1e-6),     # step 3 through the six-product GEMM
    ("bf16x3", 2, 0, 1e-5),      # step 3 with three bf16 products
])
def test_4d_dcut10_first_steps_match_golden(mode, tol_fp64, precision, fp64_steps, x6_steps, tol_split):
    """The differentiation workload's point (beta = 0.1497, h = 1e-6) at its Dcut = 10, through the
    first three steps (the third makes every bond 10, P = 1600 -> 10^4; one steady step more
    would be 2e15 flops per oracle run): d(lnZ/N)/d beta and d / d h with the isometries held
    fixed and differentiated through the eigendecomposition, against the oracle's difference
    quotients; the FP64 path to the quotients' accuracy, the split paths (step 3 on the tensor
    cores) within their bounds."""
    with open(os.path.join(GOLDEN, "deriv_d4_b0.1497_h1e-6_D10_n3.json")) as fh:
        g = json.load(fh)
    c = g["config"]
    kb, kh = ("dlnz_dbeta", "dlnz_dh") if mode == "fixed" else ("flow_dlnz_dbeta", "flow_dlnz_dh")
    tol = tol_fp64 if precision == "fp64" else tol_split
    from paper_1906_06060_gb300 import HOTRG
    with HOTRG(4, c["beta"], c["h"], c["Dcut"], derivatives=mode, precision=precision, fp64_steps=fp64_steps,
               x6_steps=x6_steps, max_steps=c["nsteps"]) as f:
        for n in range(1, c["nsteps"] + 1):
            f.step()
            db, dh, _ = derivs(f)
            assert abs(db - g[kb][n]) < tol * max(1.0, abs(g[kb][n])), n
            assert abs(dh - g[kh][n]) < tol * max(1.0, abs(g[kh][n])), n


def test_eig_mode_graph_replay_is_bitwise():
    import torch
    from paper_1906_06060_gb300 import HOTRG
    st = torch.cuda.Stream()
    out = []
    for graphs in (False, True):
        with HOTRG(4, [0.1497, 0.15], 1e-5, 5, precision="bf16x3", fp64_steps=1, max_steps=10, stream=st,
                   graphs=graphs, derivatives="eig") as f:
            for _ in range(10):
                f.step()
            out.append([derivs(f, i)[:2] for i in range(2)])
    assert out[0] == out[1]


# ------------------------------------------------------------------ torch.autograd
@pytest.mark.parametrize("mode", ["eig", "fixed"])
def test_autograd_function_returns_the_library_derivatives(mode):
    import torch
    from paper_1906_06060_gb300.autograd import lnz
    beta = torch.tensor([0.1497, 0.16], dtype=torch.float64, requires_grad=True)
    h = torch.tensor([0.0, 0.01], dtype=torch.float64, requires_grad=True)
    y = lnz(beta, h, d=4, Dcut=5, nsteps=8, mode=mode)
    gb, gh = torch.autograd.grad(y.sum(), (beta, h))
    for i, name in enumerate(["deriv_d4_b0.1497_h0_D5_n8", "deriv_d4_b0.16_h0.01_D5_n8"]):
        with open(os.path.join(GOLDEN, name + ".json")) as fh:
            g = json.load(fh)
        kb, kh = ("flow_dlnz_dbeta", "flow_dlnz_dh") if mode == "eig" else ("dlnz_dbeta", "dlnz_dh")
        assert abs(float(y.detach()[i]) - g["lnz"][8]) < 1e-12 * abs(g["lnz"][8])
        assert abs(float(gb[i]) - g[kb][8]) < 1e-8 and abs(float(gh[i]) - g[kh][8]) < 1e-8


def test_autograd_eig_mode_matches_gpu_finite_differences():
    """The derivative of the flow against central differences of the GPU's own FP64 free energy
    (step 1e-5, as the differentiation workload asks), 2D Dcut = 8, 20 steps."""
    import torch
    from paper_1906_06060_gb300 import HOTRG
    from paper_1906_06060_gb300.autograd import lnz
    b0, h0, eps = 0.4407, 0.01, 1e-5
    beta = torch.tensor([b0], dtype=torch.float64, requires_grad=True)
    h = torch.tensor([h0], dtype=torch.float64, requires_grad=True)
    y = lnz(beta, h, d=2, Dcut=8, nsteps=20, mode="eig")
    gb, gh = torch.autograd.grad(y.sum(), (beta, h))

    def f(b, hh):
        with HOTRG(2, b, hh, 8, max_steps=20) as fl:
            for _ in range(20):
                fl.step()
            return fl.free_energy()[0][0]

    fd_b = (f(b0 + eps, h0) - f(b0 - eps, h0)) / (2 * eps)
    fd_h = (f(b0, h0 + eps) - f(b0, h0 - eps)) / (2 * eps)
    # FD error: eps^2 f''' / 6 plus ~1e-16 / eps rounding of the FP64 flow
    assert abs(float(gb[0]) - fd_b) < 1e-6 and abs(float(gh[0]) - fd_h) < 1e-6
