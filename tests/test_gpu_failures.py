"""Failure detection through the C ABI: every failure is made on the host or by a wait limit
that runs out, never by a GPU fault.

* HOTRG_ETIMEOUT: probe launches of the tensor-core GEMM (one CTA, then a CTA pair) whose
  copy-issuing thread issues no copies, so that a wait is on data that never arrives (a short limit alone does not do it: a
  wait that the hardware lets block for a while is satisfied by real copies first). The wait
  gives up, the kernel frees its tensor memory and returns; the host reads the status word.
* HOTRG_ENUMERIC: a tensor with a NaN entry, loaded from the host (its Gram matrices and the norm
  of the next step are not finite: the eigensolver still orders the eigenvalues as a permutation
  and flags them); a tensor with a negative trace (the free energy has no logarithm).
* HOTRG_ENOCONV: an eigensolver sweep limit of one sweep on a generic Gram matrix.

Each error is sticky on its context, the context stays queryable (calls return the error
instead of failing), and the device stays usable for new contexts.
"""
import json
import math
import os

import numpy as np
import pytest

from tests.inputs import random_site_tensor, random_z2_site_tensor
from oracle import hotrg_ref as R

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _flow(*args, **kw):
    from paper_1906_06060_gb300 import HOTRG
    return HOTRG(*args, **kw)


def _fresh_context_still_matches_the_oracle():
    with open(os.path.join(GOLDEN, "flow_d4_b0.1497_h0_D5_n16.json")) as fh:
        g = json.load(fh)
    with _flow(4, 0.1497, 0.0, 5) as f:
        for _ in range(4):
            f.step()
        lnz = f.free_energy()[0][0]
    assert abs(lnz - g["steps"][3]["lnz"]) < 1e-12 * abs(lnz)


def test_wait_that_nothing_satisfies_gives_etimeout_and_a_usable_device():
    """The GEMM's bounded waits: probe launches (one CTA per tile, then a CTA pair) whose
    copy-issuing thread issues no copies, so the first wait for operand data can never be
    satisfied. Each must give up after its limit, record HOTRG_ETIMEOUT and leave the device
    usable: a normal GEMM on the same stream afterwards is correct, and so is a new flow context."""
    import torch
    from ctypes import c_void_p
    from paper_1906_06060_gb300 import _lib, gemm_split
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    nbytes = lib.hotrg_gemm_wait_probe_bytes()
    scratch = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    for limit in (0.05, 0.2):
        assert lib.hotrg_gemm_wait_probe(limit, c_void_p(scratch.data_ptr()), nbytes,
                                         c_void_p(stream.cuda_stream)) == _lib.HOTRG_ETIMEOUT
    assert lib.hotrg_gemm_wait_probe(0.0, c_void_p(scratch.data_ptr()), nbytes,
                                     c_void_p(stream.cuda_stream)) == _lib.HOTRG_EINVAL
    rng = np.random.default_rng(3)
    A = rng.standard_normal((256, 192)).astype(np.float32)
    B = rng.standard_normal((512, 192)).astype(np.float32)
    C = gemm_split(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), npass=6).cpu().numpy()
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.max(np.abs(C - ref)) < 1e-4 * np.max(np.abs(ref))
    _fresh_context_still_matches_the_oracle()


def test_nan_tensor_gives_enumeric():
    from paper_1906_06060_gb300 import HotrgError, _lib
    T = random_site_tensor((2, 2, 2, 2), seed=5)
    T[0, 1, 0, 1, 1, 0, 1, 0] = np.nan
    with _flow(4, 0.3, 0.0, 4) as f:
        f.set_tensor(T)
        f.step(3)
        with pytest.raises(HotrgError) as e:
            f.free_energy()
        assert e.value.code == _lib.HOTRG_ENUMERIC
        with pytest.raises(HotrgError) as e:
            f.step()
        assert e.value.code == _lib.HOTRG_ENUMERIC
    _fresh_context_still_matches_the_oracle()


def test_negative_trace_gives_enumeric_without_poisoning_the_flow():
    """d = 1: a step squares the site matrix; a quarter-turn rotation squares to -1, whose trace
    has no logarithm. free_energy refuses it (not sticky: the flow itself is valid), and a positive
    tensor afterwards gives a finite free energy."""
    from paper_1906_06060_gb300 import HotrgError, _lib
    with _flow(1, 0.3, 0.0, 4) as f:
        f.set_tensor(np.array([[0.0, -1.0], [1.0, 0.0]]))
        f.step(0)
        with pytest.raises(HotrgError) as e:
            f.free_energy()
        assert e.value.code == _lib.HOTRG_ENUMERIC
        f.set_tensor(np.array([[2.0, 1.0], [1.0, 2.0]]))
        f.step(0)
        lnz = f.free_energy()[0][0]
        assert math.isfinite(lnz)


def test_sweep_limit_gives_enoconv():
    from paper_1906_06060_gb300 import HotrgError, _lib
    T = random_site_tensor((3, 3, 3, 3), seed=9)
    with _flow(4, 0.3, 0.0, 9, max_sweeps=1) as f:
        f.set_tensor(T)
        f.step(0)
        with pytest.raises(HotrgError) as e:
            f.free_energy()
        assert e.value.code == _lib.HOTRG_ENOCONV
    # the default limit converges on the same matrix, and the result matches the oracle
    ref, _ = R.coarse_grain(T, 0, 9)
    with _flow(4, 0.3, 0.0, 9) as f:
        f.set_tensor(T)
        f.step(0)
        assert abs(f.ln_norms()[1] - math.log(R.frobenius(ref))) < 1e-12


def test_sweep_limit_out_of_range_is_refused():
    from paper_1906_06060_gb300 import HotrgError, _lib
    with pytest.raises(HotrgError) as e:
        _flow(4, 0.3, 0.0, 4, max_sweeps=1001)
    assert e.value.code == _lib.HOTRG_EINVAL


def test_batched_set_tensor_z2_keeps_the_dense_squeeze_while_an_instance_is_unstructured():
    """Two instances of a zero-field context: instance 0 gets an arbitrary tensor (set_tensor),
    instance 1 a block-structured one (set_tensor_z2). The context must keep squeezing densely,
    or instance 0's odd-parity entries would be dropped: both coarse-grained tensors match the
    oracle element by element. Once instance 0 is given a structured tensor too, the
    block-sparse squeeze resumes and the gauge-invariant results (ln c, spectra) still match."""
    dims, evens = (2, 2, 2, 2), (1, 1, 1, 1)
    T0 = random_site_tensor(dims, seed=21)
    T1 = random_z2_site_tensor(dims, evens, seed=22)
    with _flow(4, [0.2, 0.2], 0.0, 4, z2=True) as f:
        f.set_tensor(T0, instance=0)
        f.set_tensor(T1, instance=1, evens=evens)
        f.step(3)
        for i, T in enumerate((T0, T1)):
            ref, info = R.coarse_grain(T, 3, 4)
            ref /= R.frobenius(ref)
            got = f.get_tensor(i)
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    S0 = random_z2_site_tensor(dims, evens, seed=23)
    with _flow(4, [0.2, 0.2], 0.0, 4, z2=True) as f:
        f.set_tensor(T0, instance=0)
        f.set_tensor(T1, instance=1, evens=evens)
        f.set_tensor(S0, instance=0, evens=evens)  # now both structured: block-sparse again
        f.step(3)
        for i, T in enumerate((S0, T1)):
            ref, info = R.coarse_grain(T, 3, 4)
            assert abs(f.ln_norms(i)[1] - math.log(R.frobenius(ref))) < 1e-12
            for b, iso in info.isometries.items():
                np.testing.assert_allclose(f.spectra(1, b, i), iso.eigenvalues, rtol=0,
                                           atol=1e-12 * iso.eigenvalues[0])
