"""The C-ABI library builds, loads and exports every symbol include/hotrg.h declares (no GPU:
only host-side entry points are called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1906_06060_gb300 import build
    from paper_1906_06060_gb300 import _lib
    build.build()
    return _lib.load()


def declared_functions():
    with open(os.path.join(ROOT, "include", "hotrg.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hotrg_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_1906_06060_gb300 import _lib
    assert set(declared_functions()) <= set(_lib._SIGS)


def test_opts_defaults(lib):
    from paper_1906_06060_gb300 import _lib
    o = _lib.Opts()
    lib.hotrg_opts_default(ctypes.byref(o))
    assert (o.precision, o.fp64_steps, o.batch, o.max_steps) == (0, 2, 1, 64)
    assert o.wait_timeout_s == 4.0


def test_workspace_size_and_argument_checks(lib):
    from paper_1906_06060_gb300 import _lib
    n = ctypes.c_size_t()
    assert lib.hotrg_workspace_size(4, 4, None, ctypes.byref(n)) == 0
    small = n.value
    assert lib.hotrg_workspace_size(4, 10, None, ctypes.byref(n)) == 0
    big = n.value
    # T and the squeeze scratch grow like Dcut^8: Dcut=10 needs several GB, Dcut=4 far less
    assert big > 1e9 > small > 1e6
    for bad in [(0, 4), (5, 4), (4, 1), (4, 17)]:
        assert lib.hotrg_workspace_size(bad[0], bad[1], None, ctypes.byref(n)) == _lib.HOTRG_EINVAL
    assert lib.hotrg_workspace_size(4, 4, None, None) == _lib.HOTRG_EINVAL
    o = _lib.Opts()
    lib.hotrg_opts_default(ctypes.byref(o))
    o.batch = 0
    assert lib.hotrg_workspace_size(4, 4, ctypes.byref(o), ctypes.byref(n)) == _lib.HOTRG_EINVAL
    o.batch = 8
    assert lib.hotrg_workspace_size(4, 4, ctypes.byref(o), ctypes.byref(n)) == 0
    assert n.value > small  # tensors are per instance
    o.batch = 1
    o.precision = 7
    assert lib.hotrg_workspace_size(4, 4, ctypes.byref(o), ctypes.byref(n)) == _lib.HOTRG_EINVAL


def test_workspace_covers_the_block_sparse_operands(lib):
    """The block-sparse squeeze pads every operand row to round_up(P, 64) + 64 columns (its two
    k classes start at 64-aligned columns), in FP64 as in split precision: at Dcut = 10 the B
    operand alone is chi P rows of that length."""
    from paper_1906_06060_gb300 import workspace_bytes
    P, chi = 10 ** 4, 10
    ld = (P + 63) // 64 * 64 + 64
    fp64 = workspace_bytes(4, 10, "fp64", z2=True)
    bf16x3 = workspace_bytes(4, 10, "bf16x3", fp64_steps=3, z2=True)
    assert fp64 >= chi * P * ld * 8 + P * ld * 8            # Bt and Y in FP64
    assert bf16x3 >= chi * P * ld * 2 * 2 + P * ld * 2 * 2   # two bf16 planes each
    # the layout tables of the block-sparse path come on top of the dense path's needs
    assert workspace_bytes(4, 10, "bf16x3", fp64_steps=3, z2=True) >= workspace_bytes(4, 10, "bf16x3",
                                                                                       fp64_steps=3)


def test_init_rejects_bad_arguments_before_touching_a_device(lib):
    from paper_1906_06060_gb300 import _lib
    o = _lib.Opts()
    lib.hotrg_opts_default(ctypes.byref(o))
    ctx = ctypes.c_void_p()
    for d, beta, h, D in [(0, 0.1, 0, 4), (4, -0.1, 0, 4), (4, float("nan"), 0, 4), (4, 0.1, float("inf"), 4),
                          (4, 0.1, 0, 1)]:
        assert lib.hotrg_init(ctypes.byref(ctx), d, beta, h, D, ctypes.byref(o)) == _lib.HOTRG_EINVAL
    assert lib.hotrg_init(ctypes.byref(ctx), 4, 0.1, 0.0, 4, None) == _lib.HOTRG_EINVAL


def test_strerror_and_null_context(lib):
    from paper_1906_06060_gb300 import _lib
    for code in range(0, -9, -1):
        assert lib.hotrg_strerror(code)
    assert lib.hotrg_step(None, 0) == _lib.HOTRG_EINVAL
    lib.hotrg_destroy(None)
    assert lib.hotrg_gemm_scratch_bytes(0, 1, 1) == 0
    assert lib.hotrg_gemm_scratch_bytes(128, 256, 64) > 2 * (128 + 256) * 64 * 2


def test_every_context_call_rejects_a_null_context(lib):
    """No entry point dereferences a null context or null output pointers (no device needed)."""
    from paper_1906_06060_gb300 import _lib
    E = _lib.HOTRG_EINVAL
    d, n, sz = ctypes.c_double(), ctypes.c_int(), ctypes.c_size_t()
    dims = (ctypes.c_int * 4)(2, 2, 2, 2)
    buf = (ctypes.c_double * 16)()
    assert lib.hotrg_free_energy(None, ctypes.byref(d), ctypes.byref(d)) == E
    assert lib.hotrg_observables(None, 0, ctypes.byref(_lib.Obs())) == E
    assert lib.hotrg_spectra(None, 1, 0, 0, buf, 16, ctypes.byref(n)) == E
    assert lib.hotrg_ln_norms(None, 0, buf, 16, ctypes.byref(n)) == E
    assert lib.hotrg_get_tensor(None, 0, dims, buf, 16) == E
    assert lib.hotrg_set_tensor(None, 0, dims, buf) == E
    assert lib.hotrg_set_tensor_z2(None, 0, dims, dims, buf) == E
    assert lib.hotrg_state_size(None, ctypes.byref(sz)) == E
    assert lib.hotrg_state_save(None, buf, 16) == E
    assert lib.hotrg_state_load(None, buf, 16) == E
    assert lib.hotrg_timing_start(None) == E
    assert lib.hotrg_timing_stop(None, ctypes.byref(_lib.Timing())) == E
    assert lib.hotrg_autotune(None, ctypes.byref(_lib.Tuning())) == E
    assert lib.hotrg_gemm_split(None, 64, None, 64, None, 64, 128, 256, 64, 3, 64, 1, None, 0, None) == E
    assert lib.hotrg_gemm_status(None, None) == E
    assert lib.hotrg_gemm_split_noalloc(None, 64, None, 64, None, 64, 128, 256, 64, 3, None) == E


def test_product_path_fails_loudly_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("has a GPU")
    from paper_1906_06060_gb300 import HOTRG
    with pytest.raises(RuntimeError, match="CUDA device"):
        HOTRG(4, 0.1497, 0.0, 4)


def test_derivative_modes_size_the_workspace_and_reject_unknown_modes(lib):
    from paper_1906_06060_gb300 import _lib
    n = ctypes.c_size_t()
    o = _lib.Opts()
    lib.hotrg_opts_default(ctypes.byref(o))
    sizes = []
    for mode in (0, 1, 2):
        o.derivatives = mode
        assert lib.hotrg_workspace_size(4, 6, ctypes.byref(o), ctypes.byref(n)) == 0
        sizes.append(n.value)
    # tangent tensors, three operand blocks per row, and (mode 2) the Gram / isometry tangents
    assert sizes[0] < sizes[1] < sizes[2]
    for bad in (-1, 3):
        o.derivatives = bad
        assert lib.hotrg_workspace_size(4, 6, ctypes.byref(o), ctypes.byref(n)) == _lib.HOTRG_EINVAL
        ctx = ctypes.c_void_p()
        assert lib.hotrg_init(ctypes.byref(ctx), 4, 0.1, 0.0, 6, ctypes.byref(o)) == _lib.HOTRG_EINVAL


def test_autograd_entry_fails_loudly_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("has a GPU")
    from paper_1906_06060_gb300.autograd import lnz
    with pytest.raises(RuntimeError, match="CUDA device"):
        lnz(torch.tensor([0.15]), torch.tensor([0.0]), d=2, Dcut=4, nsteps=2)
    with pytest.raises(ValueError):
        lnz(torch.tensor([0.15]), torch.tensor([0.0]), mode="adjoint")
