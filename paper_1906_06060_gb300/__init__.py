"""GB300 (sm_103a) HOTRG coarse-graining of the d-dimensional Ising model (arXiv:1906.06060).

Every step of the flow runs in libhotrg.so (hand-written CUDA); this module only marshals
arguments and provides device memory and streams through PyTorch.

    from paper_1906_06060_gb300 import HOTRG
    with HOTRG(d=4, beta=0.1497, h=0.0, Dcut=10, precision="bf16x3") as flow:
        for _ in range(40):
            flow.step()
        lnz, f = flow.free_energy()
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_int, c_size_t, c_void_p

import numpy as np

from . import _lib
from ._lib import (HOTRG_BF16X3, HOTRG_BF16X4, HOTRG_BF16X6, HOTRG_FP16X3, HOTRG_FP16X4, HOTRG_FP64, HotrgError,
                   check)

__all__ = ["HOTRG", "HotrgError", "gemm_split", "workspace_bytes", "fp64_fma_tflops", "PRECISIONS"]

PRECISIONS = {"fp64": HOTRG_FP64, "bf16x3": HOTRG_BF16X3, "bf16x4": HOTRG_BF16X4, "bf16x6": HOTRG_BF16X6,
              "fp16x3": HOTRG_FP16X3, "fp16x4": HOTRG_FP16X4}
# derivative modes: isometries held fixed, or differentiated through the eigendecomposition
_DERIV = {"none": 0, "fixed": 1, "eig": 2}


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libhotrg needs a CUDA device (GB300, sm_103a); there is no CPU path")
    return torch


def _opts(precision="fp64", batch=1, fp64_steps=2, max_steps=64, wait_timeout_s=4.0, x6_steps=0, kblock=0,
          graphs=True, fold_group=0, derivatives=False, impurities=False, z2=False, max_sweeps=0, group=0,
          cta_group=0):
    lib = _lib.load()
    o = _lib.Opts()
    lib.hotrg_opts_default(byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.batch = int(batch)
    o.fp64_steps = int(fp64_steps)
    o.x6_steps = int(x6_steps)
    o.kblock = int(kblock)
    o.graphs = 1 if graphs else 0
    o.fold_group = int(fold_group)
    o.derivatives = _DERIV[derivatives] if isinstance(derivatives, str) else int(derivatives)
    o.impurities = 1 if impurities else 0
    o.z2 = 1 if z2 else 0
    o.max_steps = int(max_steps)
    o.wait_timeout_s = float(wait_timeout_s)
    o.max_sweeps = int(max_sweeps)
    o.group = int(group)
    o.cta_group = int(cta_group)
    return o


def workspace_bytes(d: int, Dcut: int, precision="fp64", batch: int = 1, fp64_steps: int = 2,
                    max_steps: int = 64, x6_steps: int = 0, derivatives=False, impurities=False,
                    z2=False, group: int = 0) -> int:
    o = _opts(precision, batch, fp64_steps, max_steps, x6_steps=x6_steps, derivatives=derivatives,
              impurities=impurities, z2=z2, group=group)
    n = c_size_t(0)
    check(_lib.load().hotrg_workspace_size(d, Dcut, byref(o), byref(n)), "hotrg_workspace_size")
    return int(n.value)


class HOTRG:
    """One HOTRG flow context (or a batch of independent (beta, h) instances).

    beta, h: scalars, or sequences of equal length `batch` for a temperature/field scan.
    precision: "fp64", "bf16x3", "bf16x4" or "bf16x6" (tensor-core squeeze with split operands);
    fp64_steps / x6_steps: precision schedule of the split modes (see include/hotrg.h).
    derivatives: False / "none", True / "fixed" (isometries held fixed) or "eig" (exact derivative
    of the truncated flow, isometries differentiated through the eigendecomposition); the
    observables then carry d(lnZ/N)/d beta, d(lnZ/N)/d h, the internal energy and magnetisation.
    impurities: also coarse-grain the impure tensors of Sec. 2; the observables then carry the
    estimates <s_i s_j> (nn_correlation) and <s_i> (spin).
    z2: zero-field block-sparse squeeze (h = 0 only; see include/hotrg.h).
    max_sweeps: Jacobi sweep limit of the eigensolver (0: the default, 40).
    group: instances squeezed together, one GEMM launch per chunk for each group (0: up to 8; the
    workspace holds that many copies of the per-step buffers).
    cta_group: CTAs per squeeze-GEMM output tile, 2 (a CTA pair, 256 x 256 tiles) or 1 (128 x 256);
    0: pairs with z2, else single CTAs, and the autotuner may change it.
    """

    def __init__(self, d: int, beta, h, Dcut: int, precision: str = "fp64", fp64_steps: int = 2,
                 max_steps: int = 64, stream=None, wait_timeout_s: float = 4.0, x6_steps: int = 0,
                 kblock: int = 0, graphs: bool = True, fold_group: int = 0, derivatives=False,
                 impurities: bool = False, z2: bool = False, max_sweeps: int = 0, group: int = 0,
                 cta_group: int = 0):
        torch = _torch()
        lib = _lib.load()
        betas = np.atleast_1d(np.asarray(beta, dtype=np.float64))
        hs = np.atleast_1d(np.asarray(h, dtype=np.float64))
        batch = max(betas.size, hs.size)
        if betas.size == 1:
            betas = np.full(batch, betas[0])
        if hs.size == 1:
            hs = np.full(batch, hs[0])
        if betas.size != batch or hs.size != batch:
            raise ValueError("beta and h must be scalars or of equal length")
        self.d, self.Dcut, self.batch, self.precision = d, Dcut, batch, precision
        self.beta = betas
        self.h = hs
        o = _opts(precision, batch, fp64_steps, max_steps, wait_timeout_s, x6_steps, kblock, graphs, fold_group,
                  derivatives, impurities, z2, max_sweeps, group, cta_group)
        n = c_size_t(0)
        check(lib.hotrg_workspace_size(d, Dcut, byref(o), byref(n)), "hotrg_workspace_size")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ws = torch.empty(int(n.value), dtype=torch.uint8, device=self.stream.device)
        self._beta_buf = (c_double * batch)(*betas)
        self._h_buf = (c_double * batch)(*hs)
        o.beta = ctypes.cast(self._beta_buf, ctypes.POINTER(c_double))
        o.h = ctypes.cast(self._h_buf, ctypes.POINTER(c_double))
        o.stream = c_void_p(self.stream.cuda_stream)
        o.workspace = c_void_p(self._ws.data_ptr())
        o.workspace_bytes = int(n.value)
        self._ctx = c_void_p()
        check(lib.hotrg_init(byref(self._ctx), d, float(betas[0]), float(hs[0]), Dcut, byref(o)), "hotrg_init")

    # -- flow ---------------------------------------------------------------------------------
    def step(self, axis: int = -1) -> None:
        check(_lib.load().hotrg_step(self._ctx, int(axis)), "hotrg_step")

    def free_energy(self):
        """(ln Z/N, f) per instance as numpy arrays."""
        lnz = (c_double * self.batch)()
        f = (c_double * self.batch)()
        check(_lib.load().hotrg_free_energy(self._ctx, lnz, f), "hotrg_free_energy")
        return np.array(lnz[:]), np.array(f[:])

    def observables(self, instance: int = 0) -> dict:
        ob = _lib.Obs()
        check(_lib.load().hotrg_observables(self._ctx, int(instance), byref(ob)), "hotrg_observables")
        return {k: getattr(ob, k) for k, _ in _lib.Obs._fields_}

    def spectra(self, step: int, axis: int, instance: int = 0) -> np.ndarray:
        buf = (c_double * 256)()
        n = c_int(0)
        check(_lib.load().hotrg_spectra(self._ctx, step, axis, instance, buf, 256, byref(n)), "hotrg_spectra")
        return np.array(buf[: n.value])

    def ln_norms(self, instance: int = 0) -> np.ndarray:
        buf = (c_double * 65)()
        n = c_int(0)
        check(_lib.load().hotrg_ln_norms(self._ctx, instance, buf, 65, byref(n)), "hotrg_ln_norms")
        return np.array(buf[: n.value])

    def step_record(self, instance: int = 0, top: int = 6) -> dict:
        """Summary of the last step of one instance, for a per-step log (one JSON object per step):
        step number n, axis, bond dimensions after the step, ln c_n, ln Z/N, X^(n), and for each
        transverse axis the leading Gram eigenvalues relative to the largest, the discarded
        weight (sum of the eigenvalues beyond the kept chi over their total) and the relative gap
        at the cut ((lam_chi - lam_chi+1) / lam_chi; null when nothing is cut). Synchronises."""
        ob = self.observables(instance)
        n, axis = ob["steps"], ob["last_axis"]
        rec = {"n": n, "axis": axis, "dims": list(self.dims()), "ln_c": ob["last_ln_c"],
               "lnz_per_site": ob["lnz_per_site"], "x": ob["x_indicator"], "cuts": {}}
        if n < 1:
            return rec
        for b, chi in enumerate(rec["dims"]):
            lam = self.spectra(n, b, instance)
            if b == axis or lam.size == 0 or lam[0] <= 0:
                continue
            lam = np.clip(lam, 0.0, None)
            total = float(lam.sum())
            cut = chi < lam.size
            rec["cuts"][str(b)] = {
                "chi": int(chi), "top": [float(x) for x in lam[:top] / lam[0]],
                "discarded_weight": float(lam[chi:].sum() / total) if cut else 0.0,
                "gap": float((lam[chi - 1] - lam[chi]) / lam[chi - 1]) if cut and lam[chi - 1] > 0 else None}
        return rec

    def dims(self) -> tuple:
        dims = (c_int * 4)()
        check(_lib.load().hotrg_get_tensor(self._ctx, 0, dims, None, 0), "hotrg_get_tensor")
        return tuple(dims[: self.d])

    def get_tensor(self, instance: int = 0) -> np.ndarray:
        dims = self.dims()
        out = np.empty(dims + dims, dtype=np.float64)
        check(_lib.load().hotrg_get_tensor(self._ctx, instance, None,
                                           out.ctypes.data_as(ctypes.POINTER(c_double)), out.size),
              "hotrg_get_tensor")
        return out

    def set_tensor(self, T: np.ndarray, instance: int = 0, evens=None) -> None:
        """Replace an instance's tensor (natural layout). evens (one count per leg, values
        ordered even-parity first) keeps the block-sparse squeeze of a context created with
        z2=True; the tensor must then have the zero-field block structure."""
        T = np.ascontiguousarray(T, dtype=np.float64)
        if T.ndim != 2 * self.d:
            raise ValueError("tensor rank must be 2d")
        dims = (c_int * 4)(*T.shape[: self.d])
        ptr = T.ctypes.data_as(ctypes.POINTER(c_double))
        if evens is None:
            check(_lib.load().hotrg_set_tensor(self._ctx, instance, dims, ptr), "hotrg_set_tensor")
        else:
            ev = (c_int * 4)(*[int(x) for x in evens])
            check(_lib.load().hotrg_set_tensor_z2(self._ctx, instance, dims, ev, ptr), "hotrg_set_tensor_z2")

    def state_save(self) -> bytes:
        lib = _lib.load()
        n = c_size_t(0)
        check(lib.hotrg_state_size(self._ctx, byref(n)), "hotrg_state_size")
        buf = ctypes.create_string_buffer(n.value)
        check(lib.hotrg_state_save(self._ctx, buf, n.value), "hotrg_state_save")
        return buf.raw

    def state_load(self, blob: bytes) -> None:
        check(_lib.load().hotrg_state_load(self._ctx, blob, len(blob)), "hotrg_state_load")

    def autotune(self) -> dict:
        """Pick the squeeze GEMM's k-block, tile raster and CTA group for the current step shape
        (call after a steady-state split-precision step)."""
        t = _lib.Tuning()
        check(_lib.load().hotrg_autotune(self._ctx, byref(t)), "hotrg_autotune")
        return {"kblock": t.kblock, "group_m": t.group_m, "fold_group": t.fold_group, "ms": t.ms,
                "cta_group": t.cta_group}

    def timing_start(self) -> None:
        check(_lib.load().hotrg_timing_start(self._ctx), "hotrg_timing_start")

    def timing_stop(self) -> dict:
        t = _lib.Timing()
        check(_lib.load().hotrg_timing_stop(self._ctx, byref(t)), "hotrg_timing_stop")
        return {k: getattr(t, k) for k, _ in _lib.Timing._fields_}

    def close(self) -> None:
        if getattr(self, "_ctx", None):
            _lib.load().hotrg_destroy(self._ctx)
            self._ctx = None
            self._ws = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gemm_split(A, Bt, npass: int = 3, C=None, stream=None, kblock: int = 0, fold_group: int = 0,
               fp16: bool = False):
    """C = A @ Bt^T through the tcgen05 kernel (A: M x K, Bt: N x K, float32 CUDA tensors);
    npass 1 / 3 / 4 / 6 selects hi*hi, BF16X3, BF16X4 or BF16X6 products; fp16=True the scaled
    fp16 planes (npass 1 / 3 / 4: hi*hi, FP16X3, FP16X4)."""
    torch = _torch()
    lib = _lib.load()
    assert A.dtype == torch.float32 and Bt.dtype == torch.float32 and A.is_cuda and Bt.is_cuda
    M, K = A.shape
    N = Bt.shape[0]
    if C is None:
        C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    stream = stream or torch.cuda.current_stream()
    nbytes = lib.hotrg_gemm_scratch_bytes(M, N, K)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=A.device)
    fn = lib.hotrg_gemm_split_f16 if fp16 else lib.hotrg_gemm_split
    check(fn(c_void_p(A.data_ptr()), A.stride(0), c_void_p(Bt.data_ptr()), Bt.stride(0),
             c_void_p(C.data_ptr()), C.stride(0), M, N, K, npass, kblock, fold_group,
             c_void_p(scratch.data_ptr()), nbytes, c_void_p(stream.cuda_stream)),
          "hotrg_gemm_split_f16" if fp16 else "hotrg_gemm_split")
    check(lib.hotrg_gemm_status(c_void_p(scratch.data_ptr()), c_void_p(stream.cuda_stream)), "gemm status")
    return C


def fp64_fma_tflops(iters: int = 1 << 14, stream=None) -> float:
    """The GPU's FP64 FMA rate in TFLOP/s (hotrg_bench_fp64_fma): the roofline denominator of
    the FP64 squeeze."""
    torch = _torch()
    stream = stream or torch.cuda.current_stream()
    sink = torch.zeros(8 * 1024, dtype=torch.float64, device=stream.device)
    out = c_double(0.0)
    check(_lib.load().hotrg_bench_fp64_fma(int(iters), c_void_p(sink.data_ptr()), byref(out),
                                           c_void_p(stream.cuda_stream)), "hotrg_bench_fp64_fma")
    return float(out.value)
