"""ln Z/N of the HOTRG flow as a differentiable function of (beta, h) for torch.autograd.

    import torch
    from paper_1906_06060_gb300.autograd import lnz
    beta = torch.tensor([0.1494, 0.1497, 0.1500], dtype=torch.float64, requires_grad=True)
    h = torch.full((3,), 1e-6, dtype=torch.float64, requires_grad=True)
    y = lnz(beta, h, d=4, Dcut=10, nsteps=40, precision="bf16x3", fp64_steps=3, x6_steps=12)
    E_per_site = -torch.autograd.grad(y.sum(), beta, retain_graph=True)[0]
    M = torch.autograd.grad(y.sum(), h)[0] / beta

The library computes the derivatives alongside the flow: every step carries the tangents
d/d beta and d/d h of the tensor (forward mode; with two parameters this costs the same as a
reverse sweep and needs no per-step checkpoints of the forward pass), so backward() only
scales them by the incoming gradient. mode="eig" differentiates the isometries through the
Gram eigendecomposition (the derivative of the truncated flow itself); mode="fixed" holds
them at their values at (beta, h) (Sec. 2's isometries treated as constants).
"""
from __future__ import annotations

import numpy as np

from . import HOTRG


class LnZ:
    """Namespace for the autograd Function (built lazily so that importing this module does not
    import torch)."""

    _fn = None

    @classmethod
    def function(cls):
        if cls._fn is None:
            import torch

            class _LnZ(torch.autograd.Function):
                @staticmethod
                def forward(ctx, beta, h, d, Dcut, nsteps, mode, kw):
                    b = beta.detach().cpu().double().numpy().reshape(-1)
                    hh = h.detach().cpu().double().numpy().reshape(-1)
                    with HOTRG(d, b, hh, Dcut, max_steps=max(1, nsteps), derivatives=mode, **kw) as flow:
                        for _ in range(nsteps):
                            flow.step()
                        lnz_v, _ = flow.free_energy()
                        obs = [flow.observables(i) for i in range(flow.batch)]
                    db = np.array([o["dlnz_dbeta"] for o in obs])
                    dh = np.array([o["dlnz_dh"] for o in obs])
                    ctx.save_for_backward(torch.as_tensor(db, dtype=beta.dtype, device=beta.device),
                                          torch.as_tensor(dh, dtype=h.dtype, device=h.device))
                    return torch.as_tensor(lnz_v, dtype=beta.dtype, device=beta.device)

                @staticmethod
                def backward(ctx, grad):
                    db, dh = ctx.saved_tensors
                    return grad * db, grad * dh, None, None, None, None, None

            cls._fn = _LnZ
        return cls._fn


def lnz(beta, h, d: int = 4, Dcut: int = 10, nsteps: int = 40, mode: str = "eig", **kw):
    """ln Z_N / N after `nsteps` steps (N = 2^nsteps sites) for each (beta[i], h[i]), as a tensor
    that autograd differentiates in beta and h. beta and h are 1-D tensors of equal length (the
    instances of one batched flow); kw are HOTRG options (precision, fp64_steps, x6_steps, ...)."""
    import torch
    beta = torch.as_tensor(beta, dtype=torch.float64)
    h = torch.as_tensor(h, dtype=beta.dtype, device=beta.device)
    if beta.dim() == 0:
        beta = beta.reshape(1)
    if h.dim() == 0:
        h = h.expand(beta.shape[0])
    if mode not in ("eig", "fixed"):
        raise ValueError("mode must be 'eig' or 'fixed'")
    return LnZ.function().apply(beta, h, d, Dcut, nsteps, mode, kw)
