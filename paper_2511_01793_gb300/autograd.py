"""Differentiable exit-wave misfit (Sec. 2.1) on the library's gradient kernel.

``ExitWaveMisfit.apply(obj, probe, ctx)`` returns
Phi(Q, z) = 1/2 sum_k ||Q . P_k z - R_k(Q, P_k z)||^2 as a float64 scalar
tensor.  Its backward calls ``emg_misfit_gradient``, which recomputes the
revised exit waves and returns the Wirtinger gradients
conj(Q) (Q z_k - R_k) and conj(z_k) (Q z_k - R_k) summed over positions,
in PyTorch's complex-gradient convention (d/dRe + i d/dIm).  Nothing is
stored between forward and backward except the two input tensors.

``gradient_descent`` is the plain gradient baseline run beside eMAGPIE.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Context, emg_misfit_gradient


def _c64(t: torch.Tensor) -> torch.Tensor:
    if t.dtype != torch.complex64 or not t.is_cuda or not t.is_contiguous():
        raise TypeError("object and probe must be contiguous complex64 CUDA tensors")
    return t


class ExitWaveMisfit(torch.autograd.Function):
    @staticmethod
    def forward(fctx, obj: torch.Tensor, probe: torch.Tensor, ctx: Context) -> torch.Tensor:
        _c64(obj)
        _c64(probe)
        phi = emg_misfit_gradient(ctx.ctx, obj.data_ptr(), probe.data_ptr(), 0, 0, True)
        fctx.save_for_backward(obj, probe)
        fctx.emg = ctx
        return torch.tensor(phi, dtype=torch.float64, device=obj.device)

    @staticmethod
    def backward(fctx, grad_out: torch.Tensor):
        obj, probe = fctx.saved_tensors
        g_obj = torch.empty_like(obj)
        g_probe = torch.empty_like(probe)
        emg_misfit_gradient(fctx.emg.ctx, obj.data_ptr(), probe.data_ptr(), g_obj.data_ptr(),
                            g_probe.data_ptr(), False)
        s = grad_out.to(torch.float32)
        return g_obj * s, g_probe * s, None


def misfit(obj: torch.Tensor, probe: torch.Tensor, ctx: Context) -> torch.Tensor:
    return ExitWaveMisfit.apply(obj, probe, ctx)


def default_step_sizes(obj: torch.Tensor, probe: torch.Tensor, pos: np.ndarray, m: int):
    """Step sizes from the diagonal curvature of Phi: 1 / (coverage max|Q|^2) for
    the object and 1 / (sum_k max|z_k|^2) for the probe, halved."""
    n_rows, n_cols = obj.shape
    cover = np.zeros((n_rows, n_cols), dtype=np.int32)
    for r, c in np.asarray(pos):
        cover[max(r, 0):max(min(r + m, n_rows), 0), max(c, 0):max(min(c + m, n_cols), 0)] += 1
    mq = float(probe.abs().max().item()) ** 2
    mz = float(obj.abs().max().item()) ** 2
    return 0.5 / (max(cover.max(), 1) * mq), 0.5 / (len(pos) * mz)


def gradient_descent(ctx: Context, obj: torch.Tensor, probe: torch.Tensor, n_iter: int,
                     lr_object: float = None, lr_probe: float = None):
    """Plain simultaneous gradient descent on (z, Q); returns (obj, probe, misfit history)."""
    pos = ctx.pos.cpu().numpy()
    obj = obj.detach().clone().contiguous()
    probe = probe.detach().clone().contiguous()
    if lr_object is None or lr_probe is None:
        lo, lp = default_step_sizes(obj, probe, pos, ctx.m)
        lr_object = lo if lr_object is None else lr_object
        lr_probe = lp if lr_probe is None else lr_probe
    hist = []
    for _ in range(n_iter):
        o = obj.requires_grad_(True)
        p = probe.requires_grad_(True)
        loss = misfit(o, p, ctx)
        loss.backward()
        with torch.no_grad():
            obj = (o - lr_object * o.grad).detach().contiguous()
            probe = (p - lr_probe * p.grad).detach().contiguous()
        hist.append(float(loss.item()))
    return obj, probe, hist
