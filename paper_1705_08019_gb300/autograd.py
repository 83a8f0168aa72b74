"""torch.autograd binding of the adjoint gradient.

``probe_energy(eps_r, spacing, dt, nsteps, sources, probes, sigma=None)``
returns J = sum_{n=1..N} sum_p (e_p^n / L_p)^2 of an FP32 leapfrog run from
zero state on a grid with per-cell permittivity ``eps_r`` (a float32 CUDA
tensor of shape (nz, ny, nx)); ``J.backward()`` gives dJ/d eps_r from the
adjoint sweep of libfitgb (fit_adjoint_grad).  ``spacing`` holds three
steps, or per-cell sizes along an axis for a graded grid; L_p is then the
size of the cell the probe edge runs through along its axis.  Torch only
holds the tensors and the stream: the run, J and its gradient all come from
the library (without a gradient request, fit_adjoint_grad runs the forward
pass and J only).
"""
from __future__ import annotations

import torch

from . import fitgb


class ProbeEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_r, spacing, dt, nsteps, sources, probes, sigma, ckpt_every, precision):
        nz, ny, nx = eps_r.shape
        dev = eps_r.device
        eps = eps_r.detach().to(torch.float32).contiguous()
        sig = None if sigma is None else sigma.detach().to(device=dev, dtype=torch.float32).contiguous()
        g = fitgb.Grid((nx, ny, nz), spacing, eps, None, sig, precision)
        stream = torch.cuda.current_stream(dev)
        try:
            J = torch.zeros(1, dtype=torch.float64, device=dev)
            # without a gradient request the library runs the forward pass only
            grad = torch.zeros((nz, ny, nx), dtype=torch.float64, device=dev) if ctx.needs_input_grad[0] else None
            fitgb.fit_adjoint_grad(g.handle, dt, nsteps, sources, probes, ckpt_every, J, grad, stream=stream)
            if grad is not None:
                ctx.save_for_backward(grad)
            torch.cuda.synchronize(dev)
        finally:
            g.close()
        return J[0]

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return (gJ * grad).to(torch.float32), None, None, None, None, None, None, None, None


def probe_energy(eps_r, spacing, dt, nsteps, sources, probes, sigma=None, ckpt_every=0, precision=32):
    """J(eps_r) with an adjoint backward; see the module docstring."""
    return ProbeEnergy.apply(eps_r, tuple(spacing), float(dt), int(nsteps), list(sources), list(probes), sigma,
                             int(ckpt_every), int(precision))
