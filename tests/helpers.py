"""Shared test helpers: error metrics and oracle/CUDA-side runners.

The oracle works in the canonical FIT layout (3, nz+1, ny+1, nx+1); the CUDA
library in the compact layout (3, nz, ny, nx).  ``oracle.to_compact`` drops
the all-zero index-n slices.
"""
import numpy as np

import oracle

# FP32 field tolerance: relative L2 error <= 1e-5 against the FP64 oracle run
# with the same float-rounded coefficients (the target of the method's FP32
# path).  FP64 paths: 1e-11 (rounding of ~1e3-1e4 steps of O(10) flops).
TOL32 = 1e-5
TOL64 = 1e-11


def relerr(x, ref, floor=None):
    """max over leading-axis slices of ||x - ref||_2 / ||ref||_2 (slices whose
    reference norm is below `floor` compare against `floor`)."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    assert x.shape == ref.shape, (x.shape, ref.shape)
    if x.ndim == 1:
        x, ref = x[None], ref[None]
    worst = 0.0
    norms = [np.linalg.norm(r) for r in ref.reshape(ref.shape[0], -1)]
    scale = floor if floor is not None else 1e-9 * max(max(norms), 1e-300)
    for a, r, n in zip(x.reshape(x.shape[0], -1), ref.reshape(ref.shape[0], -1), norms):
        worst = max(worst, np.linalg.norm(a - r) / max(n, scale))
    return worst


def probe_relerr(pr, ref):
    """Relative L2 error per probe trace (columns)."""
    pr = np.asarray(pr)
    ref = np.asarray(ref)
    return relerr(pr.T, ref.T, floor=1e-9 * max(np.abs(ref).max(), 1e-300))


def oracle_grid(w, dt, round32, scheme=0):
    return oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, sigma_scheme=scheme,
                             round32=round32)


def compact(a):
    return oracle.to_compact(a)


def canonical(a, dims):
    """Compact (3, nz, ny, nx) -> canonical (3, nz+1, ny+1, nx+1) with zero pads."""
    nx, ny, nz = dims
    out = np.zeros((3, nz + 1, ny + 1, nx + 1))
    out[:, :nz, :ny, :nx] = a
    return out
