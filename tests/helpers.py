"""Shared test helpers: error metrics and oracle/CUDA-side runners.

The oracle works in the canonical FIT layout (3, nz+1, ny+1, nx+1); the CUDA
library in the compact layout (3, nz, ny, nx).  ``oracle.to_compact`` drops
the all-zero index-n slices.
"""
import numpy as np

import oracle

# FP64 paths: relative L2 error <= 1e-11 against the FP64 oracle (rounding of
# ~1e3 steps of O(10) flops each).
TOL64 = 1e-11
# FP32 paths are compared with the FP64 oracle run on the same float-rounded
# coefficients.  The floor 1e-5 is the method's FP32 target.  Rounding every
# stored e and h value to float accumulates over the steps like a random
# walk (about 6e-8 sqrt(steps) of the field), and more in relative terms for a
# quantity whose own norm is small; no FP32-storage scheme can beat the
# "store32" model (exact arithmetic, every stored e and h rounded to float).
# The tolerance is therefore max(1e-5, FP32_FACTOR x the store32 model's own
# error) per compared quantity: FP32 arithmetic in the curl sums and updates
# adds rounding of the same order (1.3-2.2x the model in a float32 numpy
# emulation), and 4x leaves margin while a real indexing or coefficient bug
# gives errors of order one.
TOL32 = 1e-5
FP32_FACTOR = 4.0


def tol32(model, ref):
    """FP32 tolerance for one quantity from its store32-model value."""
    return max(TOL32, FP32_FACTOR * relerr(model, ref))


def tol32_probe(model, ref):
    return max(TOL32, FP32_FACTOR * probe_relerr(model, ref))


def relerr(x, ref, floor=None):
    """max over leading-axis slices of ||x - ref||_2 / ||ref||_2.

    A slice (field component, probe trace) whose reference norm is below
    `floor` -- by default 1% of the norm of the whole reference -- is measured
    against `floor` instead: components that vanish in exact arithmetic (by
    symmetry, or out of the source's reach) hold only rounding noise, whose
    relative error means nothing."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    assert x.shape == ref.shape, (x.shape, ref.shape)
    if x.ndim == 1:
        x, ref = x[None], ref[None]
    worst = 0.0
    norms = [np.linalg.norm(r) for r in ref.reshape(ref.shape[0], -1)]
    scale = floor if floor is not None else 1e-2 * max(np.linalg.norm(ref), 1e-300)
    for a, r, n in zip(x.reshape(x.shape[0], -1), ref.reshape(ref.shape[0], -1), norms):
        worst = max(worst, np.linalg.norm(a - r) / max(n, scale))
    return worst


def probe_relerr(pr, ref):
    """Relative L2 error per probe trace (columns)."""
    pr = np.asarray(pr)
    ref = np.asarray(ref)
    return relerr(pr.T, ref.T)


def oracle_grid(w, dt, round32, scheme=0, store32=False):
    return oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, sigma_scheme=scheme,
                             round32=round32, store32=store32)


def compact(a):
    return oracle.to_compact(a)


def canonical(a, dims):
    """Compact (3, nz, ny, nx) -> canonical (3, nz+1, ny+1, nx+1) with zero pads."""
    nx, ny, nz = dims
    out = np.zeros((3, nz + 1, ny + 1, nx + 1))
    out[:, :nz, :ny, :nx] = a
    return out
