"""Seeded synthetic workloads for the FIT leapfrog + ParaExp hot path.

This module holds only input generation: cell counts, spacings, per-cell
materials, source and probe positions, step counts and window bounds.  It
contains none of the method's arithmetic (no curls, no coefficients, no CFL),
so both the CUDA path and the CPU oracle can consume its output.

Per-cell arrays are float32 of shape ``(nz, ny, nx)`` (x fastest).  Random
numbers come from numpy's PCG64, which gives the same stream on every
platform.

Workloads (the paper's spiral-inductor mesh is proprietary and not public, so
every workload is synthetic):

* ``cavity16``  16^3 PEC vacuum cavity, 1 mm cells, FP64, 2000 steps, K=4.
* ``boxes256``  256^3, 0.5 mm, 40 dielectric boxes eps_r~U[2,10], sides
  U{8..40}, sigma=0.05 S/m on 5% of cells, 20000 steps, K=16, FP32.
* ``batch64``   64 PEC cavities with sides U{32..160}, eps_r~U[1,8] per 8^3
  block, lossless, 5000 steps, K=8 each, FP32.
* ``adjoint128`` 128^3, eps_r~U[1,6] per 8^3 block, sigma=0.01 S/m, 10000
  steps, functional on 4 probe edges, FP32.
* ``boxes512``  512^3, lossy boxes as boxes256 with sides doubled, 100000
  steps, K=32, FP32.
* ``wave2d``    the paper's 2-D cylindrical wave (Sec. IV-A): 20 m x 20 m x
  1 m, 40x40x1 cells, centred z line current, Gaussian pulse.
* ``boxes256_lossless`` boxes256 without conductivity (2000 steps): the
  exponential propagators need a lossless grid.
* ``wave2d_graded(k)`` / ``boxes_graded(k)`` the 2-D wave grid and the
  lossless 256^3 boxes with the central column/row (slab) of cells shrunk to
  d/k: graded tensor-product grids for the non-uniform mesh study.
* ``small_random`` / ``graded_random`` small non-cubic grids with random
  eps_r, mu_r, sigma (and random per-cell sizes) for parity tests;
  ``random_state`` seeded initial fields.

``nsteps`` and the grid size can be overridden for tests.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED = 20170523
C0 = 299792458.0


@dataclasses.dataclass
class Workload:
    name: str
    dims: tuple            # (nx, ny, nz) cells
    spacing: tuple         # (dx, dy, dz) metres
    eps_r: np.ndarray      # (nz, ny, nx) float32
    mu_r: Optional[np.ndarray]
    sigma: Optional[np.ndarray]
    sources: List[dict]    # edge currents: axis, i, j, k, waveform, amp, f0, width, delay
    probes: List[dict]     # edges: axis, i, j, k
    nsteps: int
    cfl_fraction: float
    K: int
    precision: int         # 32 or 64

    @property
    def ncells(self) -> int:
        return int(self.dims[0]) * int(self.dims[1]) * int(self.dims[2])

    def windows(self, K: Optional[int] = None, step0: int = 0) -> np.ndarray:
        """K equal windows of the step range [step0, step0 + nsteps)."""
        K = self.K if K is None else K
        return np.array([step0 + (j * self.nsteps) // K for j in range(K + 1)], dtype=np.int64)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gauss_sine(axis, i, j, k, f0, width, amp=1.0):
    """Gaussian-modulated sine edge current, centred one width after t=0."""
    return dict(axis=axis, i=i, j=j, k=k, waveform=0, amp=amp, f0=f0, width=width, delay=width)


def band_source(axis, i, j, k, d, eps_max):
    """Source resolved with 10 cells per wavelength in the densest material:
    f_max = c / (10 d sqrt(eps_max)), centre f0 = f_max / 2 and Gaussian width
    1.93 / (f_max - f0)."""
    f_max = C0 / (10.0 * d * math.sqrt(eps_max))
    f0 = 0.5 * f_max
    return gauss_sine(axis, i, j, k, f0, 1.93 / (f_max - f0))


def _boxes(rng, n, nboxes, side_lo, side_hi, eps_lo, eps_hi):
    """Background eps_r=1 with axis-aligned boxes painted in order (later
    boxes overwrite earlier ones)."""
    nx, ny, nz = n
    eps = np.ones((nz, ny, nx), dtype=np.float32)
    for _ in range(nboxes):
        sx, sy, sz = (int(rng.integers(side_lo, side_hi + 1)) for _ in range(3))
        x0 = int(rng.integers(0, nx - sx + 1))
        y0 = int(rng.integers(0, ny - sy + 1))
        z0 = int(rng.integers(0, nz - sz + 1))
        eps[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx] = np.float32(rng.uniform(eps_lo, eps_hi))
    return eps


def _blocks(rng, n, block, lo, hi):
    """Piecewise-constant eps_r on block^3 blocks, uniform in [lo, hi]."""
    nx, ny, nz = n
    bx, by, bz = (-(-v // block) for v in (nx, ny, nz))
    vals = rng.uniform(lo, hi, size=(bz, by, bx)).astype(np.float32)
    eps = np.repeat(np.repeat(np.repeat(vals, block, 0), block, 1), block, 2)
    return np.ascontiguousarray(eps[:nz, :ny, :nx])


def _centre_probes(n, k=None):
    nx, ny, nz = n
    kz = nz // 2 if k is None else k
    return [dict(axis=2, i=nx // 4, j=ny // 2, k=kz), dict(axis=2, i=(3 * nx) // 4, j=ny // 2, k=kz),
            dict(axis=2, i=nx // 2, j=ny // 4, k=kz), dict(axis=2, i=nx // 2, j=(3 * ny) // 4, k=kz)]


def cavity16(seed: int = SEED, nsteps: int = 2000) -> Workload:
    n = (16, 16, 16)
    return Workload(
        name="cavity16", dims=n, spacing=(1e-3, 1e-3, 1e-3),
        eps_r=np.ones((16, 16, 16), np.float32), mu_r=None, sigma=None,
        sources=[gauss_sine(2, 8, 8, 8, 30e9, 1.6e-9)],
        probes=[dict(axis=2, i=4, j=4, k=8), dict(axis=2, i=12, j=6, k=8), dict(axis=2, i=6, j=12, k=4)],
        nsteps=nsteps, cfl_fraction=0.95, K=4, precision=64)


def boxes(n_side: int = 256, seed: int = SEED, nsteps: int = 20000, K: int = 16,
          side_scale: float = 1.0, name: str = "boxes256", nboxes: int = 40, lossy: bool = True) -> Workload:
    rng = _rng(seed)
    n = (n_side, n_side, n_side)
    lo = max(1, int(round(8 * side_scale)))
    hi = max(lo, min(n_side, int(round(40 * side_scale))))
    eps = _boxes(rng, n, nboxes, lo, hi, 2.0, 10.0)
    sigma = np.where(rng.random((n_side, n_side, n_side)) < 0.05, 0.05, 0.0).astype(np.float32)
    d = 0.5e-3
    c = n_side // 2
    return Workload(
        name=name, dims=n, spacing=(d, d, d), eps_r=eps, mu_r=None, sigma=sigma if lossy else None,
        sources=[band_source(2, c, c, c, d, 10.0)], probes=_centre_probes(n),
        nsteps=nsteps, cfl_fraction=0.95, K=K, precision=32)


def boxes256(seed: int = SEED, nsteps: int = 20000, n_side: int = 256) -> Workload:
    return boxes(n_side=n_side, seed=seed, nsteps=nsteps, K=16, name="boxes256")


def boxes256_lossless(seed: int = SEED, nsteps: int = 2000, n_side: int = 256) -> Workload:
    """The 256^3 boxes without conductivity (the same eps_r): the exponential
    propagators need a lossless grid."""
    return boxes(n_side=n_side, seed=seed, nsteps=nsteps, K=16, name="boxes256lossless", lossy=False)


def boxes_graded(k: float, n_side: int = 256, seed: int = SEED, nsteps: int = 2000) -> Workload:
    """The lossless 256^3 boxes with the central slab of cells along each axis
    shrunk to d/k (a strongly graded tensor-product grid; largest / smallest
    cell size k)."""
    w = boxes(n_side=n_side, seed=seed, nsteps=nsteps, K=16, name=f"boxes{n_side}_k{k:g}", lossy=False)
    d = w.spacing[0]
    c = n_side // 2
    sizes = []
    for _ in range(3):
        a = np.full(n_side, d)
        a[c] = d / k
        sizes.append(a)
    w.spacing = tuple(sizes)
    return w


def boxes512(seed: int = SEED, nsteps: int = 100000, n_side: int = 512) -> Workload:
    return boxes(n_side=n_side, seed=seed, nsteps=nsteps, K=32, side_scale=2.0, name="boxes512")


def cavity_batch(count: int = 64, side_lo: int = 32, side_hi: int = 160, seed: int = SEED,
                 nsteps: int = 5000, K: int = 8) -> List[Workload]:
    rng = _rng(seed)
    out = []
    d = 0.5e-3
    for g in range(count):
        n = tuple(int(rng.integers(side_lo, side_hi + 1)) for _ in range(3))
        eps = _blocks(rng, n, 8, 1.0, 8.0)
        nx, ny, nz = n
        out.append(Workload(
            name=f"batch{count}[{g}]", dims=n, spacing=(d, d, d), eps_r=eps, mu_r=None, sigma=None,
            sources=[band_source(2, nx // 2, ny // 2, nz // 2, d, 8.0)], probes=_centre_probes(n),
            nsteps=nsteps, cfl_fraction=0.95, K=K, precision=32))
    return out


def adjoint128(seed: int = SEED, nsteps: int = 10000, n_side: int = 128) -> Workload:
    rng = _rng(seed)
    n = (n_side, n_side, n_side)
    eps = _blocks(rng, n, 8, 1.0, 6.0)
    sigma = np.full((n_side, n_side, n_side), 0.01, np.float32)
    d = 0.5e-3
    c = n_side // 2
    return Workload(
        name="adjoint128", dims=n, spacing=(d, d, d), eps_r=eps, mu_r=None, sigma=sigma,
        sources=[band_source(2, c, c, c, d, 6.0)], probes=_centre_probes(n),
        nsteps=nsteps, cfl_fraction=0.95, K=1, precision=32)


def fd_cells(w: Workload, count: int = 16, seed: int = SEED + 1) -> np.ndarray:
    """Seeded random cell indices (k, j, i) for finite-difference checks."""
    rng = _rng(seed)
    nx, ny, nz = w.dims
    return np.stack([rng.integers(0, nz, count), rng.integers(0, ny, count), rng.integers(0, nx, count)], 1)


def wave2d(n_xy: int = 40, nsteps: int = 180) -> Workload:
    """Sec. IV-A: 20 m x 20 m x 1 m PEC box in vacuum, one cell thick in z,
    z line current i(t) = exp(-4((t - s)/s)^2), s = 2e-8 s, at the centre."""
    d = 20.0 / n_xy
    c = n_xy // 2
    src = dict(axis=2, i=c, j=c, k=0, waveform=1, amp=1.0, f0=0.0, width=2e-8, delay=2e-8)
    return Workload(
        name="wave2d", dims=(n_xy, n_xy, 1), spacing=(d, d, 1.0),
        eps_r=np.ones((1, n_xy, n_xy), np.float32), mu_r=None, sigma=None,
        sources=[src], probes=[dict(axis=2, i=c + n_xy // 4, j=c, k=0), dict(axis=2, i=c, j=c + n_xy // 8, k=0)],
        nsteps=nsteps, cfl_fraction=1.0, K=6, precision=64)


def wave2d_graded(k: float, n_xy: int = 40) -> Workload:
    """The 2-D wave grid of Sec. IV-A with its central element shrunk to
    (d/k) x (d/k): on a tensor-product grid that makes the central column
    and row of cells d/k wide, so the ratio of the largest to the smallest
    element size is k (the non-uniform study of Sec. IV-A, R(k))."""
    w = wave2d(n_xy=n_xy)
    d = 20.0 / n_xy
    c = n_xy // 2
    dx = np.full(n_xy, d)
    dy = np.full(n_xy, d)
    dx[c] = d / k
    dy[c] = d / k
    w.spacing = (dx, dy, np.array([1.0]))
    w.name = f"wave2d_k{k:g}"
    return w


def small_random(dims=(12, 10, 8), spacing=(1e-3, 1.2e-3, 0.9e-3), seed: int = SEED, lossy=True,
                 mu=False, nsteps: int = 200, K: int = 4, precision: int = 64) -> Workload:
    """Small non-cubic grid with random eps (and sigma, mu) for parity tests."""
    rng = _rng(seed)
    nx, ny, nz = dims
    eps = rng.uniform(1.0, 6.0, size=(nz, ny, nx)).astype(np.float32)
    sig = rng.uniform(0.0, 0.3, size=(nz, ny, nx)).astype(np.float32) if lossy else None
    mu_r = rng.uniform(1.0, 3.0, size=(nz, ny, nx)).astype(np.float32) if mu else None
    dmin = min(spacing)
    srcs = [band_source(2, nx // 2, ny // 2, nz // 2, dmin, 6.0),
            dict(band_source(0, nx // 3, max(1, ny // 3), max(1, nz // 3), dmin, 6.0), amp=0.5)]
    prbs = [dict(axis=2, i=1, j=2, k=1), dict(axis=0, i=nx - 2, j=ny - 2, k=nz // 2),
            dict(axis=1, i=nx // 2, j=1, k=nz - 2), dict(axis=2, i=nx - 3, j=ny // 2, k=nz - 1)]
    return Workload(name=f"small{nx}x{ny}x{nz}", dims=dims, spacing=spacing, eps_r=eps, mu_r=mu_r,
                    sigma=sig, sources=srcs, probes=prbs, nsteps=nsteps, cfl_fraction=0.95, K=K,
                    precision=precision)


def graded_random(dims=(37, 19, 26), seed: int = SEED + 3, lossy=True, mu=True, ratio: float = 6.0) -> Workload:
    """small_random with per-cell sizes drawn in [1 mm / ratio, 1 mm] along
    every axis (a graded grid)."""
    w = small_random(dims=dims, seed=seed, lossy=lossy, mu=mu, precision=64)
    rng = _rng(seed + 1)
    w.spacing = tuple(rng.uniform(1e-3 / ratio, 1e-3, n) for n in dims)
    w.name = "graded" + w.name[5:]
    return w


def random_state(dims, seed: int = SEED + 7, dtype=np.float64):
    """Seeded normal (e, h) in the compact layout (3, nz, ny, nx): an initial
    value for propagation tests (entries off the degrees of freedom are
    ignored by both the library and the oracle)."""
    rng = _rng(seed)
    nx, ny, nz = dims
    e = rng.standard_normal((3, nz, ny, nx)).astype(dtype)
    h = rng.standard_normal((3, nz, ny, nx)).astype(dtype)
    return e, h


WORKLOADS = {
    "cavity16": cavity16,
    "boxes256": boxes256,
    "adjoint128": adjoint128,
    "boxes512": boxes512,
    "boxes256lossless": boxes256_lossless,
    "wave2d": wave2d,
}
