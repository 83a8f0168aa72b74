"""The allocation-free entry point fit_leapfrog_run_static, called through the
C ABI, gives the same fields and probe traces as fit_leapfrog_run on the
same inputs, on two calls in a row (the second on another grid, so leftovers
of the first call in the shared scratch array would show), and rejects a grid
larger than its fixed scratch with FIT_ERR_ARG.

This file is collected last: the entry point's scratch array is shared by
all calls, and the test must pass both alone and after every other test."""
import numpy as np
import pytest

import oracle
from helpers import TOL32, probe_relerr, relerr
from paper_1705_08019_gb300 import fitgb
from paper_1705_08019_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fitgb.load()
    return torch


def _case(torch, w, nsteps, step0):
    dev = torch.device("cuda")
    nx, ny, nz = w.dims
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    eps = torch.from_numpy(w.eps_r).to(dev)
    sig = torch.from_numpy(w.sigma).to(dev) if w.sigma is not None else None
    rng = np.random.default_rng(step0 + 1)
    e0 = torch.from_numpy((rng.standard_normal((3, nz, ny, nx)) * 1e-3).astype(np.float32)).to(dev)
    h0 = torch.zeros_like(e0)
    # the existing entry point
    g = fitgb.Grid(w.dims, w.spacing, eps, None, sig, 32)
    e_ref, h_ref = e0.clone(), h0.clone()
    pr_ref = torch.zeros((nsteps, len(w.probes)), dtype=torch.float64, device=dev)
    fitgb.fit_leapfrog_run(g.handle, dt, nsteps, step0, w.sources, w.probes, pr_ref, None, e_ref, h_ref)
    torch.cuda.synchronize()
    g.close()
    # the allocation-free one
    e, h = e0.clone(), h0.clone()
    pr = torch.full((nsteps, len(w.probes)), np.nan, dtype=torch.float64, device=dev)
    fitgb.fit_leapfrog_run_static(w.dims, w.spacing, eps, sig, dt, nsteps, step0, w.sources, w.probes, pr, e, h)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (pr, e, h, pr_ref, e_ref, h_ref)]


def test_static_entry_point_matches_leapfrog_run(torch_cuda):
    cases = [(W.small_random(dims=(37, 11, 19), lossy=True), 160, 5),
             (W.small_random(dims=(20, 14, 9), lossy=False), 120, 0)]
    for w, nsteps, step0 in cases:
        pr, e, h, pr_ref, e_ref, h_ref = _case(torch_cuda, w, nsteps, step0)
        assert np.isfinite(pr).all()
        assert probe_relerr(pr, pr_ref) <= TOL32
        assert relerr(e, e_ref) <= TOL32 and relerr(h, h_ref) <= TOL32
        assert np.abs(e).max() > 0


def test_static_entry_point_rejects_oversize_grid(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda")
    nx, ny, nz = 128, 64, 64   # beyond the fixed scratch
    eps = torch.ones((nz, ny, nx), dtype=torch.float32, device=dev)
    e = torch.zeros((3, nz, ny, nx), dtype=torch.float32, device=dev)
    h = torch.zeros_like(e)
    with pytest.raises(fitgb.FitError) as ei:
        fitgb.fit_leapfrog_run_static((nx, ny, nz), (1e-3,) * 3, eps, None, 1e-12, 4, 0, (), (), None, e, h)
    assert ei.value.status == fitgb.FIT_ERR_ARG
