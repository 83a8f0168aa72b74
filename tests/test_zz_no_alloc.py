"""The allocation-free entry point fit_leapfrog_run_static, called through the
C ABI, gives the same fields and probe traces as fit_leapfrog_run on the
same inputs, on two calls in a row (the second on another grid, so leftovers
of the first call in the shared scratch array would show); an odd step count
above its source-table chunk (32768 steps) does too; on a grid at its size
limit it matches the FP64 oracle within the FP32 tolerance model; and it
rejects a grid larger than its fixed scratch with FIT_ERR_ARG.

This file is collected last: the entry point's scratch array is shared by
all calls, and the test must pass both alone and after every other test."""
import numpy as np
import pytest

import oracle
from helpers import TOL32, check, compact, oracle_grid, probe_relerr, relerr, tol32, tol32_probe
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
        check("probes", probe_relerr(pr, pr_ref), TOL32)
        check("e", relerr(e, e_ref), TOL32)
        check("h", relerr(h, h_ref), TOL32)
        assert np.abs(e).max() > 0


def test_static_entry_point_odd_steps_beyond_one_source_chunk(torch_cuda):
    """32771 steps (odd, so the final state is in the second buffer; longer than
    one 32768-step chunk of the source table, so the table is rebuilt from
    step0 + 32768) with a source, against fit_leapfrog_run."""
    w = W.small_random(dims=(20, 14, 9), lossy=True)
    pr, e, h, pr_ref, e_ref, h_ref = _case(torch_cuda, w, 32771, 3)
    assert np.isfinite(pr).all()
    check("probes", probe_relerr(pr, pr_ref), TOL32)
    check("e", relerr(e, e_ref), TOL32)
    check("h", relerr(h, h_ref), TOL32)
    assert np.abs(pr[-100:]).max() > 0


def test_static_entry_point_at_its_size_limit_matches_oracle(torch_cuda):
    """64 x 64 x 96 cells (ceil4(nx) ny nz = 393216, the scratch's limit), lossy,
    two sources, 100 steps from zero: against the FP64 oracle on the same
    float-rounded coefficients, held to the FP32 tolerance model (4 x the
    oracle's float-storage model error)."""
    torch = torch_cuda
    dev = torch.device("cuda")
    w = W.small_random(dims=(64, 64, 96), lossy=True, nsteps=100)
    nx, ny, nz = w.dims
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    eps = torch.from_numpy(w.eps_r).to(dev)
    sig = torch.from_numpy(w.sigma).to(dev)
    e = torch.zeros((3, nz, ny, nx), dtype=torch.float32, device=dev)
    h = torch.zeros_like(e)
    pr = torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev)
    fitgb.fit_leapfrog_run_static(w.dims, w.spacing, eps, sig, dt, w.nsteps, 0, w.sources, w.probes, pr, e, h)
    torch.cuda.synchronize()
    pr, e, h = pr.cpu().numpy(), e.cpu().numpy(), h.cpu().numpy()
    w.mu_r = None
    opr, _, oe, oh = oracle_grid(w, dt, round32=True).leapfrog(w.nsteps, w.sources, w.probes)
    mpr, _, me, mh = oracle_grid(w, dt, round32=True, store32=True).leapfrog(w.nsteps, w.sources, w.probes)
    check("probes", probe_relerr(pr, opr), tol32_probe(mpr, opr))
    check("e", relerr(e, compact(oe)), tol32(compact(me), compact(oe)))
    check("h", relerr(h, compact(oh)), tol32(compact(mh), compact(oh)))
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
    # non-finite spacing or step
    nx, ny, nz = 16, 8, 8
    eps = torch.ones((nz, ny, nx), dtype=torch.float32, device=dev)
    e = torch.zeros((3, nz, ny, nx), dtype=torch.float32, device=dev)
    h = torch.zeros_like(e)
    for spacing, dt in (((float("inf"), 1e-3, 1e-3), 1e-12), ((1e-3,) * 3, float("inf"))):
        with pytest.raises(fitgb.FitError) as ei:
            fitgb.fit_leapfrog_run_static((nx, ny, nz), spacing, eps, None, dt, 4, 0, (), (), None, e, h)
        assert ei.value.status == fitgb.FIT_ERR_ARG
