"""Two leapfrog steps per launch (temporal blocking, opts.steps_per_launch = 2;
FP32, TMA) against the FP64 oracle on float coefficients, with the FP32
tolerance of test_gpu_parity.py (the oracle's store32 model), and against
the one-step kernel at the full 256^3 size."""
import numpy as np
import pytest

import oracle
from helpers import check, compact, probe_relerr, relerr, tol32, tol32_probe
from paper_1705_08019_gb300 import fitgb
from paper_1705_08019_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fitgb.load()


def two(**kw):
    return fitgb.make_opts(steps_per_launch=2, **kw)


def oracle_pair(w, dt):
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=True)
    sg = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=True, store32=True)
    return og, sg


@pytest.mark.parametrize("dims,lossy,mu,nsteps", [
    ((37, 19, 45), True, False, 101),     # odd: the last launch takes one step
    ((33, 17, 21), False, False, 60),
    ((64, 24, 70), True, True, 57),
    ((20, 40, 9), True, False, 2),
])
def test_two_step_leapfrog_equals_oracle(dims, lossy, mu, nsteps):
    w = W.small_random(dims=dims, lossy=lossy, mu=mu, seed=sum(dims))
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, 32)
    dt = w.cfl_fraction * g.cfl_dt()
    pr, _, e, h = g.leapfrog(dt, nsteps, w.sources, w.probes, opts=two())
    g.close()
    og, sg = oracle_pair(w, dt)
    opr, _, oe, oh = og.leapfrog(nsteps, w.sources, w.probes)
    mpr, _, me, mh = sg.leapfrog(nsteps, w.sources, w.probes)
    check("probes", probe_relerr(pr, opr), tol32_probe(mpr, opr))
    check("e", relerr(e, compact(oe)), tol32(compact(me), compact(oe)))
    check("h", relerr(h, compact(oh)), tol32(compact(mh), compact(oh)))


def test_two_step_sources_and_probes_on_tile_edges():
    """Sources on the halo rows and columns of 32 x 8 tiles (the first step
    recomputes them for the neighbouring tile) and probes there."""
    w = W.small_random(dims=(66, 26, 19), lossy=True, seed=77)
    w.sources = [dict(w.sources[0], i=31, j=7, k=5), dict(w.sources[0], axis=0, i=32, j=8, k=9, amp=0.7),
                 dict(w.sources[0], axis=1, i=63, j=16, k=18, amp=-0.4)]
    w.probes = [dict(axis=2, i=32, j=8, k=5), dict(axis=0, i=31, j=7, k=9), dict(axis=1, i=64, j=15, k=17)]
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, 32)
    dt = w.cfl_fraction * g.cfl_dt()
    pr, _, e, h = g.leapfrog(dt, 75, w.sources, w.probes, opts=two())
    g.close()
    og, sg = oracle_pair(w, dt)
    opr, _, oe, oh = og.leapfrog(75, w.sources, w.probes)
    mpr, _, me, mh = sg.leapfrog(75, w.sources, w.probes)
    check("probes", probe_relerr(pr, opr), tol32_probe(mpr, opr))
    check("e", relerr(e, compact(oe)), tol32(compact(me), compact(oe)))
    check("h", relerr(h, compact(oh)), tol32(compact(mh), compact(oh)))


def test_two_step_paraexp_equals_oracle():
    w = W.small_random(dims=(41, 23, 30), lossy=True, K=5, seed=88)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, 32)
    dt = w.cfl_fraction * g.cfl_dt()
    win = np.array([3, 40, 41, 90, 125, 181])
    pr, ef, hf = g.paraexp(dt, 5, win, w.sources, w.probes, opts=two())
    g.close()
    og, sg = oracle_pair(w, dt)
    opr, oef, ohf = og.paraexp(5, win, w.sources, w.probes)
    mpr, mef, mhf = sg.paraexp(5, win, w.sources, w.probes)
    check("probes", probe_relerr(pr, opr), tol32_probe(mpr, opr))
    check("ef", relerr(ef, compact(oef)), tol32(compact(mef), compact(oef)))
    check("hf", relerr(hf, compact(ohf)), tol32(compact(mhf), compact(ohf)))


def test_two_step_fullsize_paraexp_matches_one_step():
    """256^3 lossy boxes, K = 16, 600 steps: against an FP64 leapfrog run on
    the same float coefficients (FIT_FLAG_COEF_FLOAT), the two-step launch is
    as accurate as the one-step kernel (within 2x of its error, or 1e-5)."""
    import torch
    w = W.boxes256(nsteps=600)
    dev = torch.device("cuda")
    eps = torch.from_numpy(w.eps_r).to(dev)
    sig = torch.from_numpy(w.sigma).to(dev)
    g64 = fitgb.fit_grid_create(w.dims, w.spacing, eps, None, sig, 64, fitgb.FIT_FLAG_COEF_FLOAT)
    dt = w.cfl_fraction * fitgb.fit_cfl_dt(g64)
    ref = torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev)
    fitgb.fit_leapfrog_run(g64, dt, w.nsteps, 0, w.sources, w.probes, ref)
    torch.cuda.synchronize()
    fitgb.fit_grid_destroy(g64)
    ref = ref.cpu().numpy()
    g = fitgb.fit_grid_create(w.dims, w.spacing, eps, None, sig, 32)
    win = w.windows()
    errs = []
    for opts in (fitgb.make_opts(steps_per_launch=1), two()):
        pr = torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev)
        fitgb.paraexp_run(g, dt, w.K, win, w.sources, w.probes, pr, opts=opts)
        torch.cuda.synchronize()
        errs.append(probe_relerr(pr.cpu().numpy(), ref))
    fitgb.fit_grid_destroy(g)
    assert errs[1] <= max(2.0 * errs[0], 1e-5), errs
