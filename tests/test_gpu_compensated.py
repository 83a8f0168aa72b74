"""Compensated FP32 fields (precision 48): e and h kept as hi + lo float pairs
and advanced in FP32 arithmetic with error-free sums and products.  Against
the FP64 oracle on the same float-rounded coefficients the fields, probes and
energy agree to 1e-10 -- far below what plain float storage allows (see the
FP32 tolerance model in helpers.py), which is the point of the mode."""
import numpy as np
import pytest

import oracle
from helpers import compact, probe_relerr, relerr
from paper_1705_08019_gb300 import fitgb
from paper_1705_08019_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOLC = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fitgb.load()


@pytest.mark.parametrize("dims,kw", [((37, 11, 19), dict(lossy=True)), ((12, 10, 8), dict(lossy=True, mu=True)),
                                     ((70, 19, 45), dict(lossy=False)), ((5, 3, 2), dict(lossy=True))])
def test_compensated_leapfrog_matches_oracle(dims, kw):
    w = W.small_random(dims=dims, nsteps=300, **kw)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r, w.mu_r)
    g = fitgb.Grid.from_workload(w, 48)
    pr, en, e, h = g.leapfrog(dt, w.nsteps, w.sources, w.probes, energy=True)
    g.close()
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=True)
    opr, oen, oe, oh = og.leapfrog(w.nsteps, w.sources, w.probes, energy=True)
    assert probe_relerr(pr, opr) <= TOLC
    assert relerr(e, compact(oe)) <= TOLC
    assert relerr(h, compact(oh)) <= TOLC
    assert relerr(en, oen) <= 1e-6   # energy uses the float-rounded M_eps, M_mu


def test_compensated_initial_state_and_paraexp():
    w = W.small_random(dims=(21, 13, 11), nsteps=150, K=4)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=True)
    rng = np.random.default_rng(4)
    e0 = rng.standard_normal(og.field_shape)
    h0 = rng.standard_normal(og.field_shape) * 1e-2
    e0[:, -1] = 0; e0[:, :, -1] = 0; e0[:, :, :, -1] = 0
    h0[:, -1] = 0; h0[:, :, -1] = 0; h0[:, :, :, -1] = 0
    e0[0, :, 0, :] = 0; e0[0, 0, :, :] = 0; e0[1, :, :, 0] = 0; e0[1, 0, :, :] = 0
    e0[2, :, :, 0] = 0; e0[2, :, 0, :] = 0
    h0[0, :, :, 0] = 0; h0[1, :, 0, :] = 0; h0[2, 0, :, :] = 0
    g = fitgb.Grid.from_workload(w, 48)
    pr, _, e, h = g.leapfrog(dt, w.nsteps, w.sources, w.probes, e=compact(e0), h=compact(h0), step0=11)
    opr, _, oe, oh = og.leapfrog(w.nsteps, w.sources, w.probes, e=e0, h=h0, step0=11)
    assert probe_relerr(pr, opr) <= TOLC and relerr(e, compact(oe)) <= TOLC and relerr(h, compact(oh)) <= TOLC
    win = np.array([0, 20, 61, 99, 150])
    pr, ef, hf = g.paraexp(dt, 4, win, w.sources, w.probes)
    g.close()
    opr, oef, ohf = og.paraexp(4, win, w.sources, w.probes)
    assert probe_relerr(pr, opr) <= TOLC
    assert relerr(ef, compact(oef)) <= TOLC and relerr(hf, compact(ohf)) <= TOLC


def test_fullsize_boxes256_compensated_vs_fp64():
    """256^3 lossy boxes, 2000 steps: compensated FP32 against the FP64 path on
    the same grid with the same float-rounded coefficients (FIT_FLAG_COEF_FLOAT);
    plain FP32 is shown for scale."""
    import torch
    w = W.boxes256(nsteps=2000)
    dev = torch.device("cuda")
    eps = torch.from_numpy(w.eps_r).to(dev)
    sig = torch.from_numpy(w.sigma).to(dev)
    out = {}
    for prec in (64, 48, 32):
        g = fitgb.Grid(w.dims, w.spacing, eps, None, sig, prec, flags=fitgb.FIT_FLAG_COEF_FLOAT)
        dt = w.cfl_fraction * g.cfl_dt()
        T = torch.float32 if prec == 32 else torch.float64
        e = torch.zeros(g.field_shape, dtype=T, device=dev)
        h = torch.zeros_like(e)
        pr = torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev)
        fitgb.fit_leapfrog_run(g.handle, dt, w.nsteps, 0, w.sources, w.probes, pr, None, e, h)
        torch.cuda.synchronize()
        out[prec] = (pr.cpu().numpy(), e.double().cpu().numpy(), h.double().cpu().numpy())
        g.close()
        del e, h
    ec = max(relerr(out[48][1], out[64][1]), relerr(out[48][2], out[64][2]), probe_relerr(out[48][0], out[64][0]))
    e32 = max(relerr(out[32][1], out[64][1]), relerr(out[32][2], out[64][2]), probe_relerr(out[32][0], out[64][0]))
    assert ec <= 1e-9
    assert e32 > 100 * ec


def test_coef_float_flag_matches_rounded_oracle():
    """An FP64 grid with FIT_FLAG_COEF_FLOAT runs the oracle's float-rounded
    coefficients to FP64 accuracy."""
    w = W.small_random(dims=(19, 13, 11), nsteps=200, mu=True)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r, w.mu_r)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, 64, flags=fitgb.FIT_FLAG_COEF_FLOAT)
    pr, _, e, h = g.leapfrog(dt, w.nsteps, w.sources, w.probes)
    g.close()
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=True)
    opr, _, oe, oh = og.leapfrog(w.nsteps, w.sources, w.probes)
    assert probe_relerr(pr, opr) <= 1e-11 and relerr(e, compact(oe)) <= 1e-11 and relerr(h, compact(oh)) <= 1e-11
