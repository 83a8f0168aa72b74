"""Graded (tensor-product) grids on the GPU against the oracle: leapfrog,
ParaExp with leapfrog and with Leja homogeneous problems, the CFL estimate,
the spectral bound and the adjoint gradient.  Tolerances as in test_gpu_parity.py (FP64 1e-11,
FP32 from the oracle's store32 model) and test_gpu_expo.py (1e-10)."""
import numpy as np
import pytest

import oracle
from oracle import expo
from helpers import TOL64, check, compact, probe_relerr, relerr, tol32, tol32_probe
from paper_1705_08019_gb300 import fitgb
from paper_1705_08019_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fitgb.load()


def setup(lossy=True, mu=True, dims=(37, 19, 26), seed=5):
    w = W.graded_random(dims=dims, lossy=lossy, mu=mu, seed=seed)
    return w


def test_graded_cfl_and_bound_equal_oracle():
    w = setup(lossy=False)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, None, 64)
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, None)
    assert abs(g.cfl_dt() / oracle.cfl_dt(w.dims, w.spacing, w.eps_r, w.mu_r) - 1) <= 1e-15
    assert abs(g.spectral_bound() / expo.spectral_bound(og) - 1) <= 1e-15
    g.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_graded_leapfrog_equals_oracle(precision):
    w = setup()
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, precision)
    dt = 0.95 * g.cfl_dt()
    n = 150
    pr, en, e, h = g.leapfrog(dt, n, w.sources, w.probes, energy=True)
    g.close()
    r32 = precision == 32
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=r32)
    opr, oen, oe, oh = og.leapfrog(n, w.sources, w.probes, energy=True)
    if precision == 64:
        assert probe_relerr(pr, opr) <= TOL64 and relerr(en, oen) <= TOL64
        assert relerr(e, compact(oe)) <= TOL64 and relerr(h, compact(oh)) <= TOL64
    else:
        sg = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=True, store32=True)
        mpr, _, me, mh = sg.leapfrog(n, w.sources, w.probes)
        check("probes", probe_relerr(pr, opr), tol32_probe(mpr, opr))
        check("e", relerr(e, compact(oe)), tol32(compact(me), compact(oe)))
        check("h", relerr(h, compact(oh)), tol32(compact(mh), compact(oh)))


def test_graded_paraexp_equals_oracle():
    w = setup()
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, 64)
    dt = 0.95 * g.cfl_dt()
    win = [0, 30, 75, 90, 140]
    pr, ef, hf = g.paraexp(dt, 4, win, w.sources, w.probes)
    g.close()
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt)
    opr, oef, ohf = og.paraexp(4, np.array(win), w.sources, w.probes)
    assert probe_relerr(pr, opr) <= TOL64
    assert relerr(ef, compact(oef)) <= TOL64 and relerr(hf, compact(ohf)) <= TOL64


@pytest.mark.parametrize("precision", [64, 32])
def test_graded_paraexp_leja_equals_oracle(precision):
    w = setup(lossy=False, seed=6)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, None, precision)
    dt = 0.95 * g.cfl_dt()
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, None, dt=dt)
    beta = expo.spectral_bound(og)
    u = dt * beta / 2
    tol = 1e-12 if precision == 64 else 1e-6
    q, m = expo.plan("leja", u, tol, precision)
    win = [0, 40, 80, 120]
    opts = fitgb.make_opts(homogeneous="leja", expo_substep=q, expo_degree=m)
    pr, ef, hf = g.paraexp(dt, 3, win, w.sources, w.probes, opts=opts)
    g.close()
    opr, oef, ohf = expo.paraexp(og, 3, win, w.sources, w.probes, "leja", q, m, dt_cfl=2.0 / beta)
    if precision == 64:
        b = 1e-10
    else:
        S = -(-120 // q)
        b = 4.0 * (S * 2.0 * q * u * tol + 2.0 * 120 * u * 2.0 ** -24) + 1e-5
    assert probe_relerr(pr, opr) <= b
    assert relerr(ef, compact(oef)) <= b and relerr(hf, compact(ohf)) <= b


@pytest.mark.parametrize("scheme", [0, 1])
def test_graded_adjoint_fp64_equals_oracle(scheme):
    """dJ/d eps_r on a lossy graded grid with non-uniform mu_r: the GPU's
    scaled-multiplier sweep with the graded scatter against the oracle's
    reverse sweep and coefficient chain rule (two independent derivations,
    the oracle's pinned by finite differences)."""
    w = setup(dims=(14, 9, 11), seed=9)
    prbs = w.probes[:3]
    dt = 0.9 * oracle.cfl_dt(w.dims, w.spacing, w.eps_r, w.mu_r)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, 64)
    J, grad = g.adjoint(dt, 120, w.sources, prbs, ckpt_every=13, opts=fitgb.make_opts(sigma_scheme=scheme))
    g.close()
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, sigma_scheme=scheme)
    J_ref, g_ref = og.adjoint(120, w.sources, prbs)
    assert abs(J - J_ref) <= 1e-11 * abs(J_ref)
    assert relerr(grad[None], g_ref[None]) <= 1e-9


def test_graded_adjoint_fp32_equals_oracle():
    w = setup(dims=(19, 13, 11), seed=10)
    prbs = w.probes[:3]
    dt = 0.9 * oracle.cfl_dt(w.dims, w.spacing, w.eps_r, w.mu_r)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, 32)
    J, grad = g.adjoint(dt, 200, w.sources, prbs)
    g.close()
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=True)
    J_ref, g_ref = og.adjoint(200, w.sources, prbs)
    assert abs(J - J_ref) <= 1e-4 * abs(J_ref)
    assert relerr(grad[None], g_ref[None]) <= 1e-3
