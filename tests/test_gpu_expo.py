"""Exponential propagators of the homogeneous ParaExp problems on the GPU
(Sec. III-B; fit_expo_propagate and paraexp_run with
opts.homogeneous = LEJA / TAYLOR) against the oracle (oracle/expo.py).

FP64: both sides evaluate the same interpolant (same points, substep and
degree), so they agree to rounding of ~1e2 operator applications per substep
with Newton terms of size <= 1e2 relative to the result: 1e-10.
FP32: the planner's own bound -- each substep errs by at most 2 c eps_A in
the energy norm including the rounding term u_p H_m, so S substeps by
S 2 c eps_A -- plus the rounding of the float coefficients cb, ch (relative
2^-24, a frequency shift whose phase error grows like 2^-24 beta t), with a
factor 4 of margin."""
import numpy as np
import pytest

import oracle
from oracle import expo
from helpers import canonical, compact, probe_relerr, relerr
from paper_1705_08019_gb300 import fitgb
from paper_1705_08019_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL_EXPO64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fitgb.load()


def grid_pair(dims=(37, 19, 45), mu=False, seed=11, precision=64):
    w = W.small_random(dims=dims, lossy=False, mu=mu, seed=seed, precision=precision)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, None, precision)
    dtc = g.cfl_dt()
    dt = 0.95 * dtc
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, None, dt=dt)
    return w, g, og, dt, dtc


def fp32_bound(kind, nsteps, u, tol):
    q, m = expo.plan(kind, u, tol, 32)
    S = -(-nsteps // q)
    return 4.0 * (S * 2.0 * q * u * tol + 2.0 * nsteps * u * 2.0 ** -24) + 1e-6


@pytest.mark.parametrize("kind,mu", [("leja", False), ("leja", True), ("taylor", False)])
def test_propagate_fp64_equals_oracle(kind, mu):
    w, g, og, dt, dtc = grid_pair(mu=mu)
    e0, h0 = W.random_state(w.dims)
    nsteps = 71
    q, m = expo.plan(kind, dt / dtc, 1e-12, 64)
    pr, e1, h1 = g.expo_propagate(dt, nsteps, e0, h0, w.probes, kind, q=q, m=m)
    opr, oe, oh = expo.propagate(og, nsteps, canonical(e0, w.dims), canonical(h0, w.dims), w.probes, kind, q, m,
                                 dt_cfl=dtc)
    g.close()
    assert probe_relerr(pr, opr) <= TOL_EXPO64
    assert relerr(e1, compact(oe)) <= TOL_EXPO64
    assert relerr(h1, compact(oh)) <= TOL_EXPO64


def test_propagate_planned_by_the_library_and_fp32():
    w, g, og, dt, dtc = grid_pair(seed=12)
    e0, h0 = W.random_state(w.dims, seed=5)
    nsteps = 90
    pr, e1, h1 = g.expo_propagate(dt, nsteps, e0, h0, w.probes, "leja", tol=1e-12)   # planned inside
    opr, oe, oh = expo.propagate(og, nsteps, canonical(e0, w.dims), canonical(h0, w.dims), w.probes, "leja",
                                 tol=1e-12, dt_cfl=dtc)
    g.close()
    assert probe_relerr(pr, opr) <= TOL_EXPO64 and relerr(e1, compact(oe)) <= TOL_EXPO64
    g32 = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, None, 32)
    tol = 1e-6
    pr32, e32, h32 = g32.expo_propagate(dt, nsteps, e0, h0, w.probes, "leja", tol=tol)
    g32.close()
    b = fp32_bound("leja", nsteps, dt / dtc, tol)
    assert probe_relerr(pr32, opr) <= b
    assert relerr(e32, compact(oe)) <= b and relerr(h32, compact(oh)) <= b


@pytest.mark.parametrize("kind", ["leja", "taylor"])
def test_paraexp_expo_fp64_equals_oracle(kind):
    w, g, og, dt, dtc = grid_pair(dims=(33, 17, 21), seed=13)
    K, n = 4, 160
    win = [n * j // K for j in range(K + 1)]
    q, m = expo.plan(kind, dt / dtc, 1e-12, 64)
    opts = fitgb.make_opts(homogeneous=kind, expo_substep=q, expo_degree=m)
    pr, ef, hf = g.paraexp(dt, K, win, w.sources, w.probes, opts=opts)
    st = fitgb.fit_last_stats(g.handle)
    g.close()
    opr, oef, ohf = expo.paraexp(og, K, win, w.sources, w.probes, kind, q, m, dt_cfl=dtc)
    assert probe_relerr(pr, opr) <= TOL_EXPO64
    assert relerr(ef, compact(oef)) <= TOL_EXPO64
    assert relerr(hf, compact(ohf)) <= TOL_EXPO64
    # operator applications: m per substep of every homogeneous member
    want = sum(m * -(-(n - win[j]) // q) for j in range(1, K))
    assert st["expo_applications"] == want


def test_paraexp_expo_with_initial_value_and_ragged_windows():
    w, g, og, dt, dtc = grid_pair(dims=(20, 40, 9), seed=14)
    win = [5, 40, 41, 97, 130]
    K = 4
    e0, h0 = W.random_state(w.dims, seed=9)
    opts = fitgb.make_opts(homogeneous="leja", expo_tol=1e-12)
    pr, ef, hf = g.paraexp(dt, K, win, w.sources, w.probes, e0=e0, h0=h0, opts=opts)
    g.close()
    opr, oef, ohf = expo.paraexp(og, K, win, w.sources, w.probes, "leja", tol=1e-12, dt_cfl=dtc,
                                 e0=canonical(e0, w.dims), h0=canonical(h0, w.dims))
    assert probe_relerr(pr, opr) <= TOL_EXPO64
    assert relerr(ef, compact(oef)) <= TOL_EXPO64
    assert relerr(hf, compact(ohf)) <= TOL_EXPO64


def test_paraexp_expo_fp32():
    w, g64, og, dt, dtc = grid_pair(dims=(33, 17, 21), seed=15)
    g64.close()
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, None, 32)
    K, n, tol = 4, 160, 1e-6
    win = [n * j // K for j in range(K + 1)]
    pr, ef, hf = g.paraexp(dt, K, win, w.sources, w.probes, opts=fitgb.make_opts(homogeneous="leja", expo_tol=tol))
    g.close()
    q, m = expo.plan("leja", dt / dtc, tol, 32)
    opr, oef, ohf = expo.paraexp(og, K, win, w.sources, w.probes, "leja", q, m, dt_cfl=dtc)
    # the leapfrog windows add their own FP32 error (about 1e-6 here)
    b = fp32_bound("leja", n, dt / dtc, tol) + 1e-5
    assert probe_relerr(pr, opr) <= b
    assert relerr(ef, compact(oef)) <= b and relerr(hf, compact(ohf)) <= b


def test_expo_rejects_unsupported_requests():
    w = W.small_random(dims=(12, 10, 8), lossy=True)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, w.sigma, 64)
    dt = 0.95 * g.cfl_dt()
    with pytest.raises(fitgb.FitError) as ei:
        g.paraexp(dt, 2, [0, 10, 20], w.sources, w.probes, opts=fitgb.make_opts(homogeneous="leja"))
    assert ei.value.status == fitgb.FIT_ERR_UNSUPPORTED
    g.close()
    w = W.small_random(dims=(12, 10, 8), lossy=False)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, None, 64)
    with pytest.raises(fitgb.FitError) as ei:
        g.paraexp(dt, 2, [0, 10, 20], w.sources, w.probes,
                  opts=fitgb.make_opts(homogeneous="leja", sum_mode=1))
    assert ei.value.status == fitgb.FIT_ERR_ARG
    with pytest.raises(fitgb.FitError):
        g.expo_propagate(dt, 5, *W.random_state(w.dims), kind="leja", q=3, m=7)   # odd degree
    g.close()


@pytest.mark.parametrize("precision,mu", [(64, False), (64, True), (32, False)])
def test_fused_pair_kernel_equals_plain_kernels(precision, mu):
    """The TMA pair kernel (opts.kernel = 2; the FP32 default) and the two
    plain operator launches per pair (opts.kernel = 1; the FP64 default)
    evaluate the same recurrence: FP64 agrees to rounding, FP32 to a few
    float ulps of the largest terms."""
    w, g64, og, dt, dtc = grid_pair(dims=(45, 21, 70), mu=mu, seed=21)
    g64.close()
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, None, precision)
    e0, h0 = W.random_state(w.dims, seed=3)
    out = []
    for kernel in (2, 1):
        e = np.array(e0, dtype=g.dtype)
        h = np.array(h0, dtype=g.dtype)
        pr = np.zeros((100, len(w.probes)))
        opts = fitgb.make_opts(homogeneous="leja", expo_substep=12, expo_degree=24, kernel=kernel)
        fitgb.fit_expo_propagate(g.handle, dt, 100, w.probes, pr, e, h, opts)
        out.append((pr, e, h))
    g.close()
    tol = 1e-12 if precision == 64 else 2e-5
    (p1, e1, h1), (p2, e2, h2) = out
    assert probe_relerr(p1, p2) <= tol and relerr(e1, e2) <= tol and relerr(h1, h2) <= tol
