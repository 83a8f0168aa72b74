"""Failure detection without a GPU fault: every mbarrier wait of the TMA
step kernel is bounded.  A test hook announces bytes that never arrive, so
the first plane's wait of every tile runs out; the kernel records the
timeout, stores nothing, waits (bounded) for its own copies in flight and
returns.  The host reports FIT_ERR_TIMEOUT and the context stays usable."""
import numpy as np
import pytest

from paper_1705_08019_gb300 import fitgb
from paper_1705_08019_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fitgb.load()


@pytest.mark.parametrize("precision", [32, 64])
def test_bounded_wait_reports_timeout_and_recovers(precision):
    w = W.small_random(dims=(16, 12, 10), nsteps=6)
    g = fitgb.Grid.from_workload(w, precision)
    dt = 0.9 * g.cfl_dt()
    ref = g.leapfrog(dt, w.nsteps, w.sources, w.probes)
    with pytest.raises(fitgb.FitError) as ei:
        g.leapfrog(dt, w.nsteps, w.sources, w.probes,
                   opts=fitgb.make_opts(kernel=2, debug_wait_limit=2000, debug_extra_tx=16))
    assert ei.value.status == fitgb.FIT_ERR_TIMEOUT
    again = g.leapfrog(dt, w.nsteps, w.sources, w.probes)   # the context is still usable
    g.close()
    for a, b in zip(again, ref):
        if a is not None:
            assert np.array_equal(a, b)


def test_two_step_kernel_timeout_and_recovery():
    w = W.small_random(dims=(40, 20, 12), nsteps=6)
    g = fitgb.Grid.from_workload(w, 32)
    dt = 0.9 * g.cfl_dt()
    ref = g.leapfrog(dt, w.nsteps, w.sources, w.probes, opts=fitgb.make_opts(steps_per_launch=2))
    with pytest.raises(fitgb.FitError) as ei:
        g.leapfrog(dt, w.nsteps, w.sources, w.probes,
                   opts=fitgb.make_opts(steps_per_launch=2, debug_wait_limit=2000, debug_extra_tx=16))
    assert ei.value.status == fitgb.FIT_ERR_TIMEOUT
    again = g.leapfrog(dt, w.nsteps, w.sources, w.probes, opts=fitgb.make_opts(steps_per_launch=2))
    g.close()
    for a, b in zip(again, ref):
        if a is not None:
            assert np.array_equal(a, b)


def test_fused_leja_pair_timeout_and_recovery():
    w = W.small_random(dims=(40, 20, 12), lossy=False)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, None, 32)
    dt = 0.9 * g.cfl_dt()
    e0, h0 = W.random_state(w.dims, dtype=np.float32)
    ref = g.expo_propagate(dt, 8, e0, h0, w.probes, "leja", q=4, m=8)
    with pytest.raises(fitgb.FitError) as ei:
        e, h = np.array(e0), np.array(h0)
        pr = np.zeros((8, len(w.probes)))
        fitgb.fit_expo_propagate(g.handle, dt, 8, w.probes, pr, e, h,
                                 fitgb.make_opts(homogeneous="leja", expo_substep=4, expo_degree=8,
                                                 debug_wait_limit=2000, debug_extra_tx=16))
    assert ei.value.status == fitgb.FIT_ERR_TIMEOUT
    again = g.expo_propagate(dt, 8, e0, h0, w.probes, "leja", q=4, m=8)
    g.close()
    for a, b in zip(again, ref):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("nth", [0, 1, 2, 3, 5, 8])
def test_injected_oom_reports_and_grid_recovers(nth):
    """The allocator hook fails the nth device allocation of a ParaExp call on
    a fresh grid (coefficients, states, probe rows, sources, ...): the call
    returns FIT_ERR_OOM (or succeeds if it makes fewer allocations), and the
    same grid then reproduces the reference bit for bit."""
    w = W.small_random(dims=(19, 13, 11), nsteps=40, K=3)
    g0 = fitgb.Grid.from_workload(w, 32)
    dt = 0.9 * g0.cfl_dt()
    win = w.windows()
    ref = g0.paraexp(dt, w.K, win, w.sources, w.probes)
    g0.close()
    g = fitgb.Grid.from_workload(w, 32)
    fitgb.fit_debug_fail_alloc(nth)
    try:
        g.paraexp(dt, w.K, win, w.sources, w.probes)
        failed = False
    except fitgb.FitError as e:
        assert e.status == fitgb.FIT_ERR_OOM
        failed = True
    finally:
        fitgb.fit_debug_fail_alloc(-1)
    out = g.paraexp(dt, w.K, win, w.sources, w.probes)
    g.close()
    for a, b in zip(out, ref):
        assert np.array_equal(a, b)
    if nth == 0:
        assert failed
