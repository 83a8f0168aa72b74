"""The paper's 2-D cylindrical wave (Sec. IV-A) on the GPU.

20 m x 20 m x 1 m PEC box in vacuum, 40 x 40 x 1 cells (41 x 41 x 2 points,
n_dof = 20172), a z line current at the centre with the Gaussian pulse of
eq. (line_current), i(t) = exp(-4((t - s)/s)^2), s = 2e-8 s, run to
T = 2e-7 s at the CFL step of eq. (cfl).

* Energy (the experiment behind Fig. symplecticity): once the current has
  died out the interleaved discrete energy stays constant (Sec. II-A).
* Spectrum (Fig. frequencyE): ParaExp over 6 windows, with leapfrog for the
  homogeneous problems too, reproduces the leapfrog spectrum to rounding --
  the high-frequency noise the paper attributes to the Leja propagator does
  not arise.
"""
import os

import numpy as np
import pytest

import oracle
from helpers import probe_relerr, relerr
from paper_1705_08019_gb300 import fitgb
from paper_1705_08019_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fitgb.load()


def setup(n_xy=40):
    w = W.wave2d(n_xy=n_xy)
    g = fitgb.Grid.from_workload(w, 64)
    dt = g.cfl_dt()                          # eq. (cfl) at the limit, as in the paper
    nsteps = int(np.ceil(2e-7 / dt))
    return w, g, dt, nsteps


def test_wave2d_grid_and_dof_count():
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLDEN, "ndof_wave2d.txt"))
            if l.strip() and not l.startswith("#")]
    (px, py, pz, ndof) = rows[0]
    w, g, dt, nsteps = setup()
    assert (w.dims[0] + 1, w.dims[1] + 1, w.dims[2] + 1) == (px, py, pz)
    assert 2 * 3 * px * py * pz == ndof
    assert abs(dt - oracle.cfl_dt(w.dims, w.spacing, w.eps_r)) <= 1e-15 * dt
    g.close()


def test_wave2d_energy_constant_after_the_pulse():
    w, g, dt, nsteps = setup()
    pr, en, e, h = g.leapfrog(dt, nsteps, w.sources, w.probes, energy=True)
    g.close()
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, dt=dt)
    opr, oen, _, _ = og.leapfrog(nsteps, w.sources, w.probes, energy=True)
    assert relerr(en, oen) <= 1e-11 and probe_relerr(pr, opr) <= 1e-11
    s = w.sources[0]
    off = int(np.ceil((s["delay"] + 2.7 * s["width"]) / dt))   # envelope below 1e-12 afterwards
    assert off < nsteps - 20
    tail = en[off:]
    assert np.ptp(tail) <= 1e-12 * tail.mean()
    assert tail.mean() > 0


def test_wave2d_paraexp_spectrum_equals_leapfrog():
    w, g, dt, nsteps = setup()
    pr_lf, _, _, _ = g.leapfrog(dt, nsteps, w.sources, w.probes)
    win = np.array([(j * nsteps) // 6 for j in range(7)])
    pr_px, ef, hf = g.paraexp(dt, 6, win, w.sources, w.probes)
    g.close()
    assert probe_relerr(pr_px, pr_lf) <= 1e-12
    for p in range(pr_lf.shape[1]):
        a = np.abs(np.fft.rfft(pr_lf[:, p]))
        b = np.abs(np.fft.rfft(pr_px[:, p]))
        assert np.max(np.abs(a - b)) <= 1e-10 * a.max()


def test_wave2d_paraexp_leja_spectrum():
    """Fig. frequencyE: ParaExp over 6 windows with Leja's method for the
    homogeneous problems.  The GPU result equals the oracle's ParaExp-Leja to
    rounding, and its spectrum magnitude stays within 5% of the leapfrog
    spectrum below 100 MHz (the homogeneous parts propagate with the exact
    dispersion relation, the windows with the leapfrog one: at the CFL limit
    the traces drift apart in phase by O(dt^2), the spectra do not)."""
    from oracle import expo
    w, g, dt, nsteps = setup()
    pr_lf, _, _, _ = g.leapfrog(dt, nsteps, w.sources, w.probes)
    win = np.array([(j * nsteps) // 6 for j in range(7)])
    opts = fitgb.make_opts(homogeneous="leja", expo_tol=1e-10)
    pr_lj, ef, hf = g.paraexp(dt, 6, win, w.sources, w.probes, opts=opts)
    g.close()
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, dt=dt)
    opr, oef, ohf = expo.paraexp(og, 6, win, w.sources, w.probes, "leja", tol=1e-10, dt_cfl=dt)
    assert probe_relerr(pr_lj, opr) <= 1e-10
    f = np.fft.rfftfreq(nsteps, dt)
    band = f <= 1e8
    for p in range(pr_lf.shape[1]):
        a = np.abs(np.fft.rfft(pr_lf[:, p]))[band]
        b = np.abs(np.fft.rfft(pr_lj[:, p]))[band]
        assert np.linalg.norm(a - b) <= 0.05 * np.linalg.norm(a)


def test_wave2d_against_the_fine_reference():
    """Sec. IV-A compares the 41 x 41 point runs with a 121 x 121 point
    reference (Fig. frequencyE).  Here: 40 x 40 and 120 x 120 cells, probes
    at the same physical points, T = 2e-7 s, FP64 on the GPU.  Below 100 MHz
    (the pulse's band) the coarse leapfrog spectrum lies within 3% of the
    reference and the coarse ParaExp-Leja spectrum within 6% (measured:
    0.8-1.6% and 1.8-3.2%); the leapfrog trace itself within 8%."""
    T = 2e-7
    runs = {}
    for n in (40, 120):
        w = W.wave2d(n_xy=n)
        g = fitgb.Grid.from_workload(w, 64)
        dt = g.cfl_dt()
        ns = int(np.ceil(T / dt))
        pr, _, _, _ = g.leapfrog(dt, ns, w.sources, w.probes)
        if n == 40:
            win = np.array([(j * ns) // 6 for j in range(7)])
            pj, _, _ = g.paraexp(dt, 6, win, w.sources, w.probes,
                                 opts=fitgb.make_opts(homogeneous="leja", expo_tol=1e-10))
            runs["leja"] = pj
        g.close()
        runs[n] = (np.arange(1, ns + 1) * dt, pr, dt)
    tc, pc, dtc = runs[40]
    tf, pf, _ = runs[120]
    f = np.fft.rfftfreq(len(tc), dtc)
    band = f <= 1e8
    for p in range(pc.shape[1]):
        ref = np.interp(tc, tf, pf[:, p])
        assert np.linalg.norm(pc[:, p] - ref) <= 0.08 * np.linalg.norm(ref)
        A = np.abs(np.fft.rfft(ref))[band]
        B = np.abs(np.fft.rfft(pc[:, p]))[band]
        C = np.abs(np.fft.rfft(runs["leja"][:, p]))[band]
        assert np.linalg.norm(A - B) <= 0.03 * np.linalg.norm(A)
        assert np.linalg.norm(A - C) <= 0.06 * np.linalg.norm(A)
