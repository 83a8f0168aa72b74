"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every comparison is element by element on the same seeded inputs: probe
traces, the full final e and h fields, and the interleaved energy W^n.
FP64 grids must agree to 1e-11 relative L2.  FP32 grids are run against the
oracle with the same float-rounded coefficients and must agree to
max(1e-5, 4 x the error of the oracle's float-storage model) per quantity
(see helpers.py for the derivation).  Sizes span several CTA tiles with ragged tails in x, y and z, and
several z chunks; edge cases cover one-cell-thick grids, tiny grids, a
non-zero initial state, both sigma schemes and non-uniform mu.
"""
import numpy as np
import pytest

import oracle
from helpers import (ENERGY_FACTOR, TOL32, TOL64, canonical, check, compact, oracle_grid, probe_relerr, relerr, tol32,
                     tol32_probe)
from paper_1705_08019_gb300 import fitgb
from paper_1705_08019_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not _gpu_available():
        pytest.skip("no CUDA device")
    fitgb.load()


def run_pair(w, nsteps, precision, scheme=0, energy=True, e0=None, h0=None, step0=0, opts=None):
    """Run the same leapfrog on the GPU and in the oracle; returns both."""
    g = fitgb.Grid.from_workload(w, precision)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r, w.mu_r)
    og = oracle_grid(w, dt, round32=(precision == 32), scheme=scheme)
    o = opts or fitgb.make_opts(sigma_scheme=scheme)
    ge0 = None if e0 is None else compact(e0)
    gh0 = None if h0 is None else compact(h0)
    pr, en, e, h = g.leapfrog(dt, nsteps, w.sources, w.probes, step0=step0, e=ge0, h=gh0, energy=energy, opts=o)
    opr, oen, oe, oh = og.leapfrog(nsteps, w.sources, w.probes, step0=step0, e=e0, h=h0, energy=energy)
    ref = (opr, oen, compact(oe), compact(oh))
    g.close()
    if precision == 32:
        sg = oracle_grid(w, dt, round32=True, scheme=scheme, store32=True)
        mpr, men, me, mh = sg.leapfrog(nsteps, w.sources, w.probes, step0=step0, e=e0, h=h0, energy=energy)
        tol = (tol32_probe(mpr, opr), tol32(men, oen, ENERGY_FACTOR) if energy else None, tol32(compact(me), ref[2]),
               tol32(compact(mh), ref[3]))
    else:
        tol = (TOL64,) * 4
    return (pr, en, e, h), ref, tol


def check_pair(gpu, ref, tol):
    pr, en, e, h = gpu
    opr, oen, oe, oh = ref
    check("probes", probe_relerr(pr, opr), tol[0])
    check("e", relerr(e, oe), tol[2])
    check("h", relerr(h, oh), tol[3])
    if en is not None:
        check("en", relerr(en, oen), tol[1])


def test_cfl_matches_oracle():
    for w in (W.cavity16(), W.small_random(mu=True)):
        g = fitgb.Grid.from_workload(w)
        assert abs(g.cfl_dt() / oracle.cfl_dt(w.dims, w.spacing, w.eps_r, w.mu_r) - 1.0) < 1e-14
        g.close()


def test_cavity16_fp64_leapfrog():
    """The plain-method workload in full: 16^3 PEC vacuum cavity, 2000 steps, FP64."""
    w = W.cavity16()
    gpu, ref, tol = run_pair(w, w.nsteps, 64)
    check_pair(gpu, ref, tol)


def test_cavity16_fp64_paraexp():
    w = W.cavity16()
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    g = fitgb.Grid.from_workload(w, 64)
    win = w.windows()
    pr, ef, hf = g.paraexp(dt, w.K, win, w.sources, w.probes)
    og = oracle_grid(w, dt, round32=False)
    opr, oef, ohf = og.paraexp(w.K, win, w.sources, w.probes)
    assert probe_relerr(pr, opr) <= TOL64
    assert relerr(ef, compact(oef)) <= TOL64
    assert relerr(hf, compact(ohf)) <= TOL64
    # and the superposition equals one sequential run (linearity, Sec. III)
    spr, _, se, sh = g.leapfrog(dt, w.nsteps, w.sources, w.probes)
    assert probe_relerr(pr, spr) <= TOL64
    assert relerr(ef, se) <= TOL64
    g.close()


SHAPES = [
    ((12, 10, 8), dict(lossy=True, mu=True)),      # non-uniform mu, lossy
    ((37, 11, 19), dict(lossy=True)),              # ragged in x, y, z
    ((70, 19, 45), dict(lossy=False)),             # several tiles and z chunks
    ((5, 3, 2), dict(lossy=True)),                 # tiny
    ((40, 40, 1), dict(lossy=False)),              # one cell thick (2-D wave)
    ((1, 6, 7), dict(lossy=True)),                 # one cell in x
]


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("dims,kw", SHAPES)
def test_leapfrog_fp32_matches_oracle(dims, kw, kernel):
    w = W.small_random(dims=dims, nsteps=300, **kw)
    if dims[2] == 1:
        w.sources = [dict(w.sources[0], axis=2, k=0)]
        w.probes = [dict(axis=2, i=3, j=4, k=0), dict(axis=2, i=dims[0] - 2, j=dims[1] // 2, k=0)]
    if dims[0] == 1:
        w.sources = [dict(w.sources[0], axis=0, i=0, j=3, k=3)]
        w.probes = [dict(axis=0, i=0, j=2, k=5), dict(axis=0, i=0, j=4, k=1)]
    gpu, ref, tol = run_pair(w, w.nsteps, 32, opts=fitgb.make_opts(kernel=kernel))
    check_pair(gpu, ref, tol)


@pytest.mark.parametrize("dims,kw", SHAPES[:3])
def test_leapfrog_fp64_matches_oracle(dims, kw):
    w = W.small_random(dims=dims, nsteps=200, **kw)
    gpu, ref, tol = run_pair(w, w.nsteps, 64)
    check_pair(gpu, ref, tol)


@pytest.mark.parametrize("precision", [32, 64])
def test_explicit_sigma_scheme(precision):
    w = W.small_random(dims=(20, 14, 9), nsteps=150)
    gpu, ref, tol = run_pair(w, w.nsteps, precision, scheme=1)
    check_pair(gpu, ref, tol)


@pytest.mark.parametrize("precision", [32, 64])
def test_nonzero_initial_state_and_offset(precision):
    w = W.small_random(dims=(21, 13, 11), nsteps=120)
    rng = np.random.default_rng(5)
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma)
    e0 = rng.standard_normal(og.field_shape)
    h0 = rng.standard_normal(og.field_shape) * 1e-2
    # entries that are not degrees of freedom are ignored by both sides
    e0 = canonical(compact(e0), w.dims)
    h0 = canonical(compact(h0), w.dims)
    nx, ny, nz = w.dims
    e0[0, :, 0, :] = 0; e0[0, 0, :, :] = 0
    e0[1, :, :, 0] = 0; e0[1, 0, :, :] = 0
    e0[2, :, :, 0] = 0; e0[2, :, 0, :] = 0
    h0[0, :, :, 0] = 0; h0[1, :, 0, :] = 0; h0[2, 0, :, :] = 0
    if precision == 32:
        e0 = e0.astype(np.float32).astype(np.float64)
        h0 = h0.astype(np.float32).astype(np.float64)
    gpu, ref, tol = run_pair(w, w.nsteps, precision, e0=e0, h0=h0, step0=37)
    check_pair(gpu, ref, tol)


def test_paraexp_fp32_matches_oracle_and_modes_agree():
    w = W.small_random(dims=(35, 17, 21), nsteps=240, K=5)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    win = np.array([0, 30, 61, 100, 170, 240])
    g = fitgb.Grid.from_workload(w, 32)
    pr, ef, hf = g.paraexp(dt, 5, win, w.sources, w.probes)
    og = oracle_grid(w, dt, round32=True)
    opr, oef, ohf = og.paraexp(5, win, w.sources, w.probes)
    mpr, mef, mhf = oracle_grid(w, dt, round32=True, store32=True).paraexp(5, win, w.sources, w.probes)
    oef, ohf, mef, mhf = compact(oef), compact(ohf), compact(mef), compact(mhf)
    check("probes", probe_relerr(pr, opr), tol32_probe(mpr, opr))
    check("ef", relerr(ef, oef), tol32(mef, oef))
    check("hf", relerr(hf, ohf), tol32(mhf, ohf))
    # plain per-window runs (one member after another) give the same bits
    pr1, ef1, hf1 = g.paraexp(dt, 5, win, w.sources, w.probes, opts=fitgb.make_opts(members_per_pass=1))
    assert np.array_equal(pr, pr1) and np.array_equal(ef, ef1) and np.array_equal(hf, hf1)
    pr2, ef2, hf2 = g.paraexp(dt, 5, win, w.sources, w.probes, opts=fitgb.make_opts(members_per_pass=2))
    assert np.array_equal(pr, pr2) and np.array_equal(ef, ef2) and np.array_equal(hf, hf2)
    # compensated FP32 superposition stays within the FP32 tolerance
    pr3, ef3, hf3 = g.paraexp(dt, 5, win, w.sources, w.probes, opts=fitgb.make_opts(sum_mode=1))
    assert np.array_equal(pr, pr3)
    check("ef_kahan", relerr(ef3, oef), tol32(mef, oef))
    check("hf_kahan", relerr(hf3, ohf), tol32(mhf, ohf))
    g.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_paraexp_with_initial_value(precision):
    w = W.small_random(dims=(16, 12, 10), nsteps=90, K=3)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    rng = np.random.default_rng(9)
    og = oracle_grid(w, dt, round32=(precision == 32))
    e0 = canonical(compact(rng.standard_normal(og.field_shape)), w.dims)
    h0 = np.zeros(og.field_shape)
    e0[0, :, 0, :] = 0; e0[0, 0, :, :] = 0
    e0[1, :, :, 0] = 0; e0[1, 0, :, :] = 0
    e0[2, :, :, 0] = 0; e0[2, :, 0, :] = 0
    if precision == 32:
        e0 = e0.astype(np.float32).astype(np.float64)
    win = np.array([10, 40, 55, 100])
    g = fitgb.Grid.from_workload(w, precision)
    pr, ef, hf = g.paraexp(dt, 3, win, w.sources, w.probes, e0=compact(e0))
    opr, oef, ohf = og.paraexp(3, win, w.sources, w.probes, e0=e0, h0=h0)
    oef, ohf = compact(oef), compact(ohf)
    if precision == 32:
        sg = oracle_grid(w, dt, round32=True, store32=True)
        mpr, mef, mhf = sg.paraexp(3, win, w.sources, w.probes, e0=e0, h0=h0)
        tp, te, th = tol32_probe(mpr, opr), tol32(compact(mef), oef), tol32(compact(mhf), ohf)
    else:
        tp = te = th = TOL64
    check("probes", probe_relerr(pr, opr), tp)
    check("ef", relerr(ef, oef), te)
    check("hf", relerr(hf, ohf), th)
    g.close()


def test_tiles_agree():
    w = W.small_random(dims=(70, 37, 23), nsteps=60)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    g = fitgb.Grid.from_workload(w, 32)
    ref = None
    combos = [(1, 32, 8, 8), (1, 32, 4, 16), (1, 32, 16, 0), (1, 64, 4, 5), (1, 64, 2, 7), (1, 16, 8, 3),
              (2, 32, 8, 8), (2, 32, 4, 16), (2, 32, 16, 0), (2, 64, 4, 5), (2, 32, 8, 1)]
    for kern, tx, ty, tz in combos:
        out = g.leapfrog(dt, w.nsteps, w.sources, w.probes, energy=True,
                         opts=fitgb.make_opts(tile_x=tx, tile_y=ty, tile_z=tz, kernel=kern))
        if ref is None:
            ref = out
            continue
        assert probe_relerr(out[0], ref[0]) <= 1e-6
        assert relerr(out[2], ref[2]) <= 1e-6 and relerr(out[3], ref[3]) <= 1e-6
        assert relerr(out[1], ref[1]) <= 1e-6
    g.close()


def test_device_pointers_match_host():
    import torch
    w = W.small_random(dims=(24, 16, 12), nsteps=80)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    g = fitgb.Grid.from_workload(w, 32)
    pr, en, e, h = g.leapfrog(dt, w.nsteps, w.sources, w.probes, energy=True)
    dev = torch.device("cuda")
    pr_d = torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev)
    en_d = torch.zeros(w.nsteps, dtype=torch.float64, device=dev)
    e_d = torch.zeros(g.field_shape, dtype=torch.float32, device=dev)
    h_d = torch.zeros(g.field_shape, dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream()
    fitgb.fit_leapfrog_run(g.handle, dt, w.nsteps, 0, w.sources, w.probes, pr_d, en_d, e_d, h_d, None, s)
    torch.cuda.synchronize()
    assert np.array_equal(pr_d.cpu().numpy(), pr)
    assert np.array_equal(e_d.cpu().numpy(), e) and np.array_equal(h_d.cpu().numpy(), h)
    assert np.allclose(en_d.cpu().numpy(), en, rtol=1e-12, atol=0)
    # device-side ParaExp outputs
    win = w.windows(K=4)
    hp, he, hh = g.paraexp(dt, 4, win, w.sources, w.probes)
    dp = torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev)
    de = torch.zeros(g.field_shape, dtype=torch.float64, device=dev)
    dh = torch.zeros(g.field_shape, dtype=torch.float64, device=dev)
    fitgb.paraexp_run(g.handle, dt, 4, win, w.sources, w.probes, dp, de, dh, None, None, None, s)
    torch.cuda.synchronize()
    assert np.array_equal(dp.cpu().numpy(), hp) and np.array_equal(de.cpu().numpy(), he)
    assert np.array_equal(dh.cpu().numpy(), hh)
    g.close()


def test_errors_are_reported():
    w = W.small_random(dims=(8, 8, 8), nsteps=10)
    g = fitgb.Grid.from_workload(w, 32)
    dt = g.cfl_dt()
    with pytest.raises(fitgb.FitError) as ei:
        g.leapfrog(1.01 * dt, 5)
    assert ei.value.status == fitgb.FIT_ERR_CFL
    g.leapfrog(1.01 * dt, 5, opts=fitgb.make_opts(force_dt=1))   # forced: accepted
    with pytest.raises(fitgb.FitError) as ei:   # source on a PEC edge
        g.leapfrog(dt, 5, [dict(axis=2, i=0, j=3, k=3, waveform=1, width=1e-11, delay=0)])
    assert ei.value.status == fitgb.FIT_ERR_ARG
    with pytest.raises(fitgb.FitError) as ei:   # probe outside the box
        g.leapfrog(dt, 5, probes=[dict(axis=0, i=8, j=0, k=0)])
    assert ei.value.status == fitgb.FIT_ERR_ARG
    with pytest.raises(fitgb.FitError) as ei:   # windows must increase
        g.paraexp(dt, 2, [0, 5, 5], w.sources, w.probes)
    assert ei.value.status == fitgb.FIT_ERR_ARG
    g.close()
    bad = w.eps_r.copy()
    bad[1, 2, 3] = -1.0
    with pytest.raises(fitgb.FitError) as ei:
        fitgb.Grid(w.dims, w.spacing, bad)
    assert ei.value.status == fitgb.FIT_ERR_NONFINITE
    bad[1, 2, 3] = np.nan
    with pytest.raises(fitgb.FitError) as ei:
        fitgb.Grid(w.dims, w.spacing, bad)
    assert ei.value.status == fitgb.FIT_ERR_NONFINITE


def test_fullsize_boxes256_light_cone():
    """The 256^3 lossy dielectric-box workload at full size, default launch
    configuration: after N steps from rest the fields are nonzero only within
    N cells (L-inf) of the source, and inside that cone they equal the
    oracle's run on a sub-box whose walls lie beyond the cone's reach."""
    w = W.boxes256(nsteps=24)
    N = w.nsteps
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    g = fitgb.Grid.from_workload(w, 32)
    pr, _, e, h = g.leapfrog(dt, N, w.sources, w.probes)
    g.close()
    s = w.sources[0]
    ci, cj, ck = s["i"], s["j"], s["k"]
    R = 2 * N + 2
    lo = (ci - R, cj - R, ck - R)
    sl = (slice(ck - R, ck + R + 1), slice(cj - R, cj + R + 1), slice(ci - R, ci + R + 1))
    sub = oracle.OracleGrid((2 * R + 1,) * 3, w.spacing, w.eps_r[sl], None, w.sigma[sl], dt=dt, round32=True)
    src = dict(s, i=R, j=R, k=R)
    _, _, oe, oh = sub.leapfrog(N, [src])
    oe, oh = compact(oe), compact(oh)
    sub32 = oracle.OracleGrid((2 * R + 1,) * 3, w.spacing, w.eps_r[sl], None, w.sigma[sl], dt=dt, round32=True,
                              store32=True)
    _, _, me, mh = sub32.leapfrog(N, [src])
    me, mh = compact(me), compact(mh)
    core = slice(R - N - 1, R + N + 2)
    ge = e[:, ck - R:ck + R + 1, cj - R:cj + R + 1, ci - R:ci + R + 1]
    gh = h[:, ck - R:ck + R + 1, cj - R:cj + R + 1, ci - R:ci + R + 1]
    c3 = (slice(None), core, core, core)
    check("ge", relerr(ge[c3], oe[c3]), tol32(me[c3], oe[c3]))
    check("gh", relerr(gh[c3], oh[c3]), tol32(mh[c3], oh[c3]))
    # outside the cone everything is still exactly zero
    mask = np.ones(e.shape[1:], bool)
    mask[ck - N - 1:ck + N + 2, cj - N - 1:cj + N + 2, ci - N - 1:ci + N + 2] = False
    assert not np.any(e[:, mask]) and not np.any(h[:, mask])
    assert not np.any(pr)   # probes lie 64 cells away: out of reach after 24 steps
