"""FP32 fields with a bfloat16 residual (precision 40).

Each stored e and h value is a float plus the rounding residual of that float
kept as a bfloat16; updates are FP32 arithmetic with the increment summed in by
a fast two-sum, the magnetic update's curl C e formed from two error-free
same-component differences, and the coefficient products split by one FMA.

Compared with the FP64 oracle on the same float-rounded coefficients.  What
remains is the float rounding of the dual curl C~h and of the increments --
an ulp of the increment per step, not an ulp of the field -- and the
residual's own rounding (2^-9 of half an ulp).  The tolerance is therefore
stated against the plain FP32 path's own error on the same case: the
residual path must be at least RES_GAIN times more accurate; the full-size
test holds it to the method's 1e-5 target outright.  Each test records the
achieved error and the bound it was held to.
"""
import numpy as np
import pytest

import oracle
from helpers import compact, probe_relerr, relerr
from paper_1705_08019_gb300 import fitgb
from paper_1705_08019_gb300 import workloads as W

pytestmark = pytest.mark.gpu
# required gain over plain FP32 on the same case: a float32 emulation of both
# arithmetics gives 9.6-10.7x on 32^3 and 48^3 boxes over 3000-8000 steps; on
# GB300 the parity cases below gain 5.1x (the 5x3x2 grid's e) to 13.5x
RES_GAIN = 4.0
TARGET = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fitgb.load()


def _errs(pr, e, h, ref):
    opr, oe, oh = ref
    return {"probes": probe_relerr(pr, opr), "e": relerr(e, compact(oe)), "h": relerr(h, compact(oh))}


def _check(record_property, name, res, plain):
    """res[k] <= max(small floor, plain[k] / RES_GAIN) for every quantity (on
    small driven grids neither path reaches 1e-5 for every component; the
    full-size test holds the residual path to the target itself)."""
    for k in res:
        bound = max(2e-8, plain[k] / RES_GAIN)
        record_property(f"{name}_{k}_err", res[k])
        record_property(f"{name}_{k}_plain_fp32_err", plain[k])
        record_property(f"{name}_{k}_bound", bound)
        assert res[k] <= bound, (name, k, res[k], bound, plain[k])


@pytest.mark.parametrize("kernel,tile", [(2, (64, 4)), (2, (32, 8)), (3, (64, 4))])
@pytest.mark.parametrize("dims,kw", [((37, 11, 19), dict(lossy=True)), ((12, 10, 8), dict(lossy=True, mu=True)),
                                     ((70, 19, 45), dict(lossy=False)), ((5, 3, 2), dict(lossy=True)),
                                     ((67, 9, 30), dict(lossy=True)), ((131, 6, 5), dict(lossy=True, mu=True))])
def test_residual_leapfrog_matches_oracle(dims, kw, kernel, tile, record_property):
    """Both residual kernels (two cells per thread, one cell per thread) and
    both tiles of the first, on odd and even widths, one- and many-tile grids."""
    w = W.small_random(dims=dims, nsteps=600, **kw)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r, w.mu_r)
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=True)
    opr, oen, oe, oh = og.leapfrog(w.nsteps, w.sources, w.probes, energy=True)
    out = {}
    for prec in (40, 32):
        g = fitgb.Grid.from_workload(w, prec)
        opts = fitgb.make_opts(kernel=kernel, tile_x=tile[0], tile_y=tile[1]) if prec == 40 else None
        pr, en, e, h = g.leapfrog(dt, w.nsteps, w.sources, w.probes, energy=True, opts=opts)
        g.close()
        out[prec] = (_errs(pr, e, h, (opr, oe, oh)), en)
    _check(record_property, "leapfrog", out[40][0], out[32][0])
    assert relerr(out[40][1], oen) <= 1e-6   # energy uses the float-rounded M_eps, M_mu


def test_residual_initial_state_and_paraexp(record_property):
    """A run continued from a state (the oracle's fields after 150 driven
    steps, handed over in FP64 and split into float + residual), and ParaExp
    from zero; both against the oracle with the RES_GAIN bound.  A white-noise
    initial state (every mode up to the grid's highest, so the per-step
    increment is as large as the field) is only held to the plain FP32
    error."""
    w = W.small_random(dims=(21, 13, 11), nsteps=250, K=4)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=True)
    _, _, e0, h0 = og.leapfrog(150, w.sources, w.probes)
    ref = og.leapfrog(w.nsteps, w.sources, w.probes, e=e0, h=h0, step0=150)
    rng = np.random.default_rng(4)
    n0 = rng.standard_normal(og.field_shape)
    m0 = rng.standard_normal(og.field_shape) * 1e-2
    # only degrees of freedom: nothing at index n, no e tangential to a wall, no h normal to one
    n0[:, -1] = 0; n0[:, :, -1] = 0; n0[:, :, :, -1] = 0
    m0[:, -1] = 0; m0[:, :, -1] = 0; m0[:, :, :, -1] = 0
    n0[0, :, 0, :] = 0; n0[0, 0, :, :] = 0; n0[1, :, :, 0] = 0; n0[1, 0, :, :] = 0
    n0[2, :, :, 0] = 0; n0[2, :, 0, :] = 0
    m0[0, :, :, 0] = 0; m0[1, :, 0, :] = 0; m0[2, 0, :, :] = 0
    nref = og.leapfrog(w.nsteps, w.sources, w.probes, e=n0, h=m0, step0=11)
    win = np.array([0, 50, 101, 199, 250])
    pref = og.paraexp(4, win, w.sources, w.probes)
    res = {}
    for prec in (40, 32):
        g = fitgb.Grid.from_workload(w, prec)
        dtp = np.float64 if prec == 40 else np.float32
        pr, _, e, h = g.leapfrog(dt, w.nsteps, w.sources, w.probes, e=compact(e0).astype(dtp),
                                 h=compact(h0).astype(dtp), step0=150)
        lf = _errs(pr, e, h, (ref[0], ref[2], ref[3]))
        pr, _, e, h = g.leapfrog(dt, w.nsteps, w.sources, w.probes, e=compact(n0).astype(dtp),
                                 h=compact(m0).astype(dtp), step0=11)
        nz = _errs(pr, e, h, (nref[0], nref[2], nref[3]))
        pr, ef, hf = g.paraexp(dt, 4, win, w.sources, w.probes)
        g.close()
        res[prec] = (lf, _errs(pr, ef, hf, pref), nz)
    _check(record_property, "continued", res[40][0], res[32][0])
    _check(record_property, "paraexp", res[40][1], res[32][1])
    for k in res[40][2]:
        record_property(f"white_noise_{k}_err", res[40][2][k])
        record_property(f"white_noise_{k}_bound", res[32][2][k])
        assert res[40][2][k] <= res[32][2][k], (k, res[40][2][k], res[32][2][k])


def test_residual_paraexp_batching_is_bitwise():
    """All members in one launch, one member per launch and two per launch give
    identical bits (the superposition order is fixed)."""
    w = W.small_random(dims=(29, 17, 13), nsteps=240, K=5)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    g = fitgb.Grid.from_workload(w, 40)
    win = w.windows()
    outs = [g.paraexp(dt, w.K, win, w.sources, w.probes, opts=fitgb.make_opts(members_per_pass=m))
            for m in (0, 1, 2)]
    g.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


def test_residual_rejects_unsupported():
    w = W.small_random(dims=(9, 8, 7), nsteps=10)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    g = fitgb.Grid.from_workload(w, 40)
    with pytest.raises(fitgb.FitError) as ei:
        g.adjoint(dt, 10, w.sources, w.probes[:1])
    assert ei.value.status == fitgb.FIT_ERR_UNSUPPORTED
    with pytest.raises(fitgb.FitError) as ei:
        g.paraexp(dt, 2, np.array([0, 5, 10]), w.sources, w.probes, opts=fitgb.make_opts(sum_mode=1))
    assert ei.value.status == fitgb.FIT_ERR_UNSUPPORTED
    g.close()


def _fullsize(w, torch, dev, prec, paraexp, flags=0):
    """Probe trace and final e, h of the 256^3 workload (FP64 numpy)."""
    eps = torch.from_numpy(w.eps_r).to(dev)
    sig = torch.from_numpy(w.sigma).to(dev)
    g = fitgb.Grid(w.dims, w.spacing, eps, None, sig, prec, flags=flags)
    dt = w.cfl_fraction * g.cfl_dt()
    pr = torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev)
    if paraexp:
        e = torch.zeros(g.field_shape, dtype=torch.float64, device=dev)
        h = torch.zeros_like(e)
        fitgb.paraexp_run(g.handle, dt, w.K, w.windows(), w.sources, w.probes, pr, e, h)
    else:
        T = torch.float32 if prec == 32 else torch.float64
        e = torch.zeros(g.field_shape, dtype=T, device=dev)
        h = torch.zeros_like(e)
        fitgb.fit_leapfrog_run(g.handle, dt, w.nsteps, 0, w.sources, w.probes, pr, None, e, h)
    torch.cuda.synchronize()
    out = (pr.cpu().numpy(), e.double().cpu().numpy(), h.double().cpu().numpy())
    g.close()
    del e, h, pr
    torch.cuda.empty_cache()
    return out


def test_fullsize_boxes256_paraexp_field_error(record_property):
    """The 256^3 lossy boxes solved by ParaExp (K = 16, 20000 steps) on the
    residual path and on plain FP32, against one sequential FP64 leapfrog run
    on the same float-rounded coefficients (FIT_FLAG_COEF_FLOAT; ParaExp equals
    the sequential run in exact arithmetic).  The residual path meets the
    1e-5 target; plain FP32 stays within 2.5e-5."""
    import torch
    w = W.boxes256()
    dev = torch.device("cuda")
    ref = _fullsize(w, torch, dev, 64, False, flags=fitgb.FIT_FLAG_COEF_FLOAT)
    for prec, bound in ((40, TARGET), (32, 2.5e-5)):
        pr, e, h = _fullsize(w, torch, dev, prec, True)
        errs = {"probes": probe_relerr(pr, ref[0]), "e": relerr(e, ref[1]), "h": relerr(h, ref[2])}
        for k, v in errs.items():
            record_property(f"fp{prec}_{k}_err", v)
        record_property(f"fp{prec}_bound", bound)
        assert max(errs.values()) <= bound, (prec, errs)
