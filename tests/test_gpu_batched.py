"""Batched ParaExp over many grids of uneven size (paraexp_run_batched): one
persistent launch per iteration advances every member of every grid.  Its
results equal paraexp_run on each problem alone, bit for bit, with and
without CUDA-graph capture and autotuning; one member grid is also checked
against the oracle."""
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


def make_batch():
    ws = []
    shapes = [(33, 17, 21), (20, 40, 9), (64, 8, 30), (7, 9, 50), (41, 23, 16)]
    for n, dims in enumerate(shapes):
        lossy = n in (1, 3)
        w = W.small_random(dims=dims, nsteps=80 + 17 * n, K=3 + (n % 3), seed=100 + n, lossy=lossy)
        ws.append(w)
    return ws


def run_problems(ws, batched, opts=None, precisions=None):
    grids, outs, probs = [], [], []
    for n, w in enumerate(ws):
        prec = precisions[n] if precisions else 32
        g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, prec)
        dt = w.cfl_fraction * g.cfl_dt()
        win = w.windows()
        pr = np.zeros((w.nsteps, len(w.probes)))
        ef = np.zeros(g.field_shape)
        hf = np.zeros(g.field_shape)
        grids.append(g)
        outs.append((pr, ef, hf))
        probs.append(dict(grid=g.handle, dt=dt, K=w.K, win=win, sources=w.sources, probes=w.probes,
                          probe_out=pr, e_final=ef, h_final=hf))
    if batched:
        fitgb.paraexp_run_batched(probs, opts)
    else:
        for q in probs:
            fitgb.paraexp_run(q["grid"], q["dt"], q["K"], q["win"], q["sources"], q["probes"], q["probe_out"],
                              q["e_final"], q["h_final"], opts=opts)
    for g in grids:
        g.close()
    return outs


def assert_same(a, b):
    for (p1, e1, h1), (p2, e2, h2) in zip(a, b):
        assert np.array_equal(p1, p2)
        assert np.array_equal(e1, e2)
        assert np.array_equal(h1, h2)


def test_batched_equals_per_problem_runs():
    ws = make_batch()
    ref = run_problems(ws, batched=False)
    assert_same(run_problems(ws, batched=True), ref)
    assert_same(run_problems(ws, batched=True, opts=fitgb.make_opts(use_graph=1)), ref)
    assert_same(run_problems(ws, batched=True, opts=fitgb.make_opts(autotune=1)), ref)
    assert_same(run_problems(ws, batched=True, opts=fitgb.make_opts(autotune=1, use_graph=1)), ref)
    assert_same(run_problems(ws, batched=True, opts=fitgb.make_opts(tile_x=64, tile_y=4, tile_z=7)), ref)


def test_batched_many_items_per_cta():
    """Enough work items (2000 to 4400) that every persistent CTA takes several,
    with short z chunks whose plane counts are not multiples of the ring
    depth: the planes of the next item, prefetched into the ring while the
    current one finishes, land in the right stages.  Bitwise equal to the
    problems run one by one."""
    shapes = [(96, 80, 60), (70, 90, 44), (100, 33, 51)]
    ws = [W.small_random(dims=d, nsteps=24 + 5 * n, K=4, seed=300 + n, lossy=(n == 1), mu=(n == 2))
          for n, d in enumerate(shapes)]
    ref = run_problems(ws, batched=False)
    assert_same(run_problems(ws, batched=True, opts=fitgb.make_opts(tile_x=32, tile_y=8, tile_z=6)), ref)
    assert_same(run_problems(ws, batched=True, opts=fitgb.make_opts(tile_x=64, tile_y=4, tile_z=5, stages=3)),
                ref)
    assert_same(run_problems(ws, batched=True, opts=fitgb.make_opts(tile_x=32, tile_y=8, tile_z=9, stages=3,
                                                                    use_graph=1)), ref)


def test_batched_with_an_fp64_grid_and_oracle():
    ws = make_batch()[:3]
    precisions = [32, 64, 32]
    out = run_problems(ws, batched=True, precisions=precisions)
    ref = run_problems(ws, batched=False, precisions=precisions)
    assert_same(out, ref)
    w = ws[0]
    pr, ef, hf = out[0]
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r, w.mu_r)
    win = w.windows()
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=True)
    opr, oef, ohf = og.paraexp(w.K, win, w.sources, w.probes)
    sg = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt, round32=True, store32=True)
    mpr, mef, mhf = sg.paraexp(w.K, win, w.sources, w.probes)
    check("probes", probe_relerr(pr, opr), tol32_probe(mpr, opr))
    check("ef", relerr(ef, compact(oef)), tol32(compact(mef), compact(oef)))
    check("hf", relerr(hf, compact(ohf)), tol32(compact(mhf), compact(ohf)))


def test_fullsize_batch64_equals_plain_runs():
    """The 64-cavity batch in full (sides 32..160, K = 8, 5000 steps): the
    batched persistent launch gives the same probe traces as the 64 problems
    run one after another."""
    import torch
    ws = W.cavity_batch()
    dev = torch.device("cuda")
    grids, probs_b, probs_p = [], [], []
    for w in ws:
        g = fitgb.Grid(w.dims, w.spacing, torch.from_numpy(w.eps_r).to(dev), None, None, 32)
        dt = w.cfl_fraction * g.cfl_dt()
        win = w.windows()
        grids.append(g)
        for lst in (probs_b, probs_p):
            lst.append(dict(grid=g.handle, dt=dt, K=w.K, win=win, sources=w.sources, probes=w.probes,
                            probe_out=torch.zeros((w.nsteps, len(w.probes)), dtype=torch.float64, device=dev)))
    fitgb.paraexp_run_batched(probs_b, fitgb.make_opts(use_graph=1))
    torch.cuda.synchronize()
    for q in probs_p:
        fitgb.paraexp_run(q["grid"], q["dt"], q["K"], q["win"], q["sources"], q["probes"], q["probe_out"])
    torch.cuda.synchronize()
    for a, b in zip(probs_b, probs_p):
        assert torch.equal(a["probe_out"], b["probe_out"])
        assert torch.isfinite(a["probe_out"]).all() and a["probe_out"].abs().max() > 0
    for g in grids:
        g.close()


def test_batched_with_leja_homogeneous_problems():
    """opts.homogeneous reaches every problem of a batch: the results equal
    paraexp_run with the same options, problem by problem."""
    ws = [W.small_random(dims=d, lossy=False, K=3, nsteps=60, seed=200 + n)
          for n, d in enumerate([(33, 17, 21), (20, 40, 9)])]
    opts = fitgb.make_opts(homogeneous="leja", expo_tol=1e-6)   # FP32 grids: 1e-6 is reachable
    ref = run_problems(ws, batched=False, opts=opts)
    assert_same(run_problems(ws, batched=True, opts=opts), ref)
    lf = run_problems(ws, batched=False)
    assert not np.array_equal(ref[0][0], lf[0][0])   # not the leapfrog result


def test_autotune_disk_cache(tmp_path):
    """FITGB_TUNE_CACHE keeps the autotuner's choice in a file keyed by device
    name and batch signature (precision, loss, every grid's dims and K): a
    tuned run appends one line; a fresh process that finds the line (and a
    line it cannot parse) skips the tuning and gives the same bits."""
    import json
    import os
    import subprocess
    import sys
    path = tmp_path / "tune.txt"
    os.environ["FITGB_TUNE_CACHE"] = str(path)
    try:
        ws = make_batch()[:3]
        a = run_problems(ws, True, fitgb.make_opts(autotune=1))
    finally:
        del os.environ["FITGB_TUNE_CACHE"]
    lines = path.read_text().splitlines()
    assert len(lines) == 2   # the lossless and the lossy problems are tuned as two groups
    sigs = []
    for line in lines:
        key, tx, ty, kz, st = line.split()
        dev, sig = key.split("|")
        assert "GB300" in dev and sig.startswith("fp32")
        assert int(st) in (3, 4) and int(kz) >= 1
        sigs.append(sig)
    for w in ws:
        nx, ny, nz = w.dims
        tag = ("fp32L" if w.sigma is not None else "fp32N")
        assert any(s.startswith(tag) and f"{nx}x{ny}x{nz}k{w.K}" in s for s in sigs)
    n_lines = len(lines)
    with open(path, "a") as f:
        f.write("not a tile line\n")
    code = ("import sys, json, numpy as np; sys.path[:0] = [%r, %r]\n"
            "import test_gpu_batched as t\nfrom paper_1705_08019_gb300 import fitgb\n"
            "out = t.run_problems(t.make_batch()[:3], True, fitgb.make_opts(autotune=1))\n"
            "print(json.dumps([[x.tolist() for x in o] for o in out]))\n") % (
        os.path.dirname(os.path.dirname(os.path.abspath(__file__))), os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, FITGB_TUNE_CACHE=str(path))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    b = json.loads(r.stdout.strip().splitlines()[-1])
    for oa, ob in zip(a, b):
        for x, y in zip(oa, ob):
            assert np.array_equal(x, np.array(y))
    assert len(path.read_text().splitlines()) == n_lines + 1   # nothing tuned, nothing appended
