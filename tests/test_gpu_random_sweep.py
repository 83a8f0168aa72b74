"""Randomised parity sweep: seeded random grids (sizes 1..48 per axis, random
eps_r, mu_r, sigma, spacings), random source and probe edges (sources on
degrees of freedom), random step offsets and window bounds; FP64 leapfrog
and ParaExp on the GPU against the oracle at 1e-11."""
import numpy as np
import pytest

import oracle
from helpers import TOL64, compact, probe_relerr, relerr
from paper_1705_08019_gb300 import fitgb
from paper_1705_08019_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fitgb.load()


def random_case(seed):
    rng = np.random.default_rng(seed)
    dims = tuple(int(v) for v in rng.integers(2, 49, 3))
    w = W.small_random(dims=dims, lossy=bool(rng.integers(0, 2)), mu=bool(rng.integers(0, 2)), seed=seed,
                       spacing=tuple(float(v) for v in rng.uniform(0.5e-3, 2e-3, 3)))
    nx, ny, nz = dims
    srcs = []
    for _ in range(int(rng.integers(1, 4))):
        a = int(rng.integers(0, 3))
        lo = [1, 1, 1]
        lo[a] = 0
        hi = [nx - 1, ny - 1, nz - 1]
        hi[a] = [nx, ny, nz][a] - 1
        q = [int(rng.integers(l, h + 1)) for l, h in zip(lo, hi)]
        srcs.append(dict(w.sources[0], axis=a, i=q[0], j=q[1], k=q[2], amp=float(rng.uniform(-1, 1))))
    prbs = [dict(axis=int(rng.integers(0, 3)), i=int(rng.integers(0, nx)), j=int(rng.integers(0, ny)),
                 k=int(rng.integers(0, nz))) for _ in range(int(rng.integers(1, 6)))]
    return w, srcs, prbs, rng


@pytest.mark.parametrize("seed", range(10))
def test_random_leapfrog_and_paraexp(seed):
    w, srcs, prbs, rng = random_case(1000 + seed)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, 64)
    dt = float(rng.uniform(0.5, 0.99)) * g.cfl_dt()
    n = int(rng.integers(1, 120))
    step0 = int(rng.integers(0, 30))
    pr, _, e, h = g.leapfrog(dt, n, srcs, prbs, step0=step0)
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, dt=dt)
    opr, _, oe, oh = og.leapfrog(n, srcs, prbs, step0=step0)
    assert probe_relerr(pr, opr) <= TOL64
    assert relerr(e, compact(oe)) <= TOL64 and relerr(h, compact(oh)) <= TOL64
    K = int(rng.integers(1, 6))
    cuts = np.sort(rng.choice(np.arange(1, n + 6), size=K, replace=False))
    win = np.concatenate([[step0], step0 + cuts]).astype(np.int64)
    pr, ef, hf = g.paraexp(dt, K, win, srcs, prbs)
    g.close()
    opr, oef, ohf = og.paraexp(K, win, srcs, prbs)
    assert probe_relerr(pr, opr) <= TOL64
    assert relerr(ef, compact(oef)) <= TOL64 and relerr(hf, compact(ohf)) <= TOL64
