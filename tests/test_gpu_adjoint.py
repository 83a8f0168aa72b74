"""Adjoint gradient dJ/d eps_r (fit_adjoint_grad) against the CPU oracle's
adjoint and against central finite differences.

The GPU runs the reverse sweep as the forward leapfrog in scaled adjoint
variables and takes dJ/d eps_bar from the time differences of e; the oracle
follows the transpose of the step with the chain rule through ca(eps_bar)
and cb(eps_bar).  The two are different derivations of the same quantity.
"""
import numpy as np
import pytest

import oracle
from helpers import relerr
from paper_1705_08019_gb300 import fitgb
from paper_1705_08019_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fitgb.load()


def small_case(dims=(10, 8, 7), nsteps=120, scheme=0, seed=7):
    w = W.small_random(dims=dims, nsteps=nsteps, seed=seed, lossy=True)
    w.probes = w.probes[:3]
    return w


@pytest.mark.parametrize("scheme", [0, 1])
def test_adjoint_fp64_matches_oracle(scheme):
    w = small_case(scheme=scheme)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, None, w.sigma, dt=dt, sigma_scheme=scheme)
    J_ref, g_ref = og.adjoint(w.nsteps, w.sources, w.probes)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, w.sigma, 64)
    J, grad = g.adjoint(dt, w.nsteps, w.sources, w.probes, ckpt_every=11,
                        opts=fitgb.make_opts(sigma_scheme=scheme))
    g.close()
    assert abs(J - J_ref) <= 1e-11 * abs(J_ref)
    assert relerr(grad[None], g_ref[None]) <= 1e-9


def test_adjoint_fp32_matches_oracle():
    w = small_case(dims=(19, 13, 11), nsteps=200)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, None, w.sigma, dt=dt, round32=True)
    J_ref, g_ref = og.adjoint(w.nsteps, w.sources, w.probes)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, w.sigma, 32)
    J, grad = g.adjoint(dt, w.nsteps, w.sources, w.probes)
    g.close()
    assert abs(J - J_ref) <= 1e-4 * abs(J_ref)
    assert relerr(grad[None], g_ref[None]) <= 1e-3


@pytest.mark.parametrize("precision", [32, 64])
def test_checkpoint_interval_does_not_change_the_gradient(precision):
    w = small_case(dims=(14, 9, 12), nsteps=90)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, w.sigma, precision)
    outs = [g.adjoint(dt, w.nsteps, w.sources, w.probes, ckpt_every=c) for c in (0, 1, 7, 90, 200)]
    # J from a plain run's probe trace
    pr, _, _, _ = g.leapfrog(dt, w.nsteps, w.sources, w.probes)
    L = np.array([w.spacing[p["axis"]] for p in w.probes])
    J_plain = float(np.sum((pr / L) ** 2))
    g.close()
    for J, grad in outs[1:]:
        assert J == outs[0][0]
        assert np.array_equal(grad, outs[0][1])
    assert abs(outs[0][0] - J_plain) <= 1e-12 * J_plain


def test_adjoint_fp64_matches_gpu_finite_differences():
    w = small_case(dims=(12, 10, 9), nsteps=150)
    dt = 0.9 * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, w.sigma, 64)
    J, grad = g.adjoint(dt, w.nsteps, w.sources, w.probes)
    g.close()
    L = np.array([w.spacing[p["axis"]] for p in w.probes])

    def J_of(eps):
        gg = fitgb.Grid(w.dims, w.spacing, eps, None, w.sigma, 64)
        pr, _, _, _ = gg.leapfrog(dt, w.nsteps, w.sources, w.probes, opts=fitgb.make_opts(force_dt=1))
        gg.close()
        return float(np.sum((pr / L) ** 2))

    rng = np.random.default_rng(3)
    nx, ny, nz = w.dims
    for _ in range(6):
        idx = (rng.integers(1, nz - 1), rng.integers(1, ny - 1), rng.integers(1, nx - 1))
        ep, em = w.eps_r.copy(), w.eps_r.copy()
        ep[idx] = np.float32(w.eps_r[idx] + np.float32(1e-3))
        em[idx] = np.float32(w.eps_r[idx] - np.float32(1e-3))
        fd = (J_of(ep) - J_of(em)) / (float(ep[idx]) - float(em[idx]))
        assert abs(fd - grad[idx]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(grad).max())


def test_adjoint_device_outputs():
    import torch
    w = small_case()
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, w.sigma, 32)
    J, grad = g.adjoint(dt, w.nsteps, w.sources, w.probes)
    nx, ny, nz = w.dims
    Jd = torch.zeros(1, dtype=torch.float64, device="cuda")
    gd = torch.zeros((nz, ny, nx), dtype=torch.float64, device="cuda")
    fitgb.fit_adjoint_grad(g.handle, dt, w.nsteps, w.sources, w.probes, 0, Jd, gd)
    torch.cuda.synchronize()
    g.close()
    assert float(Jd.item()) == J
    assert np.array_equal(gd.cpu().numpy(), grad)


def test_fullsize_adjoint128_central_fd():
    """The 128^3 adjoint workload in full (10000 steps, checkpoints every 100):
    the FP32 adjoint gradient agrees with central finite differences
    (h = 1e-4, FP64 runs) on 16 seeded random cells to 1e-3 of the largest
    finite-difference magnitude among them."""
    w = W.adjoint128()
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, w.sigma, 32)
    J, grad = g.adjoint(dt, w.nsteps, w.sources, w.probes, ckpt_every=100)
    g.close()
    assert np.isfinite(grad).all() and J > 0
    L = np.array([w.spacing[p["axis"]] for p in w.probes])

    def J_of(eps):
        gg = fitgb.Grid(w.dims, w.spacing, eps, None, w.sigma, 64)
        pr, _, _, _ = gg.leapfrog(dt, w.nsteps, w.sources, w.probes, opts=fitgb.make_opts(force_dt=1))
        gg.close()
        return float(np.sum((pr / L) ** 2))

    fd, ad = [], []
    for k, j, i in W.fd_cells(w):
        ep, em = w.eps_r.copy(), w.eps_r.copy()
        ep[k, j, i] = np.float32(w.eps_r[k, j, i] + np.float32(1e-4))
        em[k, j, i] = np.float32(w.eps_r[k, j, i] - np.float32(1e-4))
        fd.append((J_of(ep) - J_of(em)) / (float(ep[k, j, i]) - float(em[k, j, i])))
        ad.append(grad[k, j, i])
    fd, ad = np.array(fd), np.array(ad)
    assert np.max(np.abs(fd - ad)) <= 1e-3 * np.max(np.abs(fd))


def test_autograd_function():
    import torch
    from paper_1705_08019_gb300.autograd import probe_energy
    w = small_case(dims=(16, 12, 10), nsteps=100)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    eps = torch.from_numpy(w.eps_r).cuda().requires_grad_(True)
    sig = torch.from_numpy(w.sigma).cuda()
    J = probe_energy(eps, w.spacing, dt, w.nsteps, w.sources, w.probes, sigma=sig)
    (3.0 * J).backward()
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, w.sigma, 32)
    J_ref, grad_ref = g.adjoint(dt, w.nsteps, w.sources, w.probes)
    g.close()
    assert abs(float(J.item()) - J_ref) <= 1e-12 * J_ref
    assert eps.grad.dtype == torch.float32
    assert np.allclose(eps.grad.cpu().numpy(), 3.0 * grad_ref, rtol=1e-6, atol=1e-6 * np.abs(grad_ref).max() * 3)
    # without a gradient request the library runs the forward pass and J only
    with torch.no_grad():
        J2 = probe_energy(eps.detach(), w.spacing, dt, w.nsteps, w.sources, w.probes, sigma=sig)
    assert abs(float(J2.item()) - J_ref) <= 1e-9 * J_ref


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-5)])
def test_functional_without_gradient_matches_oracle(precision, tol):
    """fit_adjoint_grad with a null gradient (the autograd binding's no-grad
    path): J = sum_n sum_p (e_p^n / L_p)^2 from the library equals the
    oracle's J on a graded lossy grid (per-probe edge lengths)."""
    import torch
    from paper_1705_08019_gb300.autograd import probe_energy
    w = W.graded_random(dims=(13, 11, 9))
    w.nsteps = 150
    w.probes = w.probes[:3]
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    og = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, None, w.sigma, dt=dt, round32=(precision == 32))
    J_ref, _ = og.adjoint(w.nsteps, w.sources, w.probes)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, w.sigma, precision)
    J = torch.zeros(1, dtype=torch.float64)
    fitgb.fit_adjoint_grad(g.handle, dt, w.nsteps, w.sources, w.probes, 0, J, None)
    g.close()
    assert abs(float(J[0]) - J_ref) <= tol * J_ref
    with torch.no_grad():
        J2 = probe_energy(torch.from_numpy(w.eps_r).cuda(), w.spacing, dt, w.nsteps, w.sources, w.probes,
                          sigma=torch.from_numpy(w.sigma).cuda(), precision=precision)
    assert float(J2.item()) == float(J[0])


def test_kept_forward_differences_give_the_same_gradient():
    """With a memory budget the forward sweep keeps e^{n+1} - e^n of its last
    checkpoint segments and the adjoint skips their recompute; the FP32
    gradient and J are the same bits with none, some or all segments kept."""
    w = small_case(dims=(64, 32, 32), nsteps=40)
    dt = w.cfl_fraction * oracle.cfl_dt(w.dims, w.spacing, w.eps_r)
    g = fitgb.Grid(w.dims, w.spacing, w.eps_r, None, w.sigma, 32)
    ref = g.adjoint(dt, w.nsteps, w.sources, w.probes, ckpt_every=4)
    per_step_mb = 3 * 64 * 32 * 32 * 4 / 2 ** 20
    for budget in (int(5.5 * 4 * per_step_mb), 64, 1024):   # 5 of 10 segments, all, all
        J, grad = g.adjoint(dt, w.nsteps, w.sources, w.probes, ckpt_every=4,
                            opts=fitgb.make_opts(adjoint_mem_mb=budget))
        assert J == ref[0]
        assert np.array_equal(grad, ref[1]), budget
    g.close()
