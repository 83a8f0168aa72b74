"""Pins of the oracle's exponential propagators (oracle/expo.py): Leja and
Taylor interpolation of the matrix exponential (Sec. III-B) and ParaExp with
exponential homogeneous problems (Sec. III, Algorithm 1, eqs. averaging1/2).

Each pin comes from outside the oracle: the dense FIT matrices built from
their incidence definitions (tests/dense_fit.py) and scipy's expm, the
eigen-decomposition of A, the interpolation property of divided
differences, a brute-force maximisation for the Leja points, and the dt^2
convergence of ParaExp to the leapfrog solution."""
import math

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from oracle import expo
from dense_fit import DenseFIT

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def tiny_grid(dims=(4, 4, 4), seed=3, u=0.95):
    rng = np.random.default_rng(seed)
    eps = rng.uniform(1.0, 4.0, size=dims[::-1]).astype(np.float32)
    mu = rng.uniform(1.0, 2.0, size=dims[::-1]).astype(np.float32)
    sp = (1e-3, 1.3e-3, 0.8e-3)
    dtc = oracle.cfl_dt(dims, sp, eps, mu)
    og = oracle.OracleGrid(dims, sp, eps, mu, dt=u * dtc)
    return og, dtc


def dense_A(og):
    """A of eq. (FIT_ode_2) over the degrees of freedom, u = [h_dofs, e_dofs]."""
    d = DenseFIT((og.nx, og.ny, og.nz))
    ie, ih = np.flatnonzero(d.edge_dof), np.flatnonzero(d.face_dof)
    me, mm = og.meps.ravel()[ie], og.mmu.ravel()[ih]
    Cr = d.C[np.ix_(ih, ie)]
    top = -np.diag(mm ** -0.5) @ Cr @ np.diag(me ** -0.5)
    A = np.block([[np.zeros((len(ih), len(ih))), top], [-top.T, np.zeros((len(ie), len(ie)))]])
    return A, ie, ih


def random_state(og, seed):
    d = DenseFIT((og.nx, og.ny, og.nz))
    rng = np.random.default_rng(seed)
    e = np.where(d.edge_dof, rng.standard_normal(d.N), 0.0).reshape(og.field_shape)
    h = np.where(d.face_dof, rng.standard_normal(d.N), 0.0).reshape(og.field_shape)
    return e, h


def test_leja_points_are_greedy_maximisers():
    etas = expo.leja_etas(12)
    assert etas[0] == 2.0
    assert abs(etas[1] - 2.0 / math.sqrt(3.0)) <= 2.0 / expo.NGRID      # argmax of eta (4 - eta^2)
    assert len(set(etas.tolist())) == len(etas) and np.all((etas > 0) & (etas <= 2))
    fine = np.linspace(0.0, 2.0, 400001)
    chosen = [0.0]
    for eta in etas:
        def logprod(x):
            s = np.zeros_like(x)
            for c in chosen:
                s += np.log(np.abs(x - c)) + (np.log(x + c) if c > 0 else 0.0)
            return s
        with np.errstate(divide="ignore"):
            best = logprod(fine).max()
        assert logprod(np.array([eta]))[0] >= best - 1e-5
        chosen.append(eta)
    xi = expo.nodes("leja", 10)
    assert xi[0] == 0 and np.all(xi[1::2] == np.conj(xi[2::2]))


@pytest.mark.parametrize("c", [0.7, 6.0, 25.0])
def test_divided_differences_interpolate_exp(c):
    xi = expo.nodes("leja", 40)
    d = expo.divided_differences(xi, c)
    for k, z in enumerate(xi):                  # Newton form at each point = exp(c z)
        w, p = 1.0 + 0j, 0j
        for l in range(len(xi)):
            p += d[l] * w
            w *= z - xi[l]
        assert abs(p - np.exp(c * z)) <= 1e-12 * max(1.0, math.exp(c))
    assert abs(d[1] - (np.exp(c * xi[1]) - 1.0) / xi[1]) <= 1e-14 * abs(d[1]) * 10
    t = expo.divided_differences(expo.nodes("taylor", 10), c)
    assert np.allclose(t, [c ** k / math.factorial(k) for k in range(11)], rtol=1e-15, atol=0)


def test_apply_A_is_the_dense_skew_matrix():
    og, _ = tiny_grid()
    A, ie, ih = dense_A(og)
    assert np.allclose(A, -A.T, atol=0)
    e, h = random_state(og, 1)
    se, sh = np.sqrt(og.meps), np.sqrt(og.mmu)
    oe, oh = og.apply_A(se * e, sh * h)
    u = np.concatenate([(sh * h).ravel()[ih], (se * e).ravel()[ie]])
    v = A @ u
    assert rel(oh.ravel()[ih], v[: len(ih)]) <= 1e-14
    assert rel(oe.ravel()[ie], v[len(ih):]) <= 1e-14
    mask_e = np.ones(oe.size, bool); mask_e[ie] = False
    mask_h = np.ones(oh.size, bool); mask_h[ih] = False
    assert not oe.ravel()[mask_e].any() and not oh.ravel()[mask_h].any()


def test_spectrum_inside_the_cfl_interval():
    """The interval i[-2/dt_CFL, 2/dt_CFL] the propagators interpolate on holds
    every eigenvalue of A (eq. (cfl) bounds ||A||_2)."""
    for seed in (3, 4, 5):
        og, dtc = tiny_grid(seed=seed)
        A, _, _ = dense_A(og)
        lam = np.linalg.eigvals(A)
        assert np.abs(lam.real).max() <= 1e-6 * np.abs(lam).max()
        assert np.abs(lam.imag).max() * dtc <= 2.0
        assert np.abs(lam.imag).max() * dtc >= 1.0           # and the bound is not loose by 2x


@pytest.mark.parametrize("kind", ["leja", "taylor"])
def test_propagate_equals_dense_exponential(kind):
    og, dtc = tiny_grid()
    A, ie, ih = dense_A(og)
    e0, h0 = random_state(og, 2)
    probes = [dict(axis=2, i=1, j=2, k=1), dict(axis=0, i=2, j=1, k=3), dict(axis=1, i=3, j=0, k=2)]
    probes = [p for p in probes]
    nsteps = 37
    q, m = expo.plan(kind, og.dt / dtc, 1e-12)
    pr, ef, hf = expo.propagate(og, nsteps, e0, h0, probes, kind, q, m, dt_cfl=dtc)
    se, sh = np.sqrt(og.meps).ravel(), np.sqrt(og.mmu).ravel()
    u0 = np.concatenate([(sh * h0.ravel())[ih], (se * e0.ravel())[ie]])
    d = DenseFIT((og.nx, og.ny, og.nz))
    for n in (1, 5, q, q + 1, nsteps):
        u = sl.expm(n * og.dt * A) @ u0
        e = np.zeros(d.N); e[ie] = u[len(ih):] / se[ie]
        e = e.reshape(og.field_shape)
        want = [e[p["axis"], p["k"], p["j"], p["i"]] for p in probes]
        assert np.allclose(pr[n - 1], want, rtol=0, atol=1e-10 * np.abs(e).max())
    u = sl.expm(nsteps * og.dt * A) @ u0
    e = np.zeros(d.N); e[ie] = u[len(ih):] / se[ie]
    h = np.zeros(d.N); h[ih] = u[: len(ih)] / sh[ih]
    assert rel(ef, e) <= 1e-10 and rel(hf, h) <= 1e-10
    _, _, hs = expo.propagate(og, nsteps, e0, h0, probes, kind, q, m, dt_cfl=dtc, stagger_h=True)
    u = sl.expm((nsteps - 0.5) * og.dt * A) @ u0
    h = np.zeros(d.N); h[ih] = u[: len(ih)] / sh[ih]
    assert rel(hs, h) <= 1e-10


def test_backward_error_condition_holds_on_the_spectrum():
    """||Delta A|| <= eps_A ||A|| (Sec. III-D) on the true eigenvalues, and the
    planned degree is the smallest that meets the sampled condition."""
    og, dtc = tiny_grid(seed=7)
    A, _, _ = dense_A(og)
    z = np.linalg.eigvals(A) * dtc                          # normalised eigenvalues
    u = og.dt / dtc
    for tol in (1e-3, 1e-8):
        q, m = expo.plan("leja", u, tol)
        c = q * u
        xi = expo.nodes("leja", m)
        d = expo.divided_differences(xi, c)
        w, p = np.ones_like(z), np.zeros_like(z)
        for k in range(m + 1):
            p += d[k] * w
            w *= z - xi[k]
        dA = np.abs(np.log(p * np.exp(-c * z))) / (q * og.dt)
        assert dA.max() <= tol * 2.0 / dtc
        err = expo._errors(xi, d, c, expo.unit_roundoff(64))
        assert err[m] <= 2 * c * tol
        lower = [expo._errors(xi[: m - 1], expo.divided_differences(xi[: m - 1], (i / q) * c), (i / q) * c,
                              expo.unit_roundoff(64))[m - 2] > 2 * (i / q) * c * tol for i in range(1, q + 1)]
        assert any(lower)                                    # m - 2 fails somewhere


def test_leja_is_cheaper_than_taylor():
    """Sec. IV-A reports Leja ahead of the Taylor-based method by about 2x in
    operator applications; with the same condition the planned m/q agree."""
    for tol in (1e-12, 1e-8):
        ql, ml = expo.plan("leja", 0.95, tol)
        qt, mt = expo.plan("taylor", 0.95, tol)
        assert ml / ql * 1.5 < mt / qt


def paraexp_setup(u, T_steps_at_unit=120):
    dims = (6, 5, 7)
    eps = np.ones(dims[::-1], np.float32)
    eps[2:5, 1:4, 2:4] = 2.5
    sp = (1e-3, 1e-3, 1e-3)
    dtc = oracle.cfl_dt(dims, sp, eps)
    og = oracle.OracleGrid(dims, sp, eps, dt=u * dtc)
    src = [dict(axis=2, i=3, j=2, k=3, waveform=1, amp=1.0, width=40 * 0.5 * dtc, delay=40 * 0.5 * dtc)]
    prb = [dict(axis=2, i=1, j=1, k=3), dict(axis=0, i=2, j=3, k=5)]
    return og, dtc, src, prb


def test_paraexp_expo_converges_to_leapfrog_at_second_order():
    """ParaExp with exact homogeneous problems differs from one leapfrog run
    by the leapfrog's O(dt^2) truncation error (Sec. III-D): halving dt
    divides the difference by 4 (a first-order synchronisation of h would
    give 2)."""
    diffs = []
    for u, n in ((0.5, 120), (0.25, 240)):
        og, dtc, src, prb = paraexp_setup(u)
        K = 4
        win = [n * j // K for j in range(K + 1)]
        pr, ef, hf = expo.paraexp(og, K, win, src, prb, "leja", tol=1e-13, dt_cfl=dtc)
        pl, _, el, hl = og.leapfrog(n, src, prb)
        diffs.append(rel(ef, el))
        assert rel(pr, pl) < 0.05
    ratio = diffs[0] / diffs[1]
    assert 3.5 < ratio < 4.5, ratio


def test_paraexp_expo_single_window_is_leapfrog():
    og, dtc, src, prb = paraexp_setup(0.95)
    pr, ef, hf = expo.paraexp(og, 1, [0, 50], src, prb, "leja", tol=1e-10, dt_cfl=dtc)
    pl, _, el, hl = og.leapfrog(50, src, prb)
    assert np.array_equal(pr, pl) and np.array_equal(ef, el) and np.array_equal(hf, hl)


def test_norm_is_conserved():
    og, dtc = tiny_grid(seed=9)
    e0, h0 = random_state(og, 4)
    q, m = expo.plan("leja", og.dt / dtc, 1e-12)
    _, ef, hf = expo.propagate(og, 90, e0, h0, (), "leja", q, m, dt_cfl=dtc)
    n0 = np.sum(og.meps * e0 ** 2) + np.sum(og.mmu * h0 ** 2)
    n1 = np.sum(og.meps * ef ** 2) + np.sum(og.mmu * hf ** 2)
    assert abs(n1 / n0 - 1.0) <= 1e-10
