"""Pins of the oracle on graded (tensor-product) grids: cell (i, j, k) of size
dx[i] x dy[j] x dz[k] (Sec. II material matrices with local sizes, eq. (cfl)
with each cell's own sizes, and the row-sum bound of A used by the
exponential propagators).

Pins from outside the oracle: the uniform grid as the limit of constant
sizes, the closed-form energy of uniform fields (the dual cells tile the
cells they cover), the dense matrix A built from the incidence definitions
(tests/dense_fit.py) and its eigenvalues, scipy's expm."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from oracle import expo
from dense_fit import DenseFIT

C0, MU0, EPS0 = oracle.constants()


def rand_graded(dims, seed, ratio=4.0):
    rng = np.random.default_rng(seed)
    return [rng.uniform(1e-3 / ratio, 1e-3, n) for n in dims]


def rand_materials(dims, seed, lossy=False, mu=True):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    eps = rng.uniform(1.0, 5.0, (nz, ny, nx)).astype(np.float32)
    sig = rng.uniform(0.0, 2.0, (nz, ny, nx)).astype(np.float32) if lossy else None
    mur = rng.uniform(1.0, 3.0, (nz, ny, nx)).astype(np.float32) if mu else None
    return eps, mur, sig


def dense_A(og):
    d = DenseFIT((og.nx, og.ny, og.nz))
    ie, ih = np.flatnonzero(d.edge_dof), np.flatnonzero(d.face_dof)
    me, mm = og.meps.ravel()[ie], og.mmu.ravel()[ih]
    top = -np.diag(mm ** -0.5) @ d.C[np.ix_(ih, ie)] @ np.diag(me ** -0.5)
    A = np.block([[np.zeros((len(ih), len(ih))), top], [-top.T, np.zeros((len(ie), len(ie)))]])
    return A, ie, ih, d


def test_constant_sizes_reduce_to_the_uniform_grid():
    dims = (5, 4, 6)
    sp = (1e-3, 1.4e-3, 0.7e-3)
    eps, mur, sig = rand_materials(dims, 3, lossy=True)
    gu = oracle.OracleGrid(dims, sp, eps, mur, sig)
    sizes = [np.full(n, v) for n, v in zip(dims, sp)]
    gg = oracle.OracleGrid(dims, sizes, eps, mur, sig, dt=gu.dt)
    assert gg.graded is not None
    assert abs(oracle.cfl_dt(dims, sizes, eps, mur) / oracle.cfl_dt(dims, sp, eps, mur) - 1) <= 1e-15
    for name in ("ca", "cb", "ch", "meps", "msig", "mmu"):
        a, b = getattr(gg, name), getattr(gu, name)
        assert np.max(np.abs(a - b)) <= 4e-16 * np.max(np.abs(b)), name


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_graded_material_matrices_give_exact_uniform_field_energy(axis):
    """A uniform field E along `axis` (e = E d_a on every free edge) has the
    discrete energy (1/2) e' M_eps e = (1/2) eps0 E^2 sum over cells of
    eps_r V_cell (covered fraction): each free edge's dual cell holds a quarter
    of each of its four cells.  A uniform B normal to `axis` (b = B A_face on
    every interior face) has (1/2) b' M_mu^{-1} b = (1/2) B^2/mu0 sum over cells
    of V_cell/mu_r (covered fraction), half of each of the face's two cells.
    This fixes the dual areas, dual lengths and both averages on a graded
    grid."""
    dims = (5, 4, 6)
    sizes = rand_graded(dims, 11, ratio=5.0)
    eps, mur, _ = rand_materials(dims, 12)
    g = oracle.OracleGrid(dims, sizes, eps, mur, None)
    nx, ny, nz = dims
    V = sizes[2][:, None, None] * sizes[1][None, :, None] * sizes[0][None, None, :]
    b, c = (axis + 1) % 3, (axis + 2) % 3
    E0, B0 = 3.0, 2e-6
    Me = g.meps[axis]
    W_disc = 0.0
    cover = np.zeros((nz, ny, nx))
    for k, j, i in np.ndindex(nz + 1, ny + 1, nx + 1):
        if Me[k, j, i] == 0:
            continue
        q = (i, j, k)
        W_disc += 0.5 * Me[k, j, i] * (E0 * sizes[axis][q[axis]]) ** 2
        for sb in (0, 1):
            for sc in (0, 1):
                r = list(q); r[b] -= sb; r[c] -= sc
                cover[r[2], r[1], r[0]] += 0.25
    W_cont = 0.5 * EPS0 * E0 ** 2 * np.sum(eps * V * cover)
    assert abs(W_disc - W_cont) <= 1e-13 * W_cont
    Mm = g.mmu[axis]
    W_disc = 0.0
    cover = np.zeros((nz, ny, nx))
    for k, j, i in np.ndindex(nz + 1, ny + 1, nx + 1):
        if Mm[k, j, i] == 0:
            continue
        q = (i, j, k)
        A = sizes[b][q[b]] * sizes[c][q[c]]
        W_disc += 0.5 * (B0 * A) ** 2 / Mm[k, j, i]
        cover[k, j, i] += 0.5
        r = list(q); r[axis] -= 1
        cover[r[2], r[1], r[0]] += 0.5
    W_cont = 0.5 * B0 ** 2 / MU0 * np.sum(V * cover / mur)
    assert abs(W_disc - W_cont) <= 1e-13 * W_cont


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_row_sum_bound_and_cfl_estimate_on_graded_grids(seed):
    """The oracle's row sums are those of the dense A; their maximum bounds
    every eigenvalue; and eq. (cfl) with local sizes leaves the leapfrog
    stable (dt_CFL <= 2/||A||_2) on these grids."""
    dims = (4, 5, 3)
    sizes = rand_graded(dims, 20 + seed, ratio=6.0)
    if seed == 4:   # one thin slab
        sizes = [np.full(n, 1e-3) for n in dims]
        sizes[0][2] = 1e-4
    eps, mur, _ = rand_materials(dims, 30 + seed)
    g = oracle.OracleGrid(dims, sizes, eps, mur, None)
    A, ie, ih, d = dense_A(g)
    rs, oe, oh = g.A_rowsum()
    dense_rows = np.abs(A).sum(1)
    assert np.allclose(oh.ravel()[ih], dense_rows[: len(ih)], rtol=1e-14, atol=0)
    assert np.allclose(oe.ravel()[ie], dense_rows[len(ih):], rtol=1e-14, atol=0)
    assert abs(rs / dense_rows.max() - 1) <= 1e-14
    lam = np.abs(np.linalg.eigvals(A)).max()
    assert lam <= rs * (1 + 1e-12)
    dtc = oracle.cfl_dt(dims, sizes, eps, mur)
    assert lam * dtc / 2 < 1.0


def test_graded_leapfrog_conserves_energy():
    dims = (8, 7, 9)
    sizes = rand_graded(dims, 41, ratio=8.0)
    eps, mur, _ = rand_materials(dims, 42)
    g = oracle.OracleGrid(dims, sizes, eps, mur, None, cfl_fraction=0.99)
    t = 20 * g.dt
    src = [dict(axis=2, i=4, j=3, k=4, waveform=1, amp=1.0, width=t, delay=t)]
    _, en, _, _ = g.leapfrog(600, src, [], energy=True)
    tail = en[150:]
    assert tail.min() > 0 and np.ptp(tail) <= 1e-11 * tail.mean()


def test_graded_propagate_equals_dense_exponential():
    dims = (4, 4, 3)
    sizes = rand_graded(dims, 51, ratio=5.0)
    eps, mur, _ = rand_materials(dims, 52)
    g = oracle.OracleGrid(dims, sizes, eps, mur, None)
    beta = expo.spectral_bound(g)
    assert beta == g.A_rowsum()[0]
    A, ie, ih, d = dense_A(g)
    rng = np.random.default_rng(3)
    e0 = np.where(d.edge_dof, rng.standard_normal(d.N), 0.0).reshape(g.field_shape)
    h0 = np.where(d.face_dof, rng.standard_normal(d.N), 0.0).reshape(g.field_shape)
    n = 40
    _, ef, hf = expo.propagate(g, n, e0, h0, (), "leja", tol=1e-12)
    se, sh = np.sqrt(g.meps).ravel(), np.sqrt(g.mmu).ravel()
    u0 = np.concatenate([(sh * h0.ravel())[ih], (se * e0.ravel())[ie]])
    u = sl.expm(n * g.dt * A) @ u0
    e = np.zeros(d.N); e[ie] = u[len(ih):] / se[ie]
    h = np.zeros(d.N); h[ih] = u[: len(ih)] / sh[ih]
    assert np.linalg.norm(ef.ravel() - e) <= 1e-10 * np.linalg.norm(e)
    assert np.linalg.norm(hf.ravel() - h) <= 1e-10 * np.linalg.norm(h)


def graded_J(og, N, srcs, prbs, sizes):
    """J = sum_n sum_p (e_p^n / L_p)^2 from the forward oracle, L_p the probe
    edge's own length on the graded grid."""
    pr, _, _, _ = og.leapfrog(N, srcs, prbs)
    L = np.array([sizes[p["axis"]][(p["i"], p["j"], p["k"])[p["axis"]]] for p in prbs])
    return float(np.sum((pr / L) ** 2))


@pytest.mark.parametrize("scheme", [0, 1])
def test_graded_adjoint_matches_finite_differences(scheme):
    """The adjoint gradient on a lossy graded grid equals central finite
    differences of J through the forward oracle, cell by cell."""
    dims = (4, 3, 3)
    sizes = rand_graded(dims, 71, ratio=4.0)
    eps, _, sig = rand_materials(dims, 72, lossy=True, mu=False)
    dt = 0.9 * oracle.cfl_dt(dims, sizes, eps)
    srcs = [dict(axis=2, i=2, j=1, k=1, waveform=0, amp=1.0, f0=80e9, width=15 * dt, delay=15 * dt)]
    prbs = [dict(axis=2, i=1, j=2, k=1), dict(axis=0, i=2, j=1, k=2), dict(axis=1, i=3, j=0, k=2)]
    N = 50
    og = oracle.OracleGrid(dims, sizes, eps, None, sig, dt=dt, sigma_scheme=scheme)
    J, grad = og.adjoint(N, srcs, prbs)
    assert abs(graded_J(og, N, srcs, prbs, sizes) - J) <= 1e-13 * J
    fd = np.zeros_like(grad)
    for idx in np.ndindex(eps.shape):
        ep, em = eps.copy(), eps.copy()
        ep[idx] = np.float32(eps[idx] + np.float32(1e-2))
        em[idx] = np.float32(eps[idx] - np.float32(1e-2))
        Jp = graded_J(oracle.OracleGrid(dims, sizes, ep, None, sig, dt=dt, sigma_scheme=scheme), N, srcs, prbs, sizes)
        Jm = graded_J(oracle.OracleGrid(dims, sizes, em, None, sig, dt=dt, sigma_scheme=scheme), N, srcs, prbs, sizes)
        fd[idx] = (Jp - Jm) / (float(ep[idx]) - float(em[idx]))
    assert np.allclose(grad, fd, rtol=2e-4, atol=2e-4 * np.abs(fd).max())


def test_graded_adjoint_with_constant_sizes_equals_uniform():
    dims = (5, 4, 3)
    sp = (1e-3, 1.3e-3, 0.8e-3)
    eps, _, sig = rand_materials(dims, 81, lossy=True, mu=False)
    gu = oracle.OracleGrid(dims, sp, eps, None, sig)
    sizes = [np.full(n, v) for n, v in zip(dims, sp)]
    gg = oracle.OracleGrid(dims, sizes, eps, None, sig, dt=gu.dt)
    srcs = [dict(axis=1, i=2, j=1, k=1, waveform=0, amp=1.0, f0=60e9, width=12 * gu.dt, delay=12 * gu.dt)]
    prbs = [dict(axis=2, i=3, j=2, k=1), dict(axis=0, i=1, j=3, k=2)]
    Ju, gru = gu.adjoint(40, srcs, prbs)
    Jg, grg = gg.adjoint(40, srcs, prbs)
    assert abs(Jg - Ju) <= 1e-13 * Ju
    assert np.max(np.abs(grg - gru)) <= 1e-12 * np.max(np.abs(gru))


def complex_step_J(dims, sizes, eps, sig, dt, scheme, srcs, prbs, N, direction, h=1e-30, spacing=None):
    """J(eps + i h direction) of an N-step run from zero state, by a dense
    complex leapfrog over the incidence matrix of tests/dense_fit.py.  The
    edge coefficients are formed from complex eps with the graded material
    matrices; Im(J) / h is then the exact directional derivative
    (complex-step differentiation), independent of the adjoint sweep.
    `spacing` (default: sizes) is what the oracle grid gets: three scalars
    make it a uniform grid.  Returns (J real part, directional derivative,
    (real ca, real cb, oracle grid))."""
    d = DenseFIT(dims)
    nx, ny, nz = dims
    Np = d.Np
    epsc = eps.astype(np.float64) + 1j * h * direction
    sigv = np.zeros(eps.shape) if sig is None else sig.astype(np.float64)
    ca = np.zeros(3 * Np, complex)
    cb = np.zeros(3 * Np, complex)
    for r in np.flatnonzero(d.edge_dof):
        a, p = divmod(int(r), Np)
        q = (p % (nx + 1), (p // (nx + 1)) % (ny + 1), p // ((nx + 1) * (ny + 1)))
        b, c = (a + 1) % 3, (a + 2) % 3
        E = S = 0.0
        for sb in (0, 1):
            for sc in (0, 1):
                cell = list(q)
                cell[b] -= sb
                cell[c] -= sc
                w = sizes[b][cell[b]] * sizes[c][cell[c]] / 4.0
                E = E + epsc[cell[2], cell[1], cell[0]] * w
                S = S + sigv[cell[2], cell[1], cell[0]] * w
        L = sizes[a][q[a]]
        me, ms = EPS0 * E / L, S / L
        av = dt * ms / (2.0 * me)
        if scheme == 0:
            ca[r], cb[r] = (1.0 - av) / (1.0 + av), dt / (me * (1.0 + av))
        else:
            ca[r], cb[r] = 1.0 - 2.0 * av, dt / me
    og = oracle.OracleGrid(dims, sizes if spacing is None else spacing, eps, None, sig, dt=dt, sigma_scheme=scheme)
    ch = og.ch.ravel()
    e = np.zeros(3 * Np, complex)
    hh = np.zeros(3 * Np, complex)
    J = 0.0
    for n in range(N):
        hh = hh - ch * (d.C @ e)
        jv = np.zeros(3 * Np)
        for s in srcs:
            jv[s["axis"] * Np + d.pidx((s["i"], s["j"], s["k"]))] += oracle.waveform(
                s["waveform"], s["amp"], s["f0"], s["width"], s["delay"], (n + 0.5) * dt)
        e = ca * e + cb * (d.C.T @ hh - jv)
        for pr in prbs:
            q = (pr["i"], pr["j"], pr["k"])
            J = J + (e[pr["axis"] * Np + d.pidx(q)] / sizes[pr["axis"]][q[pr["axis"]]]) ** 2
    return float(J.real), float(J.imag) / h, (ca.real, cb.real, og)


@pytest.mark.parametrize("graded,scheme", [(True, 0), (True, 1), (False, 0)])
def test_adjoint_matches_complex_step_derivatives(graded, scheme):
    """The oracle's adjoint gradient against exact directional derivatives of
    J (complex step through a dense complex leapfrog): grad . v = dJ(eps; v)
    for random directions v and single cells, to 1e-10."""
    dims = (4, 3, 3)
    uniform = (1e-3, 1.2e-3, 0.8e-3)
    sizes = rand_graded(dims, 91, ratio=4.0) if graded else [np.full(n, v) for n, v in zip(dims, uniform)]
    spacing = sizes if graded else uniform
    eps, _, sig = rand_materials(dims, 92, lossy=True, mu=False)
    dt = 0.9 * oracle.cfl_dt(dims, spacing, eps)
    srcs = [dict(axis=2, i=2, j=1, k=1, waveform=0, amp=1.0, f0=80e9, width=15 * dt, delay=15 * dt)]
    prbs = [dict(axis=2, i=1, j=2, k=1), dict(axis=0, i=2, j=1, k=2), dict(axis=1, i=3, j=0, k=2)]
    N = 40
    rng = np.random.default_rng(93)
    dirs = [rng.standard_normal(eps.shape) for _ in range(3)]
    for idx in [(0, 0, 0), (1, 2, 3), (2, 1, 1)]:
        v = np.zeros(eps.shape)
        v[idx] = 1.0
        dirs.append(v)
    J0, _, (ca, cb, og) = complex_step_J(dims, sizes, eps, sig, dt, scheme, srcs, prbs, N, dirs[0], spacing=spacing)
    assert (og.graded is not None) == graded
    # the restated coefficients are the oracle's, so the comparison is about the sweep
    assert np.max(np.abs(ca - og.ca.ravel())) <= 1e-15 and np.max(np.abs(cb - og.cb.ravel())) <= 1e-15 * np.abs(cb).max()
    J, grad = og.adjoint(N, srcs, prbs)
    assert abs(J - J0) <= 1e-12 * J
    for v in dirs:
        _, dJ, _ = complex_step_J(dims, sizes, eps, sig, dt, scheme, srcs, prbs, N, v, spacing=spacing)
        assert abs(float(np.sum(grad * v)) - dJ) <= 1e-10 * np.abs(grad).sum() * np.abs(v).max(), (dJ, np.sum(grad * v))
