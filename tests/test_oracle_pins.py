"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test is chosen so that a plausible mistake in the oracle (a dropped
term, a wrong sign or index, a transposed component, wrong averaging cells)
fails at least one of them:

* dense brute force: the oracle's step equals the dense one-step matrix built
  from the combinatorial incidence definition of C (Sec. II);
* exactness of the complex: C G = 0, S C = 0 (Sec. II, eq. maxwell_grid2);
* Yee dispersion: the eigenvalues of the vacuum propagator are exp(+-i w dt)
  with sin^2(w dt/2)/(c dt)^2 = sum_a sin^2(k_a d_a/2)/d_a^2 (closed form);
* the oracle's vacuum coefficients equal the closed-form material matrices;
* energy balance of the leapfrog (Sec. II-A, eq. energy) as an exact identity,
  lossless and lossy, both sigma schemes;
* Gauss law: div b and charge-free div d keep their initial values, and the
  source deposits charge only at the ends of its edge (Sec. II);
* mirror, transpose and cyclic-rotation symmetry of the solution;
* ParaExp superposition equals one sequential run (Sec. III, linearity);
* adjoint gradient equals central finite differences;
* PEC cavity resonances f = c/2 sqrt((m/a)^2+(n/b)^2+(p/d)^2) within the FIT
  dispersion error, and exactly at the discrete dispersion frequencies;
* n_dof printed for the 2-D wave of Sec. IV-A (tests/golden).
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from dense_fit import DenseFIT
from paper_1705_08019_gb300 import workloads as W

C0, MU0, EPS0 = oracle.constants()
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_materials(dims, seed, lossy=True, mu=True):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    eps = rng.uniform(1.0, 5.0, (nz, ny, nx)).astype(np.float32)
    sig = rng.uniform(0.0, 2.0, (nz, ny, nx)).astype(np.float32) if lossy else None
    mur = rng.uniform(1.0, 3.0, (nz, ny, nx)).astype(np.float32) if mu else None
    return eps, mur, sig


def rand_state(g, dense, seed):
    rng = np.random.default_rng(seed)
    e = np.zeros(dense.N)
    h = np.zeros(dense.N)
    e[dense.edge_dof] = rng.standard_normal(dense.edge_dof.sum())
    h[dense.face_dof] = rng.standard_normal(dense.face_dof.sum()) * 1e-2
    return e.reshape(g.field_shape), h.reshape(g.field_shape)


def test_constants():
    assert C0 == 299792458.0
    assert abs(MU0 - 4e-7 * math.pi) < 1e-22
    assert abs(EPS0 * MU0 * C0 * C0 - 1.0) < 1e-15


def test_ndof_golden():
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLDEN, "ndof_wave2d.txt"))
            if l.strip() and not l.startswith("#")]
    assert rows
    for px, py, pz, ndof in rows:
        g = oracle.OracleGrid((px - 1, py - 1, pz - 1), (0.5, 0.5, 1.0), np.ones((pz - 1, py - 1, px - 1)))
        assert 2 * g.zeros().size == ndof


@pytest.mark.parametrize("dims", [(3, 4, 5), (4, 4, 4), (2, 3, 2)])
def test_complex_exact(dims):
    d = DenseFIT(dims)
    assert np.count_nonzero(d.C @ d.G) == 0
    assert np.count_nonzero(d.S @ d.C) == 0
    # every face has 4 boundary edges, every cell 6 faces
    assert np.all(np.abs(d.C[d.face_exists]).sum(1) == 4)
    assert np.all(np.abs(d.S[d.cell_exists]).sum(1) == 6)


@pytest.mark.parametrize("dims,seed,scheme", [((3, 4, 5), 1, 0), ((4, 3, 3), 2, 1), ((2, 2, 3), 3, 0)])
def test_step_equals_dense_propagator(dims, seed, scheme):
    eps, mur, sig = rand_materials(dims, seed)
    g = oracle.OracleGrid(dims, (1e-3, 1.3e-3, 0.8e-3), eps, mur, sig, sigma_scheme=scheme)
    d = DenseFIT(dims)
    # the oracle's predicates agree with the geometric degrees of freedom
    assert np.array_equal(g.cb.ravel() != 0, d.edge_dof)
    assert np.array_equal(g.ch.ravel() != 0, d.face_dof)
    P, ie, ih = d.propagator(g.ca.ravel(), g.cb.ravel(), g.ch.ravel())
    e0, h0 = rand_state(g, d, seed + 10)
    nsteps = 7
    _, _, e, h = g.leapfrog(nsteps, e=e0, h=h0)
    x = np.concatenate([e0.ravel()[ie], h0.ravel()[ih]])
    for _ in range(nsteps):
        x = P @ x
    ref_e, ref_h = x[:len(ie)], x[len(ie):]
    assert np.allclose(e.ravel()[ie], ref_e, rtol=0, atol=1e-12 * np.abs(ref_e).max())
    assert np.allclose(h.ravel()[ih], ref_h, rtol=0, atol=1e-12 * np.abs(ref_h).max())
    # non-dofs stay exactly zero
    assert np.all(e.ravel()[~d.edge_dof] == 0) and np.all(h.ravel()[~d.face_dof] == 0)


def test_source_enters_with_minus_cb():
    dims = (3, 4, 3)
    eps, mur, sig = rand_materials(dims, 5)
    g = oracle.OracleGrid(dims, (1e-3, 1e-3, 1e-3), eps, mur, sig)
    d = DenseFIT(dims)
    P, ie, ih = d.propagator(g.ca.ravel(), g.cb.ravel(), g.ch.ravel())
    src = dict(axis=1, i=1, j=2, k=1, waveform=1, amp=2.0, f0=0.0, width=20 * g.dt, delay=10 * g.dt)
    nsteps, step0 = 9, 3
    _, _, e, h = g.leapfrog(nsteps, [src], step0=step0)
    x = np.zeros(len(ie) + len(ih))
    col = list(ie).index(1 * d.Np + d.pidx((1, 2, 1)))
    for n in range(nsteps):
        t = (step0 + n + 0.5) * g.dt
        amp = 2.0 * math.exp(-4.0 * ((t - 10 * g.dt) / (20 * g.dt)) ** 2)
        x = P @ x
        x[col] -= g.cb.ravel()[ie[col]] * amp
    assert np.allclose(e.ravel()[ie], x[:len(ie)], atol=1e-12 * np.abs(x).max())
    assert np.allclose(h.ravel()[ih], x[len(ie):], atol=1e-12 * np.abs(x).max())


def yee_angles(dims, spacing, dt, c=C0):
    """Closed-form Yee dispersion: the set of w*dt of a PEC box, each with its
    multiplicity (2 when no index is zero, 1 when one is)."""
    out = []
    ranges = [range(n) for n in dims]
    for m in itertools.product(*ranges):
        zeros = sum(1 for v in m if v == 0)
        if zeros > 1:
            continue
        s = sum(math.sin(m[a] * math.pi / (2 * dims[a])) ** 2 / spacing[a] ** 2 for a in range(3))
        theta = 2.0 * math.asin(c * dt * math.sqrt(s))
        out += [theta] * (2 if zeros == 0 else 1)
    return np.sort(np.array(out))


@pytest.mark.parametrize("dims,spacing", [((4, 4, 4), (1e-3, 1e-3, 1e-3)), ((3, 4, 5), (1e-3, 0.7e-3, 1.4e-3))])
def test_vacuum_dispersion_eigenvalues(dims, spacing):
    d = DenseFIT(dims)
    dx, dy, dz = spacing
    dt = 0.9 / (C0 * math.sqrt(1 / dx ** 2 + 1 / dy ** 2 + 1 / dz ** 2))
    # closed-form vacuum material matrices: M_eps,a = eps0 A_a / L_a, M_mu,a = mu0 A_a / L_a
    geo = [dy * dz / dx, dz * dx / dy, dx * dy / dz]
    Np = d.Np
    ca = np.zeros(d.N); cb = np.zeros(d.N); ch = np.zeros(d.N)
    for a in range(3):
        sl = slice(a * Np, (a + 1) * Np)
        ca[sl] = 1.0
        cb[sl] = dt / (EPS0 * geo[a])
        ch[sl] = dt / (MU0 * geo[a])
    ca *= d.edge_dof; cb *= d.edge_dof; ch *= d.face_dof
    # the oracle's own coefficients for vacuum are these closed forms
    nx, ny, nz = dims
    g = oracle.OracleGrid(dims, spacing, np.ones((nz, ny, nx)), dt=dt)
    assert np.allclose(g.ca.ravel(), ca, rtol=1e-15, atol=0)
    assert np.allclose(g.cb.ravel(), cb, rtol=1e-14, atol=0)
    assert np.allclose(g.ch.ravel(), ch, rtol=1e-14, atol=0)
    P, ie, ih = d.propagator(ca, cb, ch)
    lam = np.linalg.eigvals(P)
    assert np.allclose(np.abs(lam), 1.0, atol=1e-9)
    osc = lam[np.abs(lam.imag) > 1e-6]
    got = np.sort(np.abs(np.angle(osc)))
    want = np.sort(np.concatenate([yee_angles(dims, spacing, dt)] * 2))
    assert got.shape == want.shape
    assert np.allclose(got, want, atol=1e-9)


def run_steps(g, nsteps, sources, e=None, h=None):
    """Run one step at a time; returns e^n (n=0..N), h^{n-1/2} (n=0..N), W^n."""
    es, hs, ws = [], [], []
    e = g.zeros() if e is None else e
    h = g.zeros() if h is None else h
    es.append(e.copy()); hs.append(h.copy())
    for n in range(nsteps):
        _, en, e, h = g.leapfrog(1, sources, step0=n, e=e, h=h, energy=True)
        es.append(e.copy()); hs.append(h.copy()); ws.append(en[0])
    return es, hs, np.array(ws)


def source_vector(g, sources, t):
    j = g.zeros()
    for s in sources:
        x = (t - s["delay"]) / s["width"]
        if s["waveform"] == 0:
            v = s["amp"] * math.sin(2 * math.pi * s["f0"] * (t - s["delay"])) * math.exp(-4 * x * x)
        else:
            v = s["amp"] * math.exp(-4 * x * x)
        j[s["axis"], s["k"], s["j"], s["i"]] += v
    return j


@pytest.mark.parametrize("scheme,lossy", [(0, False), (0, True), (1, True)])
def test_energy_balance_identity(scheme, lossy):
    dims = (5, 4, 6)
    eps, mur, sig = rand_materials(dims, 11, lossy=lossy)
    g = oracle.OracleGrid(dims, (1e-3, 1.1e-3, 0.9e-3), eps, mur, sig, sigma_scheme=scheme)
    srcs = [dict(axis=2, i=2, j=2, k=3, waveform=0, amp=1.0, f0=60e9, width=30 * g.dt, delay=30 * g.dt)]
    N = 90
    es, hs, ws = run_steps(g, N, srcs)
    # W^n recomputed from the states with the material matrices
    for n in range(N):
        w = np.sum(g.meps * es[n] ** 2) + np.sum(g.mmu * hs[n] * hs[n + 1])
        assert abs(w - ws[n]) <= 1e-12 * max(abs(w), 1e-300) + 1e-300
    scale = np.abs(ws).max()
    for n in range(N - 1):
        s = es[n] + es[n + 1]
        j = source_vector(g, srcs, (n + 0.5) * g.dt)
        if scheme == 0:
            loss = -(g.dt / 2) * np.sum(g.msig * s * s)
        else:
            loss = -g.dt * np.sum(g.msig * es[n] * s)
        rhs = loss - g.dt * np.sum(j * s)
        assert abs((ws[n + 1] - ws[n]) - rhs) <= 1e-11 * scale


def test_energy_conserved_lossless_after_source():
    w = W.cavity16(nsteps=4500)
    g = oracle.OracleGrid(w.dims, w.spacing, w.eps_r)
    _, en, _, _ = g.leapfrog(w.nsteps, w.sources, w.probes, energy=True)
    # the source envelope is below 1e-12 after t = delay + 2.6 width
    tail = en[int((w.sources[0]["delay"] + 2.7 * w.sources[0]["width"]) / g.dt):]
    assert len(tail) > 100
    assert np.ptp(tail) <= 1e-12 * tail.mean()


def test_gauss_law():
    dims = (5, 6, 4)
    eps, mur, _ = rand_materials(dims, 21, lossy=False)
    g = oracle.OracleGrid(dims, (1e-3, 0.9e-3, 1.2e-3), eps, mur, None)
    d = DenseFIT(dims)
    e0, h0 = rand_state(g, d, 22)
    srcs = [dict(axis=0, i=2, j=3, k=2, waveform=0, amp=3.0, f0=40e9, width=20 * g.dt, delay=20 * g.dt)]
    N = 60
    _, _, e, h = g.leapfrog(N, srcs, e=e0, h=h0)
    Me, Mm = g.meps.ravel(), g.mmu.ravel()
    # magnetic: S b stays at its initial value on every cell
    db0 = d.S @ (Mm * h0.ravel())
    db = d.S @ (Mm * h.ravel())
    assert np.allclose(db[d.cell_exists], db0[d.cell_exists], atol=1e-12 * np.abs(db0).max())
    # electric: div d = -G^T d on interior points changes only by the source charge
    q0 = -(d.G.T @ (Me * e0.ravel()))
    q = -(d.G.T @ (Me * e.ravel()))
    jsum = np.zeros(d.N)
    for n in range(N):
        jsum += source_vector(g, srcs, (n + 0.5) * g.dt).ravel()
    dq_src = g.dt * (d.G.T @ jsum)
    inner = d.node_interior
    scale = np.abs(q0[inner]).max()
    assert np.allclose(q[inner], q0[inner] + dq_src[inner], atol=1e-10 * scale)
    # and the source charge sits only at the two end points of its edge
    nz_pts = np.flatnonzero(np.abs(dq_src) > 0)
    assert len(nz_pts) == 2


def _sym_material(dims, seed, op):
    eps, mur, sig = rand_materials(dims, seed)
    return (0.5 * (eps + op(eps))).astype(np.float32), (0.5 * (mur + op(mur))).astype(np.float32), \
        (0.5 * (sig + op(sig))).astype(np.float32)


def test_mirror_x_symmetry():
    dims = (6, 5, 4)
    flip = lambda a: a[:, :, ::-1]
    eps, mur, sig = _sym_material(dims, 31, flip)
    g = oracle.OracleGrid(dims, (1e-3, 1e-3, 1.1e-3), eps, mur, sig)
    srcs = [dict(axis=2, i=3, j=2, k=1, waveform=0, amp=1.0, f0=50e9, width=25 * g.dt, delay=25 * g.dt)]
    _, _, e, h = g.leapfrog(70, srcs)
    # x -> nx - x: points i <-> nx-i, edge/face midpoints i <-> nx-1-i
    nx = dims[0]
    pt = lambda a: a[:, :, ::-1]                     # i <-> nx - i  (on nx+1 points)
    mid = lambda a: np.concatenate([a[:, :, nx - 1::-1], a[:, :, nx:]], axis=2)  # i <-> nx-1-i
    s = np.abs(e).max()
    assert np.allclose(e[0], -mid(e[0]), atol=1e-12 * s)
    assert np.allclose(e[1], pt(e[1]), atol=1e-12 * s)
    assert np.allclose(e[2], pt(e[2]), atol=1e-12 * s)
    s = np.abs(h).max()
    assert np.allclose(h[0], pt(h[0]), atol=1e-12 * s)
    assert np.allclose(h[1], -mid(h[1]), atol=1e-12 * s)
    assert np.allclose(h[2], -mid(h[2]), atol=1e-12 * s)


def test_transpose_xy_symmetry():
    dims = (5, 5, 4)
    tr = lambda a: np.swapaxes(a, 1, 2)
    eps, mur, sig = _sym_material(dims, 41, tr)
    g = oracle.OracleGrid(dims, (1e-3, 1e-3, 0.8e-3), eps, mur, sig)
    srcs = [dict(axis=2, i=2, j=2, k=1, waveform=0, amp=1.0, f0=50e9, width=25 * g.dt, delay=25 * g.dt)]
    _, _, e, h = g.leapfrog(70, srcs)
    # (x, y) -> (y, x): E polar -> (Ey, Ex, Ez); H axial under an improper map -> -(Hy, Hx, Hz)
    s = np.abs(e).max()
    assert np.allclose(e[0], tr(e[1]), atol=1e-12 * s)
    assert np.allclose(e[2], tr(e[2]), atol=1e-12 * s)
    s = np.abs(h).max()
    assert np.allclose(h[0], -tr(h[1]), atol=1e-12 * s)
    assert np.allclose(h[2], -tr(h[2]), atol=1e-12 * s)


def test_cyclic_rotation():
    """Relabel axes (x, y, z) -> (y', z', x'): the solution maps component-wise."""
    dims = (4, 5, 6)
    spacing = (1.0e-3, 1.2e-3, 0.9e-3)
    eps, mur, sig = rand_materials(dims, 51)
    g = oracle.OracleGrid(dims, spacing, eps, mur, sig)
    src = dict(axis=2, i=2, j=2, k=3, waveform=0, amp=1.0, f0=50e9, width=25 * g.dt, delay=25 * g.dt)
    prb = dict(axis=0, i=1, j=3, k=2)
    pr, _, e, h = g.leapfrog(60, [src], [prb])
    # new axes: x' = z, y' = x, z' = y ; arrays are indexed [z, y, x] -> [z', y', x'] = [y, x, z]
    perm = lambda a: np.transpose(a, (1, 2, 0))
    dims2 = (dims[2], dims[0], dims[1])
    spacing2 = (spacing[2], spacing[0], spacing[1])
    g2 = oracle.OracleGrid(dims2, spacing2, perm(eps), perm(mur), perm(sig), dt=g.dt)
    src2 = dict(src, axis=0, i=src["k"], j=src["i"], k=src["j"])
    prb2 = dict(axis=1, i=prb["k"], j=prb["i"], k=prb["j"])
    pr2, _, e2, h2 = g2.leapfrog(60, [src2], [prb2])
    s = np.abs(e).max()
    # component a in old frame is component (a+1)%3 in the new frame
    for a in range(3):
        assert np.allclose(e2[(a + 1) % 3], perm(e[a]), atol=1e-12 * s)
        assert np.allclose(h2[(a + 1) % 3], perm(h[a]), atol=1e-12 * np.abs(h).max())
    assert np.allclose(pr, pr2, atol=1e-12 * s)


@pytest.mark.parametrize("K,u0", [(4, False), (3, True)])
def test_paraexp_equals_sequential(K, u0):
    w = W.small_random(dims=(7, 6, 5), nsteps=120, K=K)
    g = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma)
    win = np.array([0, 25, 31, 80, 120][:K + 1]) if K == 4 else np.array([5, 40, 90, 125])
    e0 = h0 = None
    if u0:
        d = DenseFIT(w.dims)
        e0, h0 = rand_state(g, d, 3)
    seq_pr, _, seq_e, seq_h = g.leapfrog(int(win[-1] - win[0]), w.sources, w.probes, step0=int(win[0]),
                                         e=e0, h=h0)
    pr, ef, hf = g.paraexp(K, win, w.sources, w.probes, e0=e0, h0=h0)
    assert np.allclose(pr, seq_pr, rtol=0, atol=1e-13 * np.abs(seq_pr).max())
    assert np.allclose(ef, seq_e, rtol=0, atol=1e-13 * np.abs(seq_e).max())
    assert np.allclose(hf, seq_h, rtol=0, atol=1e-13 * np.abs(seq_h).max())


def test_paraexp_members_are_zero_ic_windows():
    """Before its window a member contributes nothing: the sum over the first
    window equals member 1 alone, i.e. a run with the source gated to it."""
    w = W.small_random(dims=(6, 5, 5), nsteps=60, K=3)
    g = oracle.OracleGrid(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma)
    win = w.windows()
    pr, _, _ = g.paraexp(3, win, w.sources, w.probes)
    pr1, _, _, _ = g.leapfrog(int(win[1]), w.sources, w.probes, src_window=(win[0], win[1]))
    assert np.array_equal(pr[:win[1]], pr1)


@pytest.mark.parametrize("scheme", [0, 1])
def test_adjoint_matches_finite_differences(scheme):
    dims = (4, 3, 3)
    eps, _, sig = rand_materials(dims, 61, mu=False)
    spacing = (1e-3, 1.1e-3, 0.9e-3)
    dt = 0.9 * oracle.cfl_dt(dims, spacing, eps)
    srcs = [dict(axis=2, i=2, j=1, k=1, waveform=0, amp=1.0, f0=80e9, width=15 * dt, delay=15 * dt)]
    prbs = [dict(axis=2, i=1, j=2, k=1), dict(axis=0, i=2, j=1, k=2)]
    N = 50
    g = oracle.OracleGrid(dims, spacing, eps, None, sig, dt=dt, sigma_scheme=scheme)
    J, grad = g.adjoint(N, srcs, prbs)

    def J_of(eps_mod):
        gg = oracle.OracleGrid(dims, spacing, eps_mod, None, sig, dt=dt, sigma_scheme=scheme)
        pr, _, _, _ = gg.leapfrog(N, srcs, prbs)
        return float(np.sum((pr / np.array([spacing[p["axis"]] for p in prbs])) ** 2))

    assert abs(J_of(eps) - J) <= 1e-13 * J
    fd = np.zeros_like(grad)
    for idx in np.ndindex(eps.shape):
        ep, em = eps.copy(), eps.copy()
        ep[idx] = np.float32(eps[idx] + np.float32(1e-2))
        em[idx] = np.float32(eps[idx] - np.float32(1e-2))
        fd[idx] = (J_of(ep) - J_of(em)) / (float(ep[idx]) - float(em[idx]))
    assert np.allclose(grad, fd, rtol=2e-4, atol=2e-4 * np.abs(fd).max())


def test_cavity_resonances():
    """Broadband pulse in a PEC vacuum cavity: spectral peaks of a probe sit at
    the discrete Yee frequencies, and within the O((k d)^2) dispersion error
    of the continuum f = c/2 sqrt((m/a)^2 + (n/b)^2 + (p/d)^2)."""
    dims = (8, 6, 5)
    d = 1e-3
    a, b, c = (n * d for n in dims)
    nx, ny, nz = dims
    g = oracle.OracleGrid(dims, (d, d, d), np.ones((nz, ny, nx)))
    # zero-mean broadband excitation (an odd sine under a short envelope)
    f_ref = 0.5 * C0 * math.sqrt((1 / a) ** 2 + (1 / b) ** 2)
    src = dict(axis=2, i=3, j=2, k=2, waveform=0, amp=1.0, f0=f_ref, width=1.0 / f_ref, delay=1.0 / f_ref)
    prb = dict(axis=2, i=2, j=2, k=2)
    N = 16384
    pr, _, _, _ = g.leapfrog(N, [src], [prb])
    x = pr[:, 0] * np.hanning(N)
    spec = np.abs(np.fft.rfft(x))
    freqs = np.fft.rfftfreq(N, g.dt)
    # the lowest discrete modes with an E_z component (TM_mn0 and p > 0 modes)
    lowest = []
    for m in range(nx):
        for n in range(ny):
            for p in range(nz):
                if sum(v == 0 for v in (m, n, p)) > 1:
                    continue
                s = (math.sin(m * math.pi / (2 * nx)) ** 2 + math.sin(n * math.pi / (2 * ny)) ** 2
                     + math.sin(p * math.pi / (2 * nz)) ** 2) / d ** 2
                f_disc = math.asin(C0 * g.dt * math.sqrt(s)) / (math.pi * g.dt)
                f_cont = 0.5 * C0 * math.sqrt((m / a) ** 2 + (n / b) ** 2 + (p / c) ** 2)
                lowest.append((f_disc, f_cont, (m, n, p)))
    lowest.sort()
    f110_disc, f110_cont, mode = lowest[0]
    assert mode == (1, 1, 0)
    # strongest peak below 1.2 x f110 is the (1,1,0) mode
    band = (freqs > 0.5 * f110_cont) & (freqs < 1.2 * f110_cont)
    k = np.argmax(spec * band)
    # parabolic refinement of the peak
    y0, y1, y2 = np.log(spec[k - 1:k + 2])
    delta = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    f_peak = (k + delta) * (freqs[1] - freqs[0])
    binw = freqs[1] - freqs[0]
    assert abs(f_peak - f110_disc) < 0.1 * binw
    # discrete vs continuum: the FIT dispersion lowers the frequency by O((k d)^2)
    kd2 = (math.pi * d / a) ** 2 + (math.pi * d / b) ** 2
    assert f110_disc < f110_cont
    assert (f110_cont - f110_disc) / f110_cont < kd2 / 24 * 1.5
    # every strong spectral peak is a discrete mode
    peaks = [i for i in range(2, len(spec) - 2) if spec[i] == spec[i - 2:i + 3].max()
             and spec[i] > 0.05 * spec.max() and freqs[i] > 0.5 * f110_cont]
    modes = np.array([m[0] for m in lowest])
    for i in peaks:
        assert np.min(np.abs(modes - freqs[i])) < 1.5 * binw


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_material_matrices_give_exact_uniform_field_energy(axis):
    """A uniform field in a random cell-wise medium has the closed-form energy
    (1/2) int eps E^2 dV and (1/2) int B^2/mu dV.  The discrete energies
    (1/2) e' M_eps e with e = E L on every free edge along `axis`, and
    (1/2) b' M_mu^{-1} b with b = B A on every interior face normal to `axis`,
    must equal it over the region the dual cells / dual edges cover.  This
    holds for the area-weighted arithmetic mean of eps (E tangential to every
    cell interface around an edge) and the harmonic mean of mu (B normal to
    the interface the dual edge crosses), and fails for other averages."""
    dims = (5, 4, 6)
    spacing = (1e-3, 1.4e-3, 0.7e-3)
    eps, mur, _ = rand_materials(dims, 71, lossy=False)
    g = oracle.OracleGrid(dims, spacing, eps, mur, None)
    nx, ny, nz = dims
    V = spacing[0] * spacing[1] * spacing[2]
    L = spacing[axis]
    A = V / L
    E0, B0 = 3.0, 2e-6
    # electric: each free edge's dual cell takes a quarter of each of its 4 cells
    Me = g.meps[axis]
    W_disc = 0.5 * np.sum(Me * (E0 * L) ** 2)
    cover = np.zeros((nz, ny, nx))
    for k, j, i in np.ndindex(nz + 1, ny + 1, nx + 1):
        q = (i, j, k)
        if Me[k, j, i] == 0:
            continue
        b, c = (axis + 1) % 3, (axis + 2) % 3
        for sb in (0, 1):
            for sc in (0, 1):
                r = list(q); r[b] -= sb; r[c] -= sc
                cover[r[2], r[1], r[0]] += 0.25
    W_cont = 0.5 * EPS0 * E0 ** 2 * V * np.sum(eps * cover)
    assert abs(W_disc - W_cont) <= 1e-13 * W_cont
    # magnetic: each interior face's dual edge takes half of each of its 2 cells
    Mm = g.mmu[axis]
    W_disc = 0.5 * np.sum(np.where(Mm > 0, (B0 * A) ** 2 / np.where(Mm > 0, Mm, 1.0), 0.0))
    cover = np.zeros((nz, ny, nx))
    for k, j, i in np.ndindex(nz + 1, ny + 1, nx + 1):
        if Mm[k, j, i] == 0:
            continue
        r = [i, j, k]
        cover[k, j, i] += 0.5
        r[axis] -= 1
        cover[r[2], r[1], r[0]] += 0.5
    W_cont = 0.5 * B0 ** 2 / MU0 * V * np.sum(cover / mur)
    assert abs(W_disc - W_cont) <= 1e-13 * W_cont
