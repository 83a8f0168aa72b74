"""The adjoint formulation the CUDA path uses, checked on the CPU with dense
matrices (no GPU, no library code).

1. In the scaled multipliers mu = cb (.) lambda_e and nu = -ch (.) lambda_h,
   the transpose of the one-step leapfrog propagator P is P itself:
   P^T = S^-1 P S with S = diag(cb, -ch) on the degrees of freedom.  So the
   reverse sweep is the forward step, with -dJ/de^n as its impressed current.
2. With M_eps = eps0 eps_bar A / L entering Ampere's law only as
   M_eps (e^{n+1} - e^n) / dt, the gradient per edge is
   dJ/dM_eps = -(1/dt) sum_n mu^{n+1} (e^{n+1} - e^n), and each cell's share
   of M_eps gives dJ/d eps_r.  Run in numpy over tests/dense_fit.py's
   incidence matrix, this reproduces the oracle's gradient (derived
   differently: chain rule through ca, cb) on uniform and graded grids."""
import numpy as np
import pytest

import oracle
from dense_fit import DenseFIT

C0, MU0, EPS0 = oracle.constants()


def materials(dims, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    eps = rng.uniform(1.0, 5.0, (nz, ny, nx)).astype(np.float32)
    sig = rng.uniform(0.0, 2.0, (nz, ny, nx)).astype(np.float32)
    mur = rng.uniform(1.0, 3.0, (nz, ny, nx)).astype(np.float32)
    return eps, sig, mur


@pytest.mark.parametrize("scheme", [0, 1])
def test_adjoint_step_is_the_forward_step_in_scaled_variables(scheme):
    dims = (3, 4, 3)
    eps, sig, mur = materials(dims, 1)
    og = oracle.OracleGrid(dims, (1e-3, 1.3e-3, 0.8e-3), eps, mur, sig, sigma_scheme=scheme)
    d = DenseFIT(dims)
    P, ie, ih = d.propagator(og.ca.ravel(), og.cb.ravel(), og.ch.ravel())
    s = np.concatenate([og.cb.ravel()[ie], -og.ch.ravel()[ih]])
    assert np.all(s != 0)
    lhs = P.T
    rhs = (P * s[None, :]) / s[:, None]          # S^-1 P S
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(lhs))


def scaled_adjoint_gradient(og, d, sizes, N, srcs, prbs):
    """J and dJ/d eps_r by the scaled sweep and the M_eps gradient formula."""
    Np = d.Np
    ca, cb, ch = og.ca.ravel(), og.cb.ravel(), og.ch.ravel()
    C = d.C
    nx, ny, nz = d.n
    plen = [sizes[p["axis"]][(p["i"], p["j"], p["k"])[p["axis"]]] for p in prbs]
    pidx = [p["axis"] * Np + d.pidx((p["i"], p["j"], p["k"])) for p in prbs]

    def jvec(n):
        v = np.zeros(3 * Np)
        for s_ in srcs:
            v[s_["axis"] * Np + d.pidx((s_["i"], s_["j"], s_["k"]))] += oracle.waveform(
                s_["waveform"], s_["amp"], s_["f0"], s_["width"], s_["delay"], (n + 0.5) * og.dt)
        return v

    E = [np.zeros(3 * Np)]
    h = np.zeros(3 * Np)
    for n in range(N):
        h = h - ch * (C @ E[-1])
        E.append(ca * E[-1] + cb * (C.T @ h - jvec(n)))
    J = sum((E[n][q] / L) ** 2 for n in range(1, N + 1) for q, L in zip(pidx, plen))

    def dJde(n):
        v = np.zeros(3 * Np)
        for q, L in zip(pidx, plen):
            v[q] += 2.0 * E[n][q] / L ** 2
        return v

    mu = cb * dJde(N)                     # mu^N
    nu = np.zeros(3 * Np)                 # nu^{N+1/2}
    g = np.zeros(3 * Np)                  # dJ/dM_eps per edge
    for n in range(N - 1, -1, -1):
        g += -(1.0 / og.dt) * mu * (E[n + 1] - E[n])
        nu = nu - ch * (C @ mu)                                   # nu^{n+1/2}
        mu = ca * mu + cb * (C.T @ nu + (dJde(n) if n >= 1 else 0.0))   # mu^n
    # dM_eps(edge along a) / d eps_r(cell) = eps0 d_b d_c / (4 d_a) with the cell's sizes
    grad = np.zeros((nz, ny, nx))
    for r in np.flatnonzero(d.edge_dof):
        a, p = divmod(int(r), Np)
        q = (p % (nx + 1), (p // (nx + 1)) % (ny + 1), p // ((nx + 1) * (ny + 1)))
        b, c = (a + 1) % 3, (a + 2) % 3
        for sb in (0, 1):
            for sc in (0, 1):
                cell = list(q)
                cell[b] -= sb
                cell[c] -= sc
                w = EPS0 * sizes[b][cell[b]] * sizes[c][cell[c]] / (4.0 * sizes[a][q[a]])
                grad[cell[2], cell[1], cell[0]] += w * g[r]
    return J, grad


@pytest.mark.parametrize("graded,scheme", [(False, 0), (False, 1), (True, 0), (True, 1)])
def test_scaled_sweep_gradient_equals_oracle(graded, scheme):
    dims = (4, 3, 3)
    eps, sig, _ = materials(dims, 2)
    uniform = (1e-3, 1.2e-3, 0.9e-3)
    rng = np.random.default_rng(3)
    sizes = ([rng.uniform(0.3e-3, 1e-3, n) for n in dims] if graded
             else [np.full(n, v) for n, v in zip(dims, uniform)])
    spacing = sizes if graded else uniform
    dt = 0.9 * oracle.cfl_dt(dims, spacing, eps)
    og = oracle.OracleGrid(dims, spacing, eps, None, sig, dt=dt, sigma_scheme=scheme)
    srcs = [dict(axis=2, i=2, j=1, k=1, waveform=0, amp=1.0, f0=80e9, width=15 * dt, delay=15 * dt)]
    prbs = [dict(axis=2, i=1, j=2, k=1), dict(axis=0, i=2, j=1, k=2), dict(axis=1, i=3, j=0, k=2)]
    N = 40
    J_ref, g_ref = og.adjoint(N, srcs, prbs)
    J, grad = scaled_adjoint_gradient(og, DenseFIT(dims), sizes, N, srcs, prbs)
    assert abs(J - J_ref) <= 1e-12 * J_ref
    assert np.max(np.abs(grad - g_ref)) <= 1e-9 * np.max(np.abs(g_ref))
