"""Exponential propagators for the homogeneous ParaExp problems: Leja
interpolation and its Taylor special case (Sec. III-B, "Approximation of the
matrix exponential"), and ParaExp with leapfrog window problems and
exponential homogeneous problems (Sec. III, Algorithm 1, eqs. averaging1/2).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may import this module.  It shares no code with the
CUDA library: divided differences are taken at high precision with mpmath
(the recursive definition), the polynomial is evaluated in complex Newton form
on the paper's transformed unknowns u = [M_mu^{1/2} h, M_eps^{1/2} e] with the
skew matrix A of eq. (FIT_ode_2), applied by ``fit_oracle.c``.

Readings of the paper (it defers the details to its references):

* Interval.  A is skew, so its eigenvalues lie on i[-beta, beta] with
  beta >= ||A||_2.  On a uniform grid beta = 2/dt_CFL, dt_CFL of eq. (cfl)
  (the Yee bound the estimate comes from); on a graded grid, where eq. (cfl)
  is only an estimate, beta = ||A||_1, the largest absolute row sum (the norm
  Higham's parameter selection works with).  X = (2/beta) A has its spectrum
  in i[-2, 2]; a substep of length h_s is exp(c X) with c = h_s beta/2.  The
  functions take dt_cfl = 2/beta.
* Points.  Conjugate Leja points of i[-2, 2]: xi_0 = 0, then for each pair
  the point i*eta, eta in [0, 2], that maximises the product of distances to
  all points chosen so far, followed by its conjugate.  eta runs over the
  grid 2 l / 2^15, l = 0..2^15, the first maximiser wins.  Taylor: every
  point is 0 (the interpolant is the truncated Taylor series).
* Parameters (m, s) of L_{m,c}(tA/s)^s.  Substeps are whole multiples of the
  leapfrog step, h_s = q dt, so every output time of the leapfrog grid falls
  on a substep at fraction tau = i/q.  For a normal matrix the backward error
  Delta A of one substep has the eigenvalues (log p(z) - c z)/h_s, z the
  normalised eigenvalues, so the condition ||Delta A|| <= eps_A ||A|| of the
  paper, with ||A|| replaced by its bound beta, reads
      max_{z in i[-2,2]} |log(p_m(z) e^{-c z})| + u_p H_m <= 2 c eps_A,
  checked on 4097 points z = i 2 l/4096 (the conjugate half follows by
  symmetry).  H_m = max_z sum_k |d_k w_k(z)| bounds the rounding of the
  Newton sum in a precision with unit roundoff u_p.  The same condition with
  tau c must hold for every output fraction tau = i/q.  Among q with
  q dt/dt_CFL <= 32 and even m <= 120 the pair with the fewest operator
  applications per step, m/q, wins (ties: the smaller q).
* Dense output.  Within one substep the Newton basis w_k(X) b does not
  depend on the time; the value at fraction tau uses the divided differences
  of exp(tau c z) on the same points ("intermediate interpolations").
* Synchronisation.  The leapfrog window problem ends in (e^n, h^{n-1/2});
  the homogeneous problem starts from (e^n, h^n) with
  h^n = h^{n-1/2} - (dt/2) M_mu^{-1} C e^n (a half magnetic step), the
  second-order value of h at the time of e^n.
* Staggering (eqs. averaging1/2).  The homogeneous solutions are added to e
  at t^{m+1} and to h at t^{m+1/2}: the final h of a member is its value at
  T - dt/2.
* Not carried over: shifting and balancing (the spectrum of a skew matrix is
  centred at 0; balancing needs the assembled matrix) and the early
  termination of the series (the degree is fixed by the condition above).

Parity status: pinned by tests/test_oracle_expo.py (dense matrix exponential
on 4^3 grids, interpolation property of the divided differences, conjugate
Leja points against a brute-force maximisation, backward-error condition
against the eigen-decomposition, dt^2 convergence of ParaExp to the leapfrog
solution).
"""
from __future__ import annotations

import math

import mpmath
import numpy as np

NGRID = 1 << 15
NSAMPLE = 4096
CMAX = 32.0
MMAX = 120
DPS = 130


def unit_roundoff(precision):
    return 2.0 ** -24 if int(precision) == 32 else 2.0 ** -53


def leja_etas(npairs):
    """eta_1..eta_npairs of the conjugate Leja points i*eta, -i*eta on i[-2, 2]
    (xi_0 = 0 first)."""
    grid = 2.0 * np.arange(NGRID + 1) / NGRID
    with np.errstate(divide="ignore"):
        score = np.log(grid)                       # distance to xi_0 = 0
    etas = []
    for _ in range(npairs):
        l = int(np.argmax(score))
        eta = float(grid[l])
        etas.append(eta)
        with np.errstate(divide="ignore"):
            score = score + np.log(np.abs(grid - eta)) + np.log(grid + eta)
    return np.array(etas)


def nodes(kind, m):
    """The m+1 interpolation points xi_0..xi_m (complex)."""
    if kind == "taylor":
        return np.zeros(m + 1, dtype=complex)
    etas = leja_etas((m + 1) // 2)
    z = [0j]
    for eta in etas:
        z += [1j * eta, -1j * eta]
    return np.array(z[: m + 1])


def divided_differences(xi, a):
    """Newton coefficients d_k = f[xi_0..xi_k] of f(z) = exp(a z), by the
    recursive definition at high precision.  Coincident points (Taylor) use
    the confluent limit f^(k)(0)/k! = a^k/k!."""
    with mpmath.workdps(DPS):
        a = mpmath.mpf(float(a))
        if np.all(xi == 0):
            return np.array([complex(a ** k / mpmath.factorial(k)) for k in range(len(xi))])
        z = [mpmath.mpc(complex(v).real, complex(v).imag) for v in xi]
        col = [mpmath.exp(a * v) for v in z]
        out = [col[0]]
        for k in range(1, len(z)):
            col = [(col[i + 1] - col[i]) / (z[i + k] - z[i]) for i in range(len(col) - 1)]
            out.append(col[0])
        return np.array([complex(v) for v in out])


def _samples():
    return 1j * 2.0 * np.arange(NSAMPLE + 1) / NSAMPLE


def _errors(xi, d, c, up):
    """For m = 0..len(xi)-1: max over the samples of |log(p_m e^{-cz})| + u_p H_m."""
    z = _samples()
    w = np.ones_like(z)
    p = np.zeros_like(z)
    hump = np.zeros(z.shape)
    out = []
    ecz = np.exp(-c * z)
    for k in range(len(xi)):
        term = d[k] * w
        p = p + term
        hump = hump + np.abs(term)
        with np.errstate(divide="ignore", invalid="ignore"):
            delta = np.abs(np.log(p * ecz))
        out.append(float(np.max(np.nan_to_num(delta, nan=np.inf))) + up * float(np.max(hump)))
        w = w * (z - xi[k])
    return out


def plan(kind, u, tol, precision=64):
    key = (kind, float(u), float(tol), int(precision))
    if key not in _PLANS:
        _PLANS[key] = _plan(*key)
    return _PLANS[key]


_PLANS = {}


def _plan(kind, u, tol, precision):
    """(q, m): substep q*dt and degree m for the step ratio u = dt/dt_CFL and
    the backward-error tolerance tol (eps_A).  For each q the degree is the
    smallest even m whose substep (tau = 1) meets the condition, raised until
    every output fraction tau = i/q meets it too; the pair with the least
    m/q wins, ties going to the smaller q.  Raises if no pair qualifies."""
    up = unit_roundoff(precision)
    xi = nodes(kind, MMAX)
    cands = []
    q = 1
    while q * u <= CMAX:
        c = q * u
        err = _errors(xi, divided_differences(xi, c), c, up)
        ok = [m for m in range(2, MMAX + 1, 2) if err[m] <= 2.0 * c * tol]
        if ok:
            cands.append((ok[0] / q, q, ok[0]))
        q += 1
    cands.sort()
    best = None
    for cost1, q, m in cands:
        if best is not None and (cost1, q) > best:
            break                       # m/q at tau = 1 bounds the final m/q from below
        c = q * u
        while m <= MMAX:
            fails = False
            for i in range(1, q):
                tau = i / q
                err = _errors(xi[: m + 1], divided_differences(xi[: m + 1], tau * c), tau * c, up)
                if err[m] > 2.0 * tau * c * tol:
                    fails = True
                    break
            if not fails:
                break
            m += 2
        if m <= MMAX and (best is None or (m / q, q) < best):
            best = (m / q, q)
            best_m = m
    if best is None:
        raise ValueError("no substep and degree meet the tolerance")
    return best[1], best_m


class _Ops:
    """Transform and operator of the paper on an oracle grid."""

    def __init__(self, og, dt_cfl):
        self.og = og
        self.dt_cfl = float(dt_cfl)
        self.se = np.sqrt(og.meps)       # zero off the electric degrees of freedom
        self.sh = np.sqrt(og.mmu)

    def to_u(self, e, h):
        return np.concatenate([(self.sh * h).ravel(), (self.se * e).ravel()])

    def from_u(self, u):
        n = self.og.meps.size
        uh, ue = u[:n].reshape(self.og.field_shape), u[n:].reshape(self.og.field_shape)
        with np.errstate(divide="ignore", invalid="ignore"):
            e = np.where(self.se > 0, ue / np.where(self.se > 0, self.se, 1.0), 0.0)
            h = np.where(self.sh > 0, uh / np.where(self.sh > 0, self.sh, 1.0), 0.0)
        return e, h

    def A(self, u):
        n = self.og.meps.size
        oe, oh = self.og.apply_A(u[n:], u[:n])
        return np.concatenate([oh.ravel(), oe.ravel()])

    def X(self, u):
        """X = dt_CFL A (complex vectors: real and imaginary parts separately)."""
        if np.iscomplexobj(u):
            return self.dt_cfl * (self.A(u.real) + 1j * self.A(u.imag))
        return self.dt_cfl * self.A(u)


def _basis(ops, b, xi):
    """Newton basis w_0 = b, w_{k+1} = (X - xi_k) w_k for k < m."""
    w = b.astype(complex)
    out = [w]
    for k in range(len(xi) - 1):
        w = ops.X(w) - xi[k] * w
        out.append(w)
    return out


def _combine(basis, d):
    v = np.zeros_like(basis[0])
    for dk, wk in zip(d, basis):
        v = v + dk * wk
    return v.real


def spectral_bound(og):
    """beta >= ||A||_2: 2/dt_CFL of eq. (cfl) on a uniform grid (the Yee bound
    the estimate comes from), the largest absolute row sum of A (||A||_1) on a
    graded grid, where eq. (cfl) is only an estimate."""
    from . import cfl_dt
    if og.graded is None:
        return 2.0 / cfl_dt((og.nx, og.ny, og.nz), og.spacing, og.eps_r, og.mu_r)
    return og.A_rowsum()[0]


def propagate(og, nsteps, e0, h0, probes=(), kind="leja", q=None, m=None, tol=1e-12, precision=64,
              dt_cfl=None, stagger_h=False):
    """w(t) = exp((t - t0) A) u0 from the synchronised state (e0, h0) at t0,
    in substeps L_{m,c}(q dt A) with dense output at every leapfrog step.
    Returns (probes[n, p] = e at t0 + (n+1) dt, e(T), h(T) or, with
    stagger_h, h(T - dt/2)), T = t0 + nsteps dt.  dt_cfl is the normalisation
    2/beta (X = (2/beta) A); by default beta = spectral_bound(og)."""
    dt_cfl = float(dt_cfl) if dt_cfl is not None else 2.0 / spectral_bound(og)
    u = og.dt / dt_cfl
    if q is None or m is None:
        q, m = plan(kind, u, tol, precision)
    ops = _Ops(og, dt_cfl)
    xi = nodes(kind, m)
    c = q * u
    dfull = divided_differences(xi, c)
    douts = [divided_differences(xi, (i / q) * c) for i in range(1, q + 1)]
    pr = np.zeros((nsteps, len(probes)))
    b = ops.to_u(np.asarray(e0, dtype=float), np.asarray(h0, dtype=float))
    nsub = max(1, -(-nsteps // q))
    e_fin = h_fin = None
    for s in range(nsub):
        basis = _basis(ops, b, xi)
        for i in range(1, q + 1):
            n = s * q + i
            if n > nsteps:
                break
            e, _ = ops.from_u(_combine(basis, douts[i - 1]))
            for p, d in enumerate(probes):
                pr[n - 1, p] = e[int(d["axis"]), int(d["k"]), int(d["j"]), int(d["i"])]
        if s == nsub - 1:
            rem = nsteps - s * q
            e_fin, _ = ops.from_u(_combine(basis, divided_differences(xi, (rem / q) * c)))
            th = (rem - 0.5) / q if stagger_h else rem / q
            _, h_fin = ops.from_u(_combine(basis, divided_differences(xi, th * c)))
        else:
            b = _combine(basis, dfull)
    if nsteps == 0:
        e_fin, h_fin = np.array(e0, dtype=float), np.array(h0, dtype=float)
    return pr, e_fin, h_fin


def half_h_step(og, e, h):
    """h^n = h^{n-1/2} - (dt/2) M_mu^{-1} C e^n, through the operator A
    ((A u)_h = -M_mu^{-1/2} C e)."""
    n = og.meps.size
    ops = _Ops(og, 1.0)
    Au = ops.A(ops.to_u(e, h))
    with np.errstate(divide="ignore", invalid="ignore"):
        dh = np.where(ops.sh > 0, Au[:n].reshape(og.field_shape) / np.where(ops.sh > 0, ops.sh, 1.0), 0.0)
    return h + 0.5 * og.dt * dh


def paraexp(og, K, win, sources=(), probes=(), kind="leja", q=None, m=None, tol=1e-12, precision=64,
            dt_cfl=None, e0=None, h0=None):
    """ParaExp (Algorithm 1) with leapfrog window problems v_j and the
    homogeneous problems w_{j+1} = exp((t - T_j) A) v_j(T_j) by the
    propagator above.  The initial value (e0, h0) = (e^{W_0}, h^{W_0-1/2})
    (zero if both are None) gives w_1, synchronised like the v_j.  Returns
    (probes[n, p] for absolute steps win[0]+1..win[K], e(T), h(T - dt/2))."""
    win = [int(v) for v in win]
    nt = win[K] - win[0]
    if dt_cfl is None:
        dt_cfl = 2.0 / spectral_bound(og)
    if q is None or m is None:
        q, m = plan(kind, og.dt / dt_cfl, tol, precision)
    pr = np.zeros((nt, len(probes)))
    e_fin, h_fin = og.zeros(), og.zeros()
    for j in range(1, K + 1):
        lo, hi = win[j - 1], win[j]
        p1, _, e, h = og.leapfrog(hi - lo, sources, probes, step0=lo, src_window=(lo, hi))
        pr[lo - win[0]: hi - win[0]] += p1
        if j == K:
            e_fin += e
            h_fin += h
            continue
        hs = half_h_step(og, e, h)
        p2, ew, hw = propagate(og, win[K] - hi, e, hs, probes, kind, q, m, tol, precision, dt_cfl,
                               stagger_h=True)
        pr[hi - win[0]:] += p2
        e_fin += ew
        h_fin += hw
    if e0 is not None or h0 is not None:
        e = og.zeros() if e0 is None else np.asarray(e0, dtype=float)
        h = og.zeros() if h0 is None else np.asarray(h0, dtype=float)
        p2, ew, hw = propagate(og, nt, e, half_h_step(og, e, h), probes, kind, q, m, tol, precision, dt_cfl,
                               stagger_h=True)
        pr += p2
        e_fin += ew
        h_fin += hw
    return pr, e_fin, h_fin


def smvp_count(kind, nsteps, q, m):
    """Operator applications of one propagation over nsteps steps: m per
    substep (the cost C_Leja of the paper, counted in applications of A)."""
    return m * max(1, math.ceil(nsteps / q))
