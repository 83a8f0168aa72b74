"""Serial FP64 CPU oracle for the FIT leapfrog + ParaExp method.

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library: ``fit_oracle.c`` is compiled on its own with gcc and
called through ctypes.

Field arrays use the canonical FIT layout of Sec. II: every component is an
array over the (nx+1)(ny+1)(nz+1) primal points, x fastest; numpy shape
``(3, nz+1, ny+1, nx+1)``.  Per-cell materials have shape ``(nz, ny, nx)``.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(dense brute force, Yee dispersion eigenvalues, energy balance, Gauss law,
mirror/rotation symmetry, ParaExp linearity, finite differences; graded
grids: uniform limit, exact energy of uniform fields, eigenvalue bounds).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fit_oracle.c")
_SO = os.path.join(_HERE, "_build", "libfit_oracle.so")
_lock = threading.Lock()
_lib = None


class _Grid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("d", ctypes.c_double * 3), ("dt", ctypes.c_double),
        ("ca", ctypes.c_void_p), ("cb", ctypes.c_void_p), ("ch", ctypes.c_void_p),
        ("meps", ctypes.c_void_p), ("mmu", ctypes.c_void_p), ("store32", ctypes.c_int),
    ]


class _Source(ctypes.Structure):
    _fields_ = [("axis", ctypes.c_int), ("i", ctypes.c_int), ("j", ctypes.c_int), ("k", ctypes.c_int),
                ("waveform", ctypes.c_int), ("amp", ctypes.c_double), ("f0", ctypes.c_double),
                ("width", ctypes.c_double), ("delay", ctypes.c_double)]


class _Probe(ctypes.Structure):
    _fields_ = [("axis", ctypes.c_int), ("i", ctypes.c_int), ("j", ctypes.c_int), ("k", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile fit_oracle.c into a shared library (gcc, no FMA contraction)."""
    with _lock:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
            return _SO
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        D, I, L, P = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
        lib.oracle_cfl_dt.restype = D
        lib.oracle_cfl_dt.argtypes = [I, I, I, D, D, D, P, P]
        lib.oracle_coeffs.restype = I
        lib.oracle_coeffs.argtypes = [I, I, I, D, D, D, P, P, P, D, I, I, P, P, P, P, P, P]
        lib.oracle_waveform.restype = D
        lib.oracle_waveform.argtypes = [I, D, D, D, D, D]
        lib.oracle_leapfrog.restype = I
        lib.oracle_leapfrog.argtypes = [ctypes.POINTER(_Grid), L, L, L, L, P, I, P, I, P, P, P, P]
        lib.oracle_paraexp.restype = I
        lib.oracle_paraexp.argtypes = [ctypes.POINTER(_Grid), I, P, P, I, P, I, P, P, P, P, P]
        lib.oracle_adjoint.restype = I
        lib.oracle_adjoint.argtypes = [ctypes.POINTER(_Grid), P, P, I, L, L, P, I, P, I, P, P]
        lib.oracle_adjoint_graded.restype = I
        lib.oracle_adjoint_graded.argtypes = [ctypes.POINTER(_Grid), P, P, P, P, P, I, L, L, P, I, P, I, P, P]
        lib.oracle_cfl_dt_graded.restype = D
        lib.oracle_cfl_dt_graded.argtypes = [I, I, I, P, P, P, P, P]
        lib.oracle_coeffs_graded.restype = I
        lib.oracle_coeffs_graded.argtypes = [I, I, I, P, P, P, P, P, P, D, I, I, P, P, P, P, P, P]
        lib.oracle_A_rowsum.restype = D
        lib.oracle_A_rowsum.argtypes = [ctypes.POINTER(_Grid), P, P]
        lib.oracle_apply_A.restype = I
        lib.oracle_apply_A.argtypes = [ctypes.POINTER(_Grid), P, P, P, P]
        lib.oracle_constants.restype = None
        lib.oracle_constants.argtypes = [P, P, P]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a, shape):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.shape != shape:
        a = a.reshape(shape)
    return a


def constants():
    """(c0, mu0, eps0) in SI units as used by the oracle."""
    out = [ctypes.c_double() for _ in range(3)]
    _load().oracle_constants(*[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def waveform(kind, amp, f0, width, delay, t):
    return _load().oracle_waveform(int(kind), float(amp), float(f0), float(width), float(delay), float(t))


def graded_spacing(dims, spacing):
    """Per-axis cell sizes (three float64 arrays) if `spacing` holds any
    array, else None (a uniform grid)."""
    if all(np.ndim(v) == 0 for v in spacing):
        return None
    out = []
    for n, v in zip(dims, spacing):
        a = np.full(int(n), float(v)) if np.ndim(v) == 0 else np.ascontiguousarray(v, dtype=np.float64)
        if a.shape != (int(n),):
            raise ValueError("a graded spacing needs one size per cell along its axis")
        out.append(a)
    return out


def cfl_dt(dims, spacing, eps_r, mu_r=None):
    """Eq. (cfl): the largest stable step estimate (per-cell sizes on a graded grid)."""
    nx, ny, nz = dims
    e = _f32(eps_r, (nz, ny, nx))
    m = _f32(mu_r, (nz, ny, nx))
    gs = graded_spacing(dims, spacing)
    if gs is not None:
        return _load().oracle_cfl_dt_graded(nx, ny, nz, *(_ptr(a) for a in gs), _ptr(e), _ptr(m))
    return _load().oracle_cfl_dt(nx, ny, nz, *map(float, spacing), _ptr(e), _ptr(m))


def _structs(sources, probes):
    src = (_Source * max(1, len(sources)))()
    for s, d in zip(src, sources):
        s.axis, s.i, s.j, s.k = int(d["axis"]), int(d["i"]), int(d["j"]), int(d["k"])
        s.waveform = int(d.get("waveform", 0))
        s.amp, s.f0 = float(d.get("amp", 1.0)), float(d.get("f0", 0.0))
        s.width, s.delay = float(d.get("width", 1.0)), float(d.get("delay", 0.0))
    prb = (_Probe * max(1, len(probes)))()
    for p, d in zip(prb, probes):
        p.axis, p.i, p.j, p.k = int(d["axis"]), int(d["i"]), int(d["j"]), int(d["k"])
    return src, prb


class OracleGrid:
    """A grid with its FP64 material matrices and leapfrog coefficients.

    ``round32`` rounds ca, cb, ch to float, as stored by an FP32 field path.
    ``store32`` also rounds every stored e and h value to float after its
    update (arithmetic stays FP64): the error model of keeping the fields in
    float, used only to derive FP32 test tolerances.
    """

    def __init__(self, dims, spacing, eps_r, mu_r=None, sigma=None, dt=None,
                 cfl_fraction=0.95, sigma_scheme=0, round32=False, store32=False):
        self.nx, self.ny, self.nz = (int(v) for v in dims)
        self.graded = graded_spacing(dims, spacing)
        self.spacing = (tuple(float(np.mean(a)) for a in self.graded) if self.graded is not None
                        else tuple(float(v) for v in spacing))
        shp = (self.nz, self.ny, self.nx)
        self.eps_r = _f32(eps_r, shp)
        self.mu_r = _f32(mu_r, shp)
        self.sigma = _f32(sigma, shp)
        self.sigma_scheme = int(sigma_scheme)
        self.round32 = bool(round32)
        if dt is None:
            dt = cfl_fraction * cfl_dt(dims, spacing if self.graded is not None else self.spacing, self.eps_r,
                                       self.mu_r)
        self.dt = float(dt)
        fshape = (3, self.nz + 1, self.ny + 1, self.nx + 1)
        self.field_shape = fshape
        self.ca, self.cb, self.ch = (np.zeros(fshape) for _ in range(3))
        self.meps, self.msig, self.mmu = (np.zeros(fshape) for _ in range(3))
        if self.graded is not None:
            rc = _load().oracle_coeffs_graded(self.nx, self.ny, self.nz, *(_ptr(a) for a in self.graded),
                                              _ptr(self.eps_r), _ptr(self.mu_r), _ptr(self.sigma),
                                              self.dt, self.sigma_scheme, int(self.round32),
                                              _ptr(self.ca), _ptr(self.cb), _ptr(self.ch),
                                              _ptr(self.meps), _ptr(self.msig), _ptr(self.mmu))
        else:
            rc = _load().oracle_coeffs(self.nx, self.ny, self.nz, *self.spacing,
                                       _ptr(self.eps_r), _ptr(self.mu_r), _ptr(self.sigma),
                                       self.dt, self.sigma_scheme, int(self.round32),
                                       _ptr(self.ca), _ptr(self.cb), _ptr(self.ch),
                                       _ptr(self.meps), _ptr(self.msig), _ptr(self.mmu))
        if rc:
            raise ValueError(f"oracle_coeffs failed ({rc})")
        self._g = _Grid(self.nx, self.ny, self.nz, (ctypes.c_double * 3)(*self.spacing), self.dt,
                        _ptr(self.ca).value, _ptr(self.cb).value, _ptr(self.ch).value,
                        _ptr(self.meps).value, _ptr(self.mmu).value, int(bool(store32)))

    def zeros(self):
        return np.zeros(self.field_shape)

    def leapfrog(self, nsteps, sources=(), probes=(), step0=0, src_window=None,
                 e=None, h=None, energy=False):
        """Run nsteps of the leapfrog; returns (probes[n, p], energy[n] | None, e, h)."""
        e = self.zeros() if e is None else np.array(e, dtype=np.float64).reshape(self.field_shape)
        h = self.zeros() if h is None else np.array(h, dtype=np.float64).reshape(self.field_shape)
        lo, hi = src_window if src_window is not None else (-(2 ** 62), 2 ** 62)
        src, prb = _structs(sources, probes)
        pr = np.zeros((max(0, nsteps), len(probes)))
        en = np.zeros(max(0, nsteps)) if energy else None
        rc = _load().oracle_leapfrog(ctypes.byref(self._g), int(nsteps), int(step0), int(lo), int(hi),
                                     ctypes.cast(src, ctypes.c_void_p), len(sources),
                                     ctypes.cast(prb, ctypes.c_void_p), len(probes),
                                     _ptr(pr), _ptr(en), _ptr(e), _ptr(h))
        if rc:
            raise ValueError(f"oracle_leapfrog failed ({rc})")
        return pr, en, e, h

    def paraexp(self, K, win, sources=(), probes=(), e0=None, h0=None):
        """ParaExp with leapfrog members; returns (probes[n, p], e_final, h_final)."""
        win = np.ascontiguousarray(win, dtype=np.int64)
        assert len(win) == K + 1
        nt = int(win[-1] - win[0])
        src, prb = _structs(sources, probes)
        pr = np.zeros((nt, len(probes)))
        ef, hf = self.zeros(), self.zeros()
        e0 = None if e0 is None else np.ascontiguousarray(e0, dtype=np.float64).reshape(self.field_shape)
        h0 = None if h0 is None else np.ascontiguousarray(h0, dtype=np.float64).reshape(self.field_shape)
        rc = _load().oracle_paraexp(ctypes.byref(self._g), int(K), _ptr(win),
                                    ctypes.cast(src, ctypes.c_void_p), len(sources),
                                    ctypes.cast(prb, ctypes.c_void_p), len(probes),
                                    _ptr(e0), _ptr(h0), _ptr(pr), _ptr(ef), _ptr(hf))
        if rc:
            raise ValueError(f"oracle_paraexp failed ({rc})")
        return pr, ef, hf

    def apply_A(self, ue, uh):
        """The skew system matrix of eq. (FIT_ode_2) on transformed unknowns
        u = [M_mu^{1/2} h, M_eps^{1/2} e]; returns ((A u)_e, (A u)_h)."""
        ue = np.ascontiguousarray(ue, dtype=np.float64).reshape(self.field_shape)
        uh = np.ascontiguousarray(uh, dtype=np.float64).reshape(self.field_shape)
        oe, oh = self.zeros(), self.zeros()
        rc = _load().oracle_apply_A(ctypes.byref(self._g), _ptr(ue), _ptr(uh), _ptr(oe), _ptr(oh))
        if rc:
            raise ValueError(f"oracle_apply_A failed ({rc})")
        return oe, oh

    def A_rowsum(self):
        """max absolute row sum of A (= ||A||_1 = ||A||_inf, a bound on ||A||_2)
        and the sums per edge and face."""
        oe, oh = self.zeros(), self.zeros()
        best = _load().oracle_A_rowsum(ctypes.byref(self._g), _ptr(oe), _ptr(oh))
        return best, oe, oh

    def adjoint(self, nsteps, sources=(), probes=(), step0=0):
        """J = sum_n sum_p (e_p^n/L_p)^2 and dJ/d eps_r per cell (shape (nz, ny, nx)).
        L_p is the probe edge's length (on a graded grid the size of the cell
        it runs through along its axis)."""
        src, prb = _structs(sources, probes)
        J = np.zeros(1)
        g = np.zeros((self.nz, self.ny, self.nx))
        if self.graded is not None:
            rc = _load().oracle_adjoint_graded(ctypes.byref(self._g), *(_ptr(a) for a in self.graded),
                                               _ptr(self.eps_r), _ptr(self.sigma), self.sigma_scheme,
                                               int(nsteps), int(step0), ctypes.cast(src, ctypes.c_void_p),
                                               len(sources), ctypes.cast(prb, ctypes.c_void_p), len(probes),
                                               _ptr(J), _ptr(g))
        else:
            rc = _load().oracle_adjoint(ctypes.byref(self._g), _ptr(self.eps_r), _ptr(self.sigma),
                                        self.sigma_scheme, int(nsteps), int(step0),
                                        ctypes.cast(src, ctypes.c_void_p), len(sources),
                                        ctypes.cast(prb, ctypes.c_void_p), len(probes), _ptr(J), _ptr(g))
        if rc:
            raise ValueError(f"oracle_adjoint failed ({rc})")
        return float(J[0]), g


def to_compact(a):
    """Canonical (3, nz+1, ny+1, nx+1) -> compact (3, nz, ny, nx): drop the
    slices at index n along an axis, which are identically zero under PEC."""
    return np.ascontiguousarray(a[:, :-1, :-1, :-1])
