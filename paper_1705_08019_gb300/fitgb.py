"""ctypes binding of libfitgb.so (include/fitgb.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  The functions keep the C names; arrays may be numpy arrays (host)
or torch CUDA tensors (device) -- the library tells them apart itself.  If the
library is not built or cannot be loaded, every call raises ``RuntimeError``;
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfitgb.so")

FIT_OK = 0
FIT_ERR_ARG = -1
FIT_ERR_CFL = -2
FIT_ERR_OOM = -3
FIT_ERR_CUDA = -4
FIT_ERR_TIMEOUT = -5
FIT_ERR_NONFINITE = -6
FIT_ERR_UNSUPPORTED = -7

WAVE_GAUSS_SINE, WAVE_GAUSS, WAVE_SINE = 0, 1, 2
FIT_FLAG_COEF_FLOAT = 1

HOMOG_LEAPFROG, HOMOG_LEJA, HOMOG_TAYLOR = 0, 1, 2
HOMOG = {"leapfrog": HOMOG_LEAPFROG, "leja": HOMOG_LEJA, "taylor": HOMOG_TAYLOR}

EXPORTED = ("fit_grid_create", "fit_grid_destroy", "fit_cfl_dt", "fit_grid_info", "fit_leapfrog_run",
            "paraexp_run", "paraexp_run_batched", "fit_adjoint_grad", "fit_sync", "fit_strerror",
            "fit_version", "fit_last_stats", "fit_leapfrog_run_static", "fit_expo_plan", "fit_expo_coeffs",
            "fit_expo_propagate", "fit_grid_create_graded", "fit_spectral_bound", "fit_debug_fail_alloc",
            "fit_debug_chunk_length")


class FitError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})")


class fit_source(ctypes.Structure):
    _fields_ = [("axis", ctypes.c_int), ("i", ctypes.c_int), ("j", ctypes.c_int), ("k", ctypes.c_int),
                ("waveform", ctypes.c_int), ("amp", ctypes.c_double), ("f0", ctypes.c_double),
                ("width", ctypes.c_double), ("delay", ctypes.c_double)]


class fit_probe(ctypes.Structure):
    _fields_ = [("axis", ctypes.c_int), ("i", ctypes.c_int), ("j", ctypes.c_int), ("k", ctypes.c_int)]


class fit_run_opts(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("tile_z", ctypes.c_int),
                ("autotune", ctypes.c_int), ("use_graph", ctypes.c_int), ("sigma_scheme", ctypes.c_int),
                ("sum_mode", ctypes.c_int), ("members_per_pass", ctypes.c_int), ("force_dt", ctypes.c_int),
                ("profile", ctypes.c_int), ("kernel", ctypes.c_int), ("stages", ctypes.c_int),
                ("debug_wait_limit", ctypes.c_int), ("debug_extra_tx", ctypes.c_int),
                ("homogeneous", ctypes.c_int), ("expo_substep", ctypes.c_int), ("expo_degree", ctypes.c_int),
                ("expo_tol", ctypes.c_double), ("steps_per_launch", ctypes.c_int), ("adjoint_mem_mb", ctypes.c_int)]


class fit_run_stats(ctypes.Structure):
    _fields_ = [("step_launches", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong),
                ("cell_updates", ctypes.c_longlong), ("alg_bytes", ctypes.c_double), ("step_ms", ctypes.c_double),
                ("expo_launches", ctypes.c_longlong), ("expo_applications", ctypes.c_longlong),
                ("expo_alg_bytes", ctypes.c_double), ("expo_ms", ctypes.c_double)]


class fit_paraexp_problem(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_void_p), ("dt", ctypes.c_double), ("K", ctypes.c_int),
                ("win", ctypes.c_void_p), ("src", ctypes.c_void_p), ("nsrc", ctypes.c_int),
                ("prb", ctypes.c_void_p), ("nprb", ctypes.c_int), ("probe_out", ctypes.c_void_p),
                ("e_final", ctypes.c_void_p), ("h_final", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def load():
    """Load libfitgb.so (raises RuntimeError if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfitgb.so is not built ({LIB_PATH}); run "
                               "`python -m paper_1705_08019_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(LIB_PATH)
        I, L, D, P, U = ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_void_p, ctypes.c_uint
        lib.fit_grid_create.argtypes = [I, I, I, D, D, D, P, P, P, I, U, ctypes.POINTER(P)]
        lib.fit_grid_create.restype = I
        lib.fit_grid_create_graded.argtypes = [I, I, I, P, P, P, P, P, P, I, U, ctypes.POINTER(P)]
        lib.fit_grid_create_graded.restype = I
        lib.fit_spectral_bound.argtypes = [P, ctypes.POINTER(D)]
        lib.fit_spectral_bound.restype = I
        lib.fit_grid_destroy.argtypes = [P]
        lib.fit_grid_destroy.restype = None
        lib.fit_cfl_dt.argtypes = [P, ctypes.POINTER(D)]
        lib.fit_cfl_dt.restype = I
        lib.fit_grid_info.argtypes = [P, P, P, P, P, P]
        lib.fit_grid_info.restype = I
        lib.fit_leapfrog_run.argtypes = [P, D, L, L, P, I, P, I, P, P, P, P, P, P]
        lib.fit_leapfrog_run.restype = I
        lib.paraexp_run.argtypes = [P, D, I, P, P, I, P, I, P, P, P, P, P, P, P]
        lib.paraexp_run.restype = I
        lib.paraexp_run_batched.argtypes = [P, I, P, P]
        lib.paraexp_run_batched.restype = I
        lib.fit_adjoint_grad.argtypes = [P, D, L, P, I, P, I, I, P, P, P, P]
        lib.fit_adjoint_grad.restype = I
        lib.fit_leapfrog_run_static.argtypes = [I, I, I, D, D, D, P, P, D, L, L, P, I, P, I, P, P, P, P]
        lib.fit_leapfrog_run_static.restype = I
        lib.fit_expo_plan.argtypes = [I, D, D, I, ctypes.POINTER(I), ctypes.POINTER(I)]
        lib.fit_expo_plan.restype = I
        lib.fit_expo_coeffs.argtypes = [I, I, D, P, P, P]
        lib.fit_expo_coeffs.restype = I
        lib.fit_expo_propagate.argtypes = [P, D, L, P, I, P, P, P, P, P]
        lib.fit_expo_propagate.restype = I
        lib.fit_last_stats.argtypes = [P, ctypes.POINTER(fit_run_stats)]
        lib.fit_last_stats.restype = I
        lib.fit_sync.argtypes = [P, P]
        lib.fit_sync.restype = I
        lib.fit_debug_fail_alloc.argtypes = [ctypes.c_longlong]
        lib.fit_debug_fail_alloc.restype = I
        lib.fit_debug_chunk_length.argtypes = [I, I, I, I, I, I, I, ctypes.c_longlong]
        lib.fit_debug_chunk_length.restype = I
        lib.fit_strerror.argtypes = [I]
        lib.fit_strerror.restype = ctypes.c_char_p
        lib.fit_version.argtypes = []
        lib.fit_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def fit_debug_fail_alloc(after: int):
    """Test hook: the device allocation `after` allocations from now fails as
    out of memory (negative: off)."""
    _check(load().fit_debug_fail_alloc(int(after)), "fit_debug_fail_alloc")


def fit_debug_chunk_length(dims, tile, kz_max, nmem, slots):
    """Test hook: the z chunk length the library takes for a single-grid step
    launch (host computation, no device call)."""
    nx, ny, nz = dims
    r = load().fit_debug_chunk_length(int(nx), int(ny), int(nz), int(tile[0]), int(tile[1]), int(kz_max), int(nmem),
                                      int(slots))
    if r < 0:
        _check(r, "fit_debug_chunk_length")
    return r


def strerror(status: int) -> str:
    return load().fit_strerror(int(status)).decode()


def fit_version() -> str:
    return load().fit_version().decode()


# ----------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------

def _addr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def sources_array(sources):
    arr = (fit_source * max(1, len(sources)))()
    for s, d in zip(arr, sources):
        s.axis, s.i, s.j, s.k = int(d["axis"]), int(d["i"]), int(d["j"]), int(d["k"])
        s.waveform = int(d.get("waveform", 0))
        s.amp, s.f0 = float(d.get("amp", 1.0)), float(d.get("f0", 0.0))
        s.width, s.delay = float(d.get("width", 1.0)), float(d.get("delay", 0.0))
    return arr


def probes_array(probes):
    arr = (fit_probe * max(1, len(probes)))()
    for p, d in zip(arr, probes):
        p.axis, p.i, p.j, p.k = int(d["axis"]), int(d["i"]), int(d["j"]), int(d["k"])
    return arr


def make_opts(**kw):
    """fit_run_opts from keyword arguments; homogeneous may be given by name
    ("leapfrog", "leja", "taylor")."""
    o = fit_run_opts()
    for k, v in kw.items():
        if k == "homogeneous" and isinstance(v, str):
            v = HOMOG[v]
        setattr(o, k, float(v) if k == "expo_tol" else int(v))
    return o


def _check(rc, where):
    if rc != FIT_OK:
        raise FitError(rc, where)


# ----------------------------------------------------------------------------
# the C entry points, same names
# ----------------------------------------------------------------------------

def fit_grid_create(dims, spacing, eps_r, mu_r=None, sigma=None, precision=32, flags=0):
    """Returns an opaque grid handle (int).  Materials: float32, (nz, ny, nx)."""
    nx, ny, nz = (int(v) for v in dims)
    keep = []

    def f32(a):
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=np.float32)
            if a.size != nx * ny * nz:
                raise ValueError("material array has the wrong size")
        keep.append(a)
        return _addr(a)

    out = ctypes.c_void_p()
    rc = load().fit_grid_create(nx, ny, nz, *(float(v) for v in spacing), f32(eps_r), f32(mu_r), f32(sigma),
                                int(precision), int(flags), ctypes.byref(out))
    _check(rc, "fit_grid_create")
    return out.value


def fit_grid_create_graded(dims, sizes, eps_r, mu_r=None, sigma=None, precision=32, flags=0):
    """Graded grid: sizes = (dx[nx], dy[ny], dz[nz]) per-cell sizes in metres."""
    nx, ny, nz = (int(v) for v in dims)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in sizes]
    if [a.size for a in arrs] != [nx, ny, nz]:
        raise ValueError("one size per cell along each axis")
    keep = list(arrs)

    def f32(a):
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=np.float32)
            if a.size != nx * ny * nz:
                raise ValueError("material array has the wrong size")
        keep.append(a)
        return _addr(a)

    out = ctypes.c_void_p()
    rc = load().fit_grid_create_graded(nx, ny, nz, *(_addr(a) for a in arrs), f32(eps_r), f32(mu_r), f32(sigma),
                                       int(precision), int(flags), ctypes.byref(out))
    _check(rc, "fit_grid_create_graded")
    return out.value


def fit_spectral_bound(g):
    v = ctypes.c_double()
    _check(load().fit_spectral_bound(g, ctypes.byref(v)), "fit_spectral_bound")
    return v.value


def fit_grid_destroy(g):
    load().fit_grid_destroy(g)


def fit_cfl_dt(g):
    v = ctypes.c_double()
    _check(load().fit_cfl_dt(g, ctypes.byref(v)), "fit_cfl_dt")
    return v.value


def fit_leapfrog_run(g, dt, nsteps, step0=0, sources=(), probes=(), probe_out=None, energy_out=None,
                     e_io=None, h_io=None, opts=None, stream=None):
    src, prb = sources_array(sources), probes_array(probes)
    rc = load().fit_leapfrog_run(g, float(dt), int(nsteps), int(step0), ctypes.cast(src, ctypes.c_void_p),
                                 len(sources), ctypes.cast(prb, ctypes.c_void_p), len(probes), _addr(probe_out),
                                 _addr(energy_out), _addr(e_io), _addr(h_io),
                                 ctypes.byref(opts) if opts is not None else None, _stream(stream))
    _check(rc, "fit_leapfrog_run")


def paraexp_run(g, dt, K, win, sources=(), probes=(), probe_out=None, e_final=None, h_final=None,
                e0=None, h0=None, opts=None, stream=None):
    win = np.ascontiguousarray(win, dtype=np.int64)
    if len(win) != K + 1:
        raise ValueError("win needs K+1 entries")
    src, prb = sources_array(sources), probes_array(probes)
    rc = load().paraexp_run(g, float(dt), int(K), _addr(win), ctypes.cast(src, ctypes.c_void_p), len(sources),
                            ctypes.cast(prb, ctypes.c_void_p), len(probes), _addr(probe_out), _addr(e_final),
                            _addr(h_final), _addr(e0), _addr(h0),
                            ctypes.byref(opts) if opts is not None else None, _stream(stream))
    _check(rc, "paraexp_run")


def paraexp_run_batched(problems, opts=None, stream=None):
    """problems: list of dicts with keys grid, dt, K, win, sources, probes,
    probe_out, e_final, h_final."""
    arr = (fit_paraexp_problem * max(1, len(problems)))()
    keep = []
    for q, d in zip(arr, problems):
        win = np.ascontiguousarray(d["win"], dtype=np.int64)
        src, prb = sources_array(d.get("sources", ())), probes_array(d.get("probes", ()))
        keep += [win, src, prb]
        q.grid = d["grid"]
        q.dt = float(d["dt"])
        q.K = int(d["K"])
        q.win = _addr(win)
        q.src = ctypes.cast(src, ctypes.c_void_p)
        q.nsrc = len(d.get("sources", ()))
        q.prb = ctypes.cast(prb, ctypes.c_void_p)
        q.nprb = len(d.get("probes", ()))
        q.probe_out = _addr(d.get("probe_out"))
        q.e_final = _addr(d.get("e_final"))
        q.h_final = _addr(d.get("h_final"))
    rc = load().paraexp_run_batched(ctypes.cast(arr, ctypes.c_void_p), len(problems),
                                    ctypes.byref(opts) if opts is not None else None, _stream(stream))
    _check(rc, "paraexp_run_batched")


def fit_adjoint_grad(g, dt, nsteps, sources=(), probes=(), ckpt_every=0, J_out=None, grad_out=None,
                     opts=None, stream=None):
    src, prb = sources_array(sources), probes_array(probes)
    rc = load().fit_adjoint_grad(g, float(dt), int(nsteps), ctypes.cast(src, ctypes.c_void_p), len(sources),
                                 ctypes.cast(prb, ctypes.c_void_p), len(probes), int(ckpt_every), _addr(J_out),
                                 _addr(grad_out), ctypes.byref(opts) if opts is not None else None,
                                 _stream(stream))
    _check(rc, "fit_adjoint_grad")


def fit_leapfrog_run_static(dims, spacing, eps_r, sigma, dt, nsteps, step0=0, sources=(), probes=(),
                            probe_out=None, e_io=None, h_io=None, stream=None):
    """The allocation-free FP32 leapfrog run; every array argument is a
    device tensor (e_io, h_io: float32, shape (3, nz, ny, nx), in/out)."""
    nx, ny, nz = (int(v) for v in dims)
    src, prb = sources_array(sources), probes_array(probes)
    rc = load().fit_leapfrog_run_static(nx, ny, nz, *(float(v) for v in spacing), _addr(eps_r), _addr(sigma),
                                        float(dt), int(nsteps), int(step0), ctypes.cast(src, ctypes.c_void_p),
                                        len(sources), ctypes.cast(prb, ctypes.c_void_p), len(probes),
                                        _addr(probe_out), _addr(e_io), _addr(h_io), _stream(stream))
    _check(rc, "fit_leapfrog_run_static")


def fit_expo_plan(kind, dt_ratio, tol, precision=64):
    """(substep q, degree m) of the Leja/Taylor propagator (host only)."""
    q, m = ctypes.c_int(), ctypes.c_int()
    _check(load().fit_expo_plan(HOMOG.get(kind, kind), float(dt_ratio), float(tol), int(precision),
                                ctypes.byref(q), ctypes.byref(m)), "fit_expo_plan")
    return q.value, m.value


def fit_expo_coeffs(kind, degree, a):
    """(alpha, gamma, eta^2) of the real Newton form of the interpolant of
    exp(a z), each of length degree/2 (host only)."""
    J = int(degree) // 2
    al, ga, et = np.zeros(J), np.zeros(J), np.zeros(J)
    _check(load().fit_expo_coeffs(HOMOG.get(kind, kind), int(degree), float(a), _addr(al), _addr(ga), _addr(et)),
           "fit_expo_coeffs")
    return al, ga, et


def fit_expo_propagate(g, dt, nsteps, probes=(), probe_out=None, e_io=None, h_io=None, opts=None, stream=None):
    prb = probes_array(probes)
    rc = load().fit_expo_propagate(g, float(dt), int(nsteps), ctypes.cast(prb, ctypes.c_void_p), len(probes),
                                   _addr(probe_out), _addr(e_io), _addr(h_io),
                                   ctypes.byref(opts) if opts is not None else None, _stream(stream))
    _check(rc, "fit_expo_propagate")


def fit_last_stats(g):
    st = fit_run_stats()
    _check(load().fit_last_stats(g, ctypes.byref(st)), "fit_last_stats")
    return dict(step_launches=st.step_launches, kernel_launches=st.kernel_launches,
                cell_updates=st.cell_updates, alg_bytes=st.alg_bytes, step_ms=st.step_ms,
                expo_launches=st.expo_launches, expo_applications=st.expo_applications,
                expo_alg_bytes=st.expo_alg_bytes, expo_ms=st.expo_ms)


def fit_sync(g, stream=None):
    _check(load().fit_sync(g, _stream(stream)), "fit_sync")


# ----------------------------------------------------------------------------
# convenience object
# ----------------------------------------------------------------------------

class Grid:
    """Owns a fit_grid; field arrays use the compact layout (3, nz, ny, nx)."""

    def __init__(self, dims, spacing, eps_r, mu_r=None, sigma=None, precision=32, flags=0):
        self.dims = tuple(int(v) for v in dims)
        self.precision = int(precision)
        # precision 40 (FP32 + bfloat16 residual) and 48 (float pairs): FP64 I/O
        self.dtype = np.float64 if precision in (64, 48, 40) else np.float32
        if all(np.ndim(v) == 0 for v in spacing):
            self.spacing = tuple(float(v) for v in spacing)
            self.handle = fit_grid_create(dims, spacing, eps_r, mu_r, sigma, precision, flags)
        else:   # graded: per-cell sizes along each axis (a scalar stands for a constant axis)
            sizes = [np.full(n, float(v)) if np.ndim(v) == 0 else np.asarray(v, np.float64)
                     for n, v in zip(self.dims, spacing)]
            self.spacing = tuple(sizes)
            self.handle = fit_grid_create_graded(dims, sizes, eps_r, mu_r, sigma, precision, flags)

    @classmethod
    def from_workload(cls, w, precision=None):
        return cls(w.dims, w.spacing, w.eps_r, w.mu_r, w.sigma, precision or w.precision)

    @property
    def field_shape(self):
        nx, ny, nz = self.dims
        return (3, nz, ny, nx)

    def cfl_dt(self):
        return fit_cfl_dt(self.handle)

    def spectral_bound(self):
        return fit_spectral_bound(self.handle)

    def leapfrog(self, dt, nsteps, sources=(), probes=(), step0=0, e=None, h=None, energy=False, opts=None):
        """Host-side convenience: returns (probes[n, p], energy | None, e, h) as numpy."""
        e = np.zeros(self.field_shape, self.dtype) if e is None else np.array(e, dtype=self.dtype)
        h = np.zeros(self.field_shape, self.dtype) if h is None else np.array(h, dtype=self.dtype)
        pr = np.zeros((nsteps, len(probes))) if probes else None
        en = np.zeros(nsteps) if energy else None
        fit_leapfrog_run(self.handle, dt, nsteps, step0, sources, probes, pr, en, e, h, opts)
        return pr, en, e, h

    def paraexp(self, dt, K, win, sources=(), probes=(), e0=None, h0=None, opts=None, finals=True):
        nt = int(win[-1] - win[0])
        pr = np.zeros((nt, len(probes))) if probes else None
        ef = np.zeros(self.field_shape) if finals else None
        hf = np.zeros(self.field_shape) if finals else None
        if e0 is not None:
            e0 = np.ascontiguousarray(e0, dtype=self.dtype)
        if h0 is not None:
            h0 = np.ascontiguousarray(h0, dtype=self.dtype)
        paraexp_run(self.handle, dt, K, win, sources, probes, pr, ef, hf, e0, h0, opts)
        return pr, ef, hf

    def expo_propagate(self, dt, nsteps, e, h, probes=(), kind="leja", tol=0.0, q=0, m=0):
        """Host-side convenience: exp(nsteps dt A) of a synchronised state;
        returns (probes[n, p], e, h) as numpy."""
        e = np.array(e, dtype=self.dtype)
        h = np.array(h, dtype=self.dtype)
        pr = np.zeros((nsteps, len(probes))) if probes else None
        opts = make_opts(homogeneous=kind, expo_tol=tol, expo_substep=q, expo_degree=m)
        fit_expo_propagate(self.handle, dt, nsteps, probes, pr, e, h, opts)
        return pr, e, h

    def adjoint(self, dt, nsteps, sources=(), probes=(), ckpt_every=0, opts=None):
        nx, ny, nz = self.dims
        J = np.zeros(1)
        g = np.zeros((nz, ny, nx))
        fit_adjoint_grad(self.handle, dt, nsteps, sources, probes, ckpt_every, J, g, opts)
        return float(J[0]), g

    def close(self):
        if getattr(self, "handle", None):
            fit_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
