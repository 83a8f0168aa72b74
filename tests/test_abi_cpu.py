"""Host-side checks of the C ABI library (no GPU needed): it builds, loads,
and exports every function include/fitgb.h declares; the binding knows them."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fitgb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\([^;]*\)\s*;", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fit_grid_create", "fit_leapfrog_run", "paraexp_run", "fit_adjoint_grad"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1705_08019_gb300 import build, fitgb
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    fitgb.load()   # dlopen works without a GPU
    assert set(fitgb.EXPORTED) == set(declared_functions())
    assert fitgb.fit_version().startswith("fitgb")
    assert fitgb.strerror(fitgb.FIT_ERR_CFL) == "time step above the CFL estimate"


def test_product_path_does_not_import_oracle():
    """The CUDA path and its binding never touch the oracle."""
    pkg = os.path.join(ROOT, "paper_1705_08019_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "fit_oracle" not in text, f


def test_injected_allocation_failure_gives_oom():
    """The allocator hook fails the first device allocation of fit_grid_create
    before cudaMalloc is reached: FIT_ERR_OOM with no GPU involved, the grid
    handle stays null, and the hook is one-shot."""
    import ctypes
    import numpy as np
    from paper_1705_08019_gb300 import build, fitgb
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    build.build()
    lib = fitgb.load()
    eps = np.ones((4, 5, 6), np.float32)
    out = ctypes.c_void_p(0)
    # control: without the hook the call either succeeds (a GPU is present) or
    # fails in the CUDA runtime (FIT_ERR_CUDA: no device), never with OOM
    rc = lib.fit_grid_create(6, 5, 4, 1e-3, 1e-3, 1e-3, eps.ctypes.data_as(ctypes.c_void_p), None, None, 32, 0,
                             ctypes.byref(out))
    if rc == fitgb.FIT_OK:
        lib.fit_grid_destroy(out)
        out = ctypes.c_void_p(0)
    else:
        assert rc == fitgb.FIT_ERR_CUDA
    fitgb.fit_debug_fail_alloc(0)
    try:
        rc = lib.fit_grid_create(6, 5, 4, 1e-3, 1e-3, 1e-3, eps.ctypes.data_as(ctypes.c_void_p), None, None, 32, 0,
                                 ctypes.byref(out))
    finally:
        fitgb.fit_debug_fail_alloc(-1)
    assert rc == fitgb.FIT_ERR_OOM
    assert out.value is None
    assert fitgb.strerror(rc) == "device out of memory"



def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of fit_run_opts, fit_source, fit_probe and
    fit_run_stats have the C header's size and field offsets (gcc compiles the
    header and prints them)."""
    import ctypes
    import shutil
    from paper_1705_08019_gb300 import fitgb
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    structs = {"fit_run_opts": fitgb.fit_run_opts, "fit_source": fitgb.fit_source, "fit_probe": fitgb.fit_probe,
               "fit_run_stats": fitgb.fit_run_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fitgb.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append('return 0; }')
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True)
               .stdout.splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
