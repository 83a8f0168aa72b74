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
