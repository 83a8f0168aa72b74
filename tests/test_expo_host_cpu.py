"""Host logic of the exponential propagators through the C ABI (no GPU):
the library's planner and real Newton coefficients (fit_expo_plan,
fit_expo_coeffs) against the oracle's, which takes the divided differences
from their recursive definition at high precision (Sec. III-B, III-D)."""
import numpy as np
import pytest

from oracle import expo


@pytest.fixture(scope="module")
def fitgb():
    from paper_1705_08019_gb300 import build, fitgb
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    build.build()
    fitgb.load()
    return fitgb


@pytest.mark.parametrize("kind,u,tol,prec", [
    ("leja", 0.95, 1e-12, 64), ("leja", 0.5, 1e-8, 64), ("leja", 0.95, 1e-6, 32), ("leja", 0.95, 1e-2, 64),
    ("taylor", 0.95, 1e-12, 64), ("taylor", 0.95, 1e-6, 32),
])
def test_plan_equals_oracle(fitgb, kind, u, tol, prec):
    assert fitgb.fit_expo_plan(kind, u, tol, prec) == expo.plan(kind, u, tol, prec)


@pytest.mark.parametrize("kind,m,a", [("leja", 40, 10.0), ("leja", 96, 31.35), ("leja", 20, 0.3),
                                      ("taylor", 30, 4.0)])
def test_pair_coefficients_equal_oracle(fitgb, kind, m, a):
    al, ga, et = fitgb.fit_expo_coeffs(kind, m, a)
    xi = expo.nodes(kind, m)
    d = expo.divided_differences(xi, a)
    J = m // 2
    eta = np.array([xi[2 * j - 1].imag for j in range(1, J + 1)])
    oal = np.array([(d[2 * j - 1] - 1j * eta[j - 1] * d[2 * j]).real for j in range(1, J + 1)])
    oga = np.array([d[2 * j].real for j in range(1, J + 1)])
    scale = max(1.0, np.abs(oal).max(), np.abs(oga).max())
    assert np.abs(al - oal).max() <= 1e-13 * scale
    assert np.abs(ga - oga).max() <= 1e-13 * scale
    assert np.array_equal(et, eta ** 2)
    # the imaginary parts the real form drops are zero (conjugate points)
    assert max(abs((d[2 * j - 1] - 1j * eta[j - 1] * d[2 * j]).imag) for j in range(1, J + 1)) <= 1e-13 * scale


def test_real_pair_form_equals_newton_form(fitgb):
    """p(z) = 1 + sum_j R_{j-1}(z)(alpha_j + gamma_j z), R_0 = z,
    R_j = (z^2 + eta_j^2) R_{j-1}, is the Newton interpolant of exp(a z):
    it matches exp at the Leja points."""
    m, a = 60, 12.0
    al, ga, et = fitgb.fit_expo_coeffs("leja", m, a)
    for z in expo.nodes("leja", m):
        R, p = z, 1.0 + 0j
        for j in range(m // 2):
            p += R * (al[j] + ga[j] * z)
            R = (z * z + et[j]) * R
        assert abs(p - np.exp(a * z)) <= 1e-11


def test_bad_arguments_are_rejected(fitgb):
    FitError = fitgb.FitError
    with pytest.raises(FitError):
        fitgb.fit_expo_plan("leja", 0.95, 1e-30, 64)          # below what FP64 can reach
    with pytest.raises(FitError):
        fitgb.fit_expo_plan("leapfrog", 0.95, 1e-8, 64)
    with pytest.raises(FitError):
        fitgb.fit_expo_coeffs("leja", 7, 1.0)                # odd degree
