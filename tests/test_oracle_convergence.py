"""Pins of the Appendix B convergence study in the oracle (oracle/convergence.py)."""
from math import factorial

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermeval

from oracle import convergence as CV

integrate = pytest.importorskip("scipy.integrate")


def _maxwellian(x, u, th):
    return np.exp(-(x - u) ** 2 / (2 * th)) / np.sqrt(2 * np.pi * th)


def test_exact_for_the_weight_itself():
    """Appendix B: at u = 0, theta = 1 the weight is the Maxwellian and f_0 is exact."""
    n, err = CV.min_order(0.0, 1.0)
    assert n == 0 and err < 1e-12


@pytest.mark.parametrize("u,th", [(0.7, 0.6), (1.3, 1.4)])
def test_coefficients_equal_direct_projection(u, th):
    """a^(n) = int f He_n dxi (numerical quadrature, no closed form)."""
    for n in range(13):
        c = [0] * n + [1]
        want, _ = integrate.quad(lambda x: _maxwellian(x, u, th) * hermeval(x, c), -40, 40, limit=400,
                                 epsabs=1e-13, epsrel=1e-12)
        assert abs(float(CV.coefficient(n, u, th)) - want) < 1e-9 * max(1.0, abs(want))


@pytest.mark.parametrize("u,th,N", [(1.0, 0.8, 4), (2.0, 1.5, 9), (0.5, 0.3, 7)])
def test_simpson_error_matches_adaptive_quadrature(u, th, N):
    """The study's L1 error against adaptive quadrature of |f - f_N| with f_N summed by numpy's
    own Hermite series from the exact coefficients. |f - f_N| has kinks where it changes sign,
    at which composite Simpson is only second order: agreement to 5e-5 relative."""
    coef = [float(CV.coefficient(n, u, th)) / factorial(n) for n in range(N + 1)]
    g = lambda x: abs(_maxwellian(x, u, th) - np.exp(-x * x / 2) / np.sqrt(2 * np.pi) * hermeval(x, coef))  # noqa: E731
    pts = np.linspace(-30, 30, 61)
    want = sum(integrate.quad(g, a, b, limit=200, epsabs=1e-14)[0] for a, b in zip(pts[:-1], pts[1:]))
    got = CV.errors(u, th, N)[N]
    assert abs(got - want) < 5e-5 * max(0.1, want)


def test_no_convergence_at_theta_two():
    """Appendix B: theta = 2 is the convergence boundary; u = 0 does not reach 1 % by N = 99."""
    n, err = CV.min_order(0.0, 2.0)
    assert n == 100 and err >= 0.01


def test_symmetric_in_u():
    np.testing.assert_allclose(CV.errors(1.7, 0.9, 30), CV.errors(-1.7, 0.9, 30), rtol=1e-12, atol=1e-15)


def test_trends_stated_in_appendix_b():
    """Convergence slows as u moves away from 0 and as theta nears the boundary 2."""
    nu = [CV.min_order(u, 1.0)[0] for u in (0.5, 1.5, 2.5, 3.5)]
    assert nu == sorted(nu) and nu[0] < nu[-1]
    nt = [CV.min_order(0.0, th)[0] for th in (1.2, 1.5, 1.8, 1.9)]
    assert nt == sorted(nt) and nt[0] < nt[-1]
