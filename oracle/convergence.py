"""Appendix B: convergence of the Hermite expansion of a 1D Maxwellian (oracle; test
infrastructure only).

The expansion (Appendix B, Eq. fexp) of f(xi) = exp(-(xi - u)^2 / (2 theta)) / sqrt(2 pi theta)
is f_N = omega(xi) sum_{n<=N} a^(n) He_n(xi) / n!, omega the unit Gaussian, with the closed
forms He_n(xi) = sum_k (-1)^k n! xi^(n-2k) / (2^k k! (n-2k)!) and
a^(n) = sum_k n! (theta - 1)^k u^(n-2k) / (2^k k! (n-2k)!). The study reports the smallest N
with int |f - f_N| dxi < tol (0.01 in the paper's figure).

Evaluation: a^(n) is summed exactly from the closed form in rational arithmetic (u and theta
are binary floats, hence exact rationals) and only then divided by sqrt(n!); He_n(xi) comes
from its three-term recurrence (the recurrence of the closed form, pinned in the tests) in
the normalised form phi_n = He_n(xi) exp(-xi^2/4) / sqrt(n!), which stays bounded for the
orders of the study (n <= 99 in the paper's contours), so that
  omega(xi) a^(n) He_n(xi) / n! = [exp(-xi^2/4) / sqrt(2 pi)] [a^(n) / sqrt(n!)] phi_n(xi).
The integral is composite Simpson on the grid of ``xi_grid``.

Parity: pinned (exact expansion at u = 0, theta = 1; coefficients against direct numerical
projection; the Simpson error against adaptive quadrature of the same integrand; no
convergence at theta = 2; symmetry in u).
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial, sqrt

import numpy as np

NXI = 4097          # Simpson points (odd)


def xi_grid(u: float, theta: float, nmax: int):
    """xi in [-L, L], L = max(|u| + 12 sqrt(theta), 2 sqrt(nmax + 1) + 10): the Maxwellian and
    every Hermite function up to order nmax are negligible beyond it."""
    L = max(abs(u) + 12.0 * sqrt(theta), 2.0 * sqrt(nmax + 1.0) + 10.0)
    xi = np.linspace(-L, L, NXI)
    h = 2.0 * L / (NXI - 1)
    w = np.full(NXI, 2.0)
    w[1::2] = 4.0
    w[0] = w[-1] = 1.0
    return xi, w * h / 3.0


def coefficient(n: int, u: float, theta: float) -> Fraction:
    """a^(n) of Appendix B, exactly."""
    U, T = Fraction(u), Fraction(theta)
    s = Fraction(0)
    for k in range(n // 2 + 1):
        s += Fraction(factorial(n), 2 ** k * factorial(k) * factorial(n - 2 * k)) * (T - 1) ** k * U ** (n - 2 * k)
    return s


def scaled_coefficients(u: float, theta: float, nmax: int) -> np.ndarray:
    """a^(n) / sqrt(n!), n = 0..nmax (sign kept, magnitude rounded once)."""
    out = np.empty(nmax + 1)
    for n in range(nmax + 1):
        a = coefficient(n, u, theta)
        mag = sqrt(float(a * a / factorial(n)))
        out[n] = mag if a >= 0 else -mag
    return out


def errors(u: float, theta: float, nmax: int) -> np.ndarray:
    """int |f - f_N| dxi for N = 0..nmax."""
    xi, w = xi_grid(u, theta, nmax)
    f = np.exp(-(xi - u) ** 2 / (2.0 * theta)) / np.sqrt(2.0 * np.pi * theta)
    env = np.exp(-xi ** 2 / 4.0) / np.sqrt(2.0 * np.pi)
    alpha = scaled_coefficients(u, theta, nmax)
    out = np.empty(nmax + 1)
    phi_prev, phi = np.zeros_like(xi), np.exp(-xi ** 2 / 4.0)          # phi_{-1}, phi_0
    fN = np.zeros_like(xi)
    for n in range(nmax + 1):
        fN = fN + env * alpha[n] * phi
        out[n] = np.sum(w * np.abs(f - fN))
        # He_{n+1} = xi He_n - n He_{n-1}, normalised by sqrt((n+1)!)
        phi_prev, phi = phi, (xi * phi - sqrt(n) * phi_prev) / sqrt(n + 1.0)
    return out


def min_order(u: float, theta: float, tol: float = 0.01, nmax: int = 99):
    """(smallest N with error < tol, that error), or (nmax + 1, error at nmax)."""
    e = errors(u, theta, nmax)
    hit = np.nonzero(e < tol)[0]
    if len(hit):
        return int(hit[0]), float(e[hit[0]])
    return nmax + 1, float(e[-1])
