"""Hermite polynomials in multi-index and full-tensor form (oracle; test infrastructure only).

* 1D probabilists' Hermite polynomials He_n by the three-term recurrence
  He_{n+1}(x) = x He_n(x) - n He_{n-1}(x); their explicit sum is the closed form of Appendix B
  (Eq. fexp's H^(n)), which the tests compare against.
* The rank-n tensor Hermite polynomial H^(n)(xi) of Sec. 2.2 (the polynomials orthogonal under
  omega(xi), Eq. hermite) has the component H^(n)_{i1..in} = prod_k He_{alpha_k}(xi_k), where
  alpha_k counts how many of i1..in equal k. A symmetric rank-n tensor is therefore stored by
  its (n+1)(n+2)/2 distinct components, one per multi-index alpha with |alpha| = n
  (``multi_indices``), or in full as a 3^n array (``full_tensor``).
* The contraction A^(n):H^(n)/n! of Eq. hermite1 in multi-index form is
  sum_{|alpha|=n} A_alpha He_alpha / alpha!, alpha! = prod_k alpha_k!.

Parity: pinned (recurrence vs Appendix B closed form; Table 1 entries; orthonormality on the
velocity sets by brute-force quadrature).
"""
from __future__ import annotations

import itertools
from math import factorial

import numpy as np


def multi_indices(n: int, dim: int = 3) -> list[tuple[int, ...]]:
    """Multi-indices alpha with |alpha| = n, in descending lexicographic order."""
    out = [a for a in itertools.product(range(n, -1, -1), repeat=dim) if sum(a) == n]
    return out


def multi_indices_upto(N: int, dim: int = 3) -> list[tuple[int, ...]]:
    out = []
    for n in range(N + 1):
        out += multi_indices(n, dim)
    return out


def alpha_factorial(alpha) -> int:
    out = 1
    for a in alpha:
        out *= factorial(a)
    return out


def he_1d(nmax: int, x):
    """He_0..He_nmax at x (array); returns a list of arrays, by the three-term recurrence."""
    x = np.asarray(x)
    out = [np.ones_like(x), x.copy()]
    for n in range(1, nmax):
        out.append(x * out[n] - n * out[n - 1])
    return out[: nmax + 1]


def he_1d_closed(n: int, x):
    """Appendix B closed form: sum_k (-1)^k n! x^(n-2k) / (2^k k! (n-2k)!)."""
    x = np.asarray(x, dtype=np.result_type(x, np.float64))
    s = np.zeros_like(x)
    for k in range(n // 2 + 1):
        s = s + (-1) ** k * factorial(n) * x ** (n - 2 * k) / (2 ** k * factorial(k) * factorial(n - 2 * k))
    return s


def he_multi(alphas, xi):
    """He_alpha(xi) for each alpha in ``alphas``; xi has shape (..., 3). Returns (..., len)."""
    xi = np.asarray(xi)
    nmax = max(max(a) for a in alphas)
    per_axis = [he_1d(nmax, xi[..., k]) for k in range(xi.shape[-1])]
    cols = []
    for a in alphas:
        v = per_axis[0][a[0]]
        for k in range(1, len(a)):
            v = v * per_axis[k][a[k]]
        cols.append(v)
    return np.stack(cols, axis=-1)


def full_tensor(comp: dict, n: int, dim: int = 3) -> np.ndarray:
    """Expand multi-index components {alpha: value} of a symmetric rank-n tensor to 3^n."""
    sample = next(iter(comp.values())) if comp else 0.0
    T = np.zeros((dim,) * n, dtype=np.result_type(np.asarray(sample), np.float64))
    for idx in itertools.product(range(dim), repeat=n):
        alpha = tuple(idx.count(k) for k in range(dim))
        T[idx] = comp[alpha]
    return T


def components(T: np.ndarray, dim: int = 3) -> dict:
    """Read the multi-index components of a (symmetric) full tensor at representative indices."""
    n = T.ndim
    out = {}
    for alpha in multi_indices(n, dim):
        idx = tuple(k for k in range(dim) for _ in range(alpha[k]))
        out[alpha] = T[idx] if n else T[()]
    return out


def hermite_tensor(n: int, xi) -> np.ndarray:
    """Full rank-n tensor H^(n)(xi) at a single point xi (length 3)."""
    vals = he_multi(multi_indices(n), np.asarray(xi)[None, :])[0]
    return full_tensor(dict(zip(multi_indices(n), vals)), n)
