"""Symmetric tensors and their irreducible decomposition (oracle; test infrastructure only).

Everything here works on full 3^n arrays by explicit permutation sums, exactly as the
definitions read; it is slow and meant to be obviously correct.

* ``sym``: the symmetrisation operator of Sec. 2.2 (average over the r! index permutations).
* ``sprod``: the symmetric product AB = sym(A (x) B) (Eq. symm); ``delta_power(m)`` = delta^m.
* ``trace``: contraction of one index pair; ``trace_pow(A, m)`` applies it m times.
* ``B_coef`` / ``D_coef``: the constants of Eq. bd (Appendix A), as exact fractions.
* ``Q0`` and ``Qm``: the projection operators of Appendix A,
  Q^(n)_0 = sum_k D(n,k) delta^k tr^k and Q^(n)_m = B(n,m) Q^(n-2m)_0 tr^m, which give the
  traceless rank-(n-2m) tensors A^(n,m) of Eq. IrrDecomp, A^(n) = sum_m A^(n,m) delta^m.
* ``projector_matrices(n)``: the maps A^(n) -> A^(n,m) delta^m written as matrices on the
  multi-index components of order n (built once by applying the full-tensor operators to each
  basis tensor). They are what the oracle's collision uses.

Parity: pinned (Table 5 values of B and D; Table 1 rows; the projector identities
P_m P_m = P_m, P_m P_k = 0 for m != k, sum_m P_m = I; traceless outputs).
"""
from __future__ import annotations

import itertools
from fractions import Fraction
from functools import lru_cache
from math import factorial

import numpy as np

from .hermite import components, full_tensor, multi_indices


def sym(A: np.ndarray) -> np.ndarray:
    r = A.ndim
    if r < 2:
        return A.copy()
    acc = np.zeros_like(A)
    for p in itertools.permutations(range(r)):
        acc = acc + np.transpose(A, p)
    return acc / factorial(r)


def sprod(A, B) -> np.ndarray:
    """Symmetric product sym(A (x) B); a rank-0 factor multiplies."""
    A = np.asarray(A)
    B = np.asarray(B)
    if A.ndim == 0 or B.ndim == 0:
        return A * B
    return sym(np.multiply.outer(A, B))


def delta_power(m: int, dim: int = 3) -> np.ndarray:
    out = np.array(1.0)
    for _ in range(m):
        out = sprod(out, np.eye(dim))
    return out


def trace(A: np.ndarray) -> np.ndarray:
    return np.trace(A, axis1=0, axis2=1)


def trace_pow(A: np.ndarray, m: int) -> np.ndarray:
    for _ in range(m):
        A = trace(A)
    return A


def dfact(n: int) -> int:
    """n!! with (-1)!! = 0!! = 1."""
    out = 1
    while n > 1:
        out *= n
        n -= 2
    return out


def B_coef(n: int, m: int) -> Fraction:
    """Eq. bd: n! (2n-4m+1)!! / (m! 2^m (n-2m)! (2n-2m+1)!!)."""
    return Fraction(factorial(n) * dfact(2 * n - 4 * m + 1),
                    factorial(m) * 2 ** m * factorial(n - 2 * m) * dfact(2 * n - 2 * m + 1))


def D_coef(n: int, m: int) -> Fraction:
    """Eq. bd: (-1)^m n! (2n-2m-1)!! / (m! 2^m (n-2m)! (2n-1)!!)."""
    return Fraction((-1) ** m * factorial(n) * dfact(2 * n - 2 * m - 1),
                    factorial(m) * 2 ** m * factorial(n - 2 * m) * dfact(2 * n - 1))


def Q0(A: np.ndarray) -> np.ndarray:
    """Q^(n)_0 A = sum_k D(n,k) delta^k tr^k A  (traceless part of a rank-n tensor)."""
    n = A.ndim
    if n == 0:
        return A.copy()
    out = np.zeros_like(A)
    for k in range(n // 2 + 1):
        out = out + float(D_coef(n, k)) * sprod(delta_power(k), trace_pow(A, k))
    return out


def Qm(A: np.ndarray, m: int) -> np.ndarray:
    """A^(n,m) = Q^(n)_m A = B(n,m) Q^(n-2m)_0 tr^m A, a traceless rank-(n-2m) tensor."""
    n = A.ndim
    return float(B_coef(n, m)) * Q0(trace_pow(A, m))


def decompose(A: np.ndarray) -> list[np.ndarray]:
    """[A^(n,0), A^(n,1), ...] of Eq. IrrDecomp."""
    return [Qm(A, m) for m in range(A.ndim // 2 + 1)]


def reassemble(parts) -> np.ndarray:
    """sum_m A^(n,m) delta^m."""
    out = None
    for m, P in enumerate(parts):
        term = sprod(P, delta_power(m)) if m else P
        out = term if out is None else out + term
    return out


@lru_cache(maxsize=None)
def projector_matrices(n: int) -> tuple[np.ndarray, ...]:
    """P^(n)_m as matrices on the multi-index components of order n: A -> A^(n,m) delta^m."""
    idx = multi_indices(n)
    K = len(idx)
    mats = [np.zeros((K, K)) for _ in range(n // 2 + 1)]
    for j, alpha in enumerate(idx):
        basis = full_tensor({b: (1.0 if b == alpha else 0.0) for b in idx}, n)
        for m in range(n // 2 + 1):
            part = Qm(basis, m)
            lifted = sprod(part, delta_power(m)) if m else part
            comp = components(lifted)
            for i, beta in enumerate(idx):
                mats[m][i, j] = comp[beta]
    return tuple(mats)
