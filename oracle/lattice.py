"""Velocity sets as Gauss-Hermite quadratures (oracle; test infrastructure only).

A velocity set is a list of integer vectors e_i, weights w_i and a scale c, with abscissae
xi_i = c e_i. It is a degree-Q Gauss-Hermite rule when sum_i w_i p(xi_i) equals the integral of
p against the unit Gaussian omega(xi) for every polynomial p of degree <= Q (Sec. 3, Eq. an and
the remark after Eq. fi that exactness needs degree >= 2N).

The weights and c are found here by solving those moment conditions directly (scipy least
squares on all unknowns at once) and every set is then checked by brute force over all
monomials of degree <= Q (``quadrature_error``).

Sets provided:

* ``d1q9_p1`` / ``d1q17_p1``: the paper's 1D rules (Table 3: degree 11 with c_l = 0.6780039,
  degree 19 with c_l = 0.5638701). The paper prints only d, Q and c_l; the abscissae
  c*{0,+-1,+-2,+-3,+-5} and c*{0,+-1..+-7,+-9} are the reading under which the printed c_l is
  the root of the moment conditions (pinned in the tests).
* ``d3q729``: tensor product of D1Q9-P1 (Sec. 4.2, "three-dimensional tensor products").
* ``d3q39``: degree 7, shells (0,0,0) (1,0,0) (1,1,1) (2,0,0) (2,2,0) (3,0,0).
* ``d3q103``: degree 9, shells (1,1,1) (2,0,0) (2,1,1) (2,2,0) (2,2,2) (3,0,0) (4,0,0)
  (3,3,3) (4,2,0) plus rest. Neither 3D set is in the paper; both are cubic-symmetric
  Gauss-Hermite rules solved from the same moment conditions.

Parity: pinned (brute-force quadrature; paper's printed c_l for the 1D rules).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np
from scipy.optimize import least_squares


def gaussian_moment(alpha) -> float:
    """Integral of xi^alpha against the unit Gaussian: prod_k (alpha_k - 1)!!, 0 if any odd."""
    out = 1.0
    for a in alpha:
        if a % 2:
            return 0.0
        out *= float(np.prod(np.arange(a - 1, 0, -2))) if a > 0 else 1.0
    return out


def signed_permutations(v) -> list[tuple[int, ...]]:
    """All distinct vectors obtained from v by permuting components and flipping signs."""
    out = set()
    for p in itertools.permutations(v):
        for s in itertools.product((1, -1), repeat=len(v)):
            out.add(tuple(int(a * b) for a, b in zip(p, s)))
    return sorted(out)


@dataclass
class Lattice:
    name: str
    e: np.ndarray            # (Q, D) integer velocity vectors
    w: np.ndarray            # (Q,) weights
    c: float                 # lattice scale, xi_i = c e_i
    degree: int              # quadrature degree
    shells: list = field(default_factory=list)

    @property
    def q(self) -> int:
        return self.e.shape[0]

    @property
    def xi(self) -> np.ndarray:
        return self.c * self.e.astype(np.float64)


def quadrature_error(lat: Lattice, degree: int | None = None) -> float:
    """Largest |sum_i w_i xi_i^alpha - E[xi^alpha]| over all multi-indices |alpha| <= degree."""
    degree = lat.degree if degree is None else degree
    xi = lat.xi
    dim = xi.shape[1]
    worst = 0.0
    for total in range(degree + 1):
        for alpha in itertools.product(range(total + 1), repeat=dim):
            if sum(alpha) != total:
                continue
            mono = np.prod(xi ** np.array(alpha), axis=1)
            val = float(np.sum(lat.w * mono))
            worst = max(worst, abs(val - gaussian_moment(alpha)))
    return worst


def _even_conditions(degree: int, dim: int):
    """Distinct even exponent patterns a >= b >= ... (all even) with sum <= degree."""
    conds = []
    for total in range(0, degree + 1, 2):
        for alpha in itertools.product(range(0, total + 1, 2), repeat=dim):
            if sum(alpha) == total and list(alpha) == sorted(alpha, reverse=True):
                conds.append(alpha)
    return conds


def _solve_shells(shells, degree: int, c0: float, dim: int):
    """Solve shell weights W_s and scale c from the even moment conditions.

    Every member of a shell carries the shell's weight; odd moments vanish by the shells'
    sign symmetry, so only the even patterns of ``_even_conditions`` remain.
    """
    members = [np.array(signed_permutations(s), dtype=np.float64) for s in shells]
    conds = _even_conditions(degree, dim)
    target = np.array([gaussian_moment(a) for a in conds])

    def design(c):
        A = np.empty((len(conds), len(shells)))
        for j, mem in enumerate(members):
            for r, a in enumerate(conds):
                A[r, j] = np.sum(np.prod((c * mem) ** np.array(a), axis=1))
        return A

    W0, *_ = np.linalg.lstsq(design(c0), target, rcond=None)

    def resid(x):
        return (design(x[-1]) @ x[:-1] - target) / np.maximum(target, 1.0)

    sol = least_squares(resid, np.concatenate([W0, [c0]]), xtol=1e-15, ftol=1e-15, gtol=1e-15)
    W, c = sol.x[:-1], float(sol.x[-1])
    return members, W, c


def _from_shells(name, shells, degree, c0, dim=3) -> Lattice:
    members, W, c = _solve_shells(shells, degree, c0, dim)
    e = np.concatenate([m for m in members]).astype(np.int64)
    w = np.concatenate([np.full(len(m), W[j]) for j, m in enumerate(members)])
    return Lattice(name=name, e=e, w=w, c=c, degree=degree, shells=list(shells))


def d1q9_p1() -> Lattice:
    """Degree-11 1D rule on c*{0,+-1,+-2,+-3,+-5} (Table 3, d = 9, Q = 11)."""
    return _from_shells("D1Q9-P1", [(0,), (1,), (2,), (3,), (5,)], 11, 0.678, dim=1)


def d1q17_p1() -> Lattice:
    """Degree-19 1D rule on c*{0,+-1..+-7,+-9} (Table 3, d = 17, Q = 19)."""
    shells = [(0,)] + [(k,) for k in range(1, 8)] + [(9,)]
    return _from_shells("D1Q17-P1", shells, 19, 0.5639, dim=1)


def tensor_product3(l1: Lattice, name: str) -> Lattice:
    """3D tensor product of a 1D rule (Sec. 4.2): e = (a, b, c), w = w_a w_b w_c."""
    idx = list(itertools.product(range(l1.q), repeat=3))
    e = np.array([[l1.e[i, 0], l1.e[j, 0], l1.e[k, 0]] for i, j, k in idx], dtype=np.int64)
    w = np.array([l1.w[i] * l1.w[j] * l1.w[k] for i, j, k in idx])
    return Lattice(name=name, e=e, w=w, c=l1.c, degree=l1.degree)


def d3q729() -> Lattice:
    return tensor_product3(d1q9_p1(), "D3Q729")


def d3q4913() -> Lattice:
    """Tensor product of D1Q17-P1 (Sec. 4.2: the Ma = 7 runs, d = 17, degree 19)."""
    return tensor_product3(d1q17_p1(), "D3Q4913")


D3Q39_SHELLS = [(0, 0, 0), (1, 0, 0), (1, 1, 1), (2, 0, 0), (2, 2, 0), (3, 0, 0)]
D3Q103_SHELLS = [(0, 0, 0), (1, 1, 1), (2, 0, 0), (2, 1, 1), (2, 2, 0), (2, 2, 2),
                 (3, 0, 0), (4, 0, 0), (3, 3, 3), (4, 2, 0)]


def d3q39() -> Lattice:
    return _from_shells("D3Q39", D3Q39_SHELLS, 7, 1.2)


def d3q103() -> Lattice:
    return _from_shells("D3Q103", D3Q103_SHELLS, 9, 0.736)


def by_name(name: str) -> Lattice:
    return {"D3Q39": d3q39, "D3Q103": d3q103, "D3Q729": d3q729, "D3Q4913": d3q4913,
            "D1Q9-P1": d1q9_p1, "D1Q17-P1": d1q17_p1}[name]()
