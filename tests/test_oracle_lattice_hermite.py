"""Pins of the oracle's velocity sets, Hermite polynomials and tensor projectors.

Every check here compares the oracle with something other than itself: brute-force quadrature
against Gaussian moments, the paper's printed Table 1/3/5 entries, or the Appendix B closed form.
"""
import itertools

import numpy as np
import pytest

from oracle import hermite as H
from oracle import lattice as L
from oracle import tensors as T
from _golden import frac, rows

LATTICES = ["D3Q39", "D3Q103", "D1Q9-P1", "D1Q17-P1"]


@pytest.fixture(scope="module")
def lattices():
    return {n: L.by_name(n) for n in LATTICES + ["D3Q729", "D3Q4913"]}


@pytest.mark.parametrize("name", LATTICES + ["D3Q729", "D3Q4913"])
def test_quadrature_exact_to_degree(lattices, name):
    """Sec. 3 (Eq. an): the set integrates every monomial of degree <= Q exactly."""
    lat = lattices[name]
    deg = lat.degree if name not in ("D3Q729", "D3Q4913") else 9  # 3D brute force capped for time
    tol = 1e-12 if name != "D1Q17-P1" else 1e-8      # xi^18 moments reach 3e7
    assert L.quadrature_error(lat, deg) < tol * max(1.0, 1.0)
    assert np.all(lat.w > 0)
    assert abs(lat.w.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("name", ["D3Q39", "D3Q103"])
def test_quadrature_fails_one_degree_higher(lattices, name):
    """The stated degree is sharp: some even monomial of degree Q+1 is not integrated."""
    lat = lattices[name]
    assert L.quadrature_error(lat, lat.degree + 1) > 1e-6


def test_paper_1d_scales_table3(lattices):
    """Table 3: c_l = 0.6780039 (d = 9, Q = 11) and 0.5638701 (d = 17, Q = 19)."""
    want = {(int(r[1]), int(r[2])): float(r[3]) for r in rows("table3_implementation.txt")}
    assert lattices["D1Q9-P1"].q == 9 and lattices["D1Q9-P1"].degree == 11
    assert abs(lattices["D1Q9-P1"].c - want[(9, 11)]) < 5e-8
    assert lattices["D1Q17-P1"].q == 17 and lattices["D1Q17-P1"].degree == 19
    assert abs(lattices["D1Q17-P1"].c - want[(17, 19)]) < 5e-8


def test_he_recurrence_matches_appendix_b_closed_form():
    x = np.linspace(-4, 4, 41)
    he = H.he_1d(9, x)
    for n in range(10):
        np.testing.assert_allclose(he[n], H.he_1d_closed(n, x), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("name", ["D3Q39", "D3Q103"])
def test_hermite_orthonormal_on_lattice(lattices, name):
    """sum_i w_i He_a(xi_i) He_b(xi_i) = a! delta_ab for |a| + |b| <= Q (Sec. 2.2, Eq. an)."""
    lat = lattices[name]
    top = lat.degree // 2 + 1
    al = H.multi_indices_upto(top)
    Hm = H.he_multi(al, lat.xi)
    G = (Hm * lat.w[:, None]).T @ Hm
    for i, a in enumerate(al):
        for j, b in enumerate(al):
            if sum(a) + sum(b) > lat.degree:
                continue
            want = H.alpha_factorial(a) if a == b else 0.0
            assert abs(G[i, j] - want) < 1e-11 * max(1.0, want), (a, b)


def _sp(*ts):
    out = np.array(1.0)
    for t in ts:
        out = T.sprod(out, t)
    return out


def test_table1_hermite_and_traceless_parts():
    """Table 1: H^(n) and its traceless parts H^(n,m), n = 2..4, pointwise at random xi."""
    rng = np.random.default_rng(3)
    d = np.eye(3)
    for _ in range(3):
        xi = rng.standard_normal(3)
        s = float(xi @ xi)
        x1, x2 = xi, np.multiply.outer(xi, xi)
        x3, x4 = _sp(xi, xi, xi), _sp(xi, xi, xi, xi)
        table = {
            2: (x2 - d, [x2 - s / 3 * d, (s - 3) / 3]),
            3: (x3 - 3 * _sp(x1, d), [x3 - 3 / 5 * s * _sp(x1, d), 3 / 5 * (s - 5) * x1]),
            4: (x4 - 6 * _sp(x2, d) + 3 * _sp(d, d),
                [x4 - 6 / 7 * s * _sp(x2, d) + 3 / 35 * s * s * _sp(d, d),
                 6 / 7 * (s - 7) * (x2 - s / 3 * d),
                 s * s / 5 - 2 * s + 3]),
        }
        for n, (Hn, parts) in table.items():
            Hfull = H.hermite_tensor(n, xi)
            np.testing.assert_allclose(Hfull, Hn, atol=1e-12)
            got = T.decompose(Hfull)
            for m, want in enumerate(parts):
                np.testing.assert_allclose(got[m], want, atol=1e-12)
                if np.ndim(got[m]) >= 2:
                    np.testing.assert_allclose(T.trace(got[m]), 0.0, atol=1e-12)
            np.testing.assert_allclose(T.reassemble(got), Hfull, atol=1e-12)


def test_table5_b_and_d():
    for n, m, b, dd in rows("table5_bd.txt"):
        assert T.B_coef(int(n), int(m)) == frac(b)
        assert T.D_coef(int(n), int(m)) == frac(dd)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_projector_identities(n):
    """Eq. IrrDecomp: the parts sum to the tensor, are traceless, and the split is a projection."""
    P = T.projector_matrices(n)
    K = P[0].shape[0]
    np.testing.assert_allclose(sum(P), np.eye(K), atol=1e-13)
    for i, Pi in enumerate(P):
        np.testing.assert_allclose(Pi @ Pi, Pi, atol=1e-13)
        for j, Pj in enumerate(P):
            if i != j:
                np.testing.assert_allclose(Pi @ Pj, 0.0, atol=1e-13)
    # rank of each part = number of independent components 2(n-2m)+1 of a traceless tensor
    for m, Pm in enumerate(P):
        assert np.linalg.matrix_rank(Pm, tol=1e-9) == 2 * (n - 2 * m) + 1


def test_table2_trace_relations():
    """Table 2 (linearised, u = 0, theta = 1): a^(3,1) = 6/5 q and a^(4,2) = tr^2 R/5 - 6p + 3 rho."""
    rng = np.random.default_rng(7)
    c = rng.standard_normal((200, 3))
    f = rng.random(200)
    c = c - (f @ c) / f.sum()                          # zero mean peculiar velocity
    rho = f.sum()
    P = np.einsum("s,si,sj->ij", f, c, c)
    Q3 = np.einsum("s,si,sj,sk->ijk", f, c, c, c)
    R = np.einsum("s,si,sj,sk,sl->ijkl", f, c, c, c, c)
    p = np.trace(P) / 3
    q = 0.5 * np.einsum("ikk->i", Q3)
    np.testing.assert_allclose(T.Qm(Q3, 1), 6 / 5 * q, rtol=1e-12)
    a4 = R - 6 * T.sprod(P, np.eye(3)) + 3 * rho * T.delta_power(2)
    np.testing.assert_allclose(T.Qm(a4, 2), T.trace_pow(R, 2) / 5 - 6 * p + 3 * rho, rtol=1e-12)
