"""The CUDA path's per-cell adjoint arithmetic (csrc/adjoint.cuh), compiled as host code,
against the oracle's complex-step vector-Jacobian products. Runs on the CPU (nvcc needed)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import adjoint as OA
from oracle import hermite as OH
from oracle import lattice as OL
from oracle import smrt as OS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "adjoint_host.cu")
OUT = os.path.join(ROOT, "paper_2401_11086_gb300", "_build", "adjoint_host_test.so")


@pytest.fixture(scope="module")
def host():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    deps = [SRC] + [os.path.join(ROOT, "paper_2401_11086_gb300", "csrc", n)
                    for n in ("adjoint.cuh", "core.cuh", "lattices.cuh")]
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < max(os.path.getmtime(d) for d in deps):
        subprocess.run([nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-shared",
                        "-Xcompiler", "-fPIC", SRC, "-o", OUT], check=True)
    lib = ctypes.CDLL(OUT)
    P = ctypes.POINTER(ctypes.c_double)
    for n in ("collide_vjp_d3q39_n3", "collide_vjp_d3q103_n4"):
        getattr(lib, n).argtypes = [P, P, ctypes.c_double, P, P, P, ctypes.c_double, ctypes.c_double, P, P]
    for n in ("moments_vjp_d3q39_n3", "moments_vjp_d3q103_n4"):
        getattr(lib, n).argtypes = [P, ctypes.c_double, P, P]
    return lib


def _ptr(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lib_order(olat):
    import paper_2401_11086_gb300 as P
    from _lb import lib_from_oracle
    d = P.lb_lattice_named(olat.name)
    return d, lib_from_oracle(olat, d)


CASES = [("D3Q39", 3, "collide_vjp_d3q39_n3", "moments_vjp_d3q39_n3"),
         ("D3Q103", 4, "collide_vjp_d3q103_n4", "moments_vjp_d3q103_n4")]


@pytest.mark.parametrize("name,N,cfn,mfn", CASES)
@pytest.mark.parametrize("maxwell", [True, False])
def test_collide_vjp_matches_oracle(host, name, N, cfn, mfn, maxwell):
    olat = OL.by_name(name)
    d, idx = _lib_order(olat)
    rng = np.random.default_rng(3)
    ncell = 3
    rho, u, th = 1 + 0.2 * rng.random(ncell), 0.3 * rng.standard_normal((3, ncell)), 0.8 + 0.4 * rng.random(ncell)
    f = OS.equilibrium(rho, u, th, olat, N) * (1 + 0.05 * rng.standard_normal((olat.q, ncell)))
    lam = rng.standard_normal(f.shape)
    model = OS.Model(olat, N, tau_ref=1.0, maxwell_law=maxwell, rho_ref=1.3)
    taus = OA.model_taus(model) * (1 + 0.2 * rng.random(len(OA.tau_keys(N))))
    fbar, gtau = OA.collide_vjp(f, lam, model, taus)
    tauA = taus * model.rho_ref if maxwell else np.zeros_like(taus)
    tauB = np.full_like(taus, 0.5) if maxwell else taus + 0.5
    dA, dB = (model.rho_ref, 0.0) if maxwell else (0.0, 1.0)
    wp = np.concatenate([[d.w[0]], d.w[1::2]])
    gsum = np.zeros(len(taus))
    for cidx in range(ncell):
        fl = f[idx, cidx] - d.w
        ll = lam[idx, cidx]
        fb = np.zeros(olat.q)
        tb = np.zeros(len(taus))
        getattr(host, cfn)(_ptr(fl), _ptr(ll), d.c, _ptr(wp), _ptr(tauA), _ptr(tauB), dA, dB,
                           fb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           tb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        want = fbar[idx, cidx]
        assert np.abs(fb - want).max() < 1e-11 * max(1.0, np.abs(want).max()), cidx
        gsum += tb
    np.testing.assert_allclose(gsum, gtau, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("name,N,cfn,mfn", CASES)
def test_moments_vjp_matches_oracle(host, name, N, cfn, mfn):
    olat = OL.by_name(name)
    d, idx = _lib_order(olat)
    rng = np.random.default_rng(4)
    rho, u, th = np.array([1.1]), np.array([[0.3], [-0.1], [0.2]]), np.array([0.9])
    f = (OS.equilibrium(rho, u, th, olat, N) * (1 + 0.05 * rng.standard_normal((olat.q, 1))))[:, 0]
    bar = rng.standard_normal(8)
    Nd = max(N, 3)
    al = OH.multi_indices_upto(Nd)
    pos = {a: k for k, a in enumerate(al)}

    def moments(fc):
        r, uu, t = OS.conserved(fc[:, None], olat)
        dd = OS.local_direct(fc[:, None], olat, Nd, uu, t)
        q = [0.5 * t ** 1.5 * sum(dd[pos[tuple(np.eye(3, dtype=int)[k] + 2 * np.eye(3, dtype=int)[l])]]
                                   for l in range(3)) for k in range(3)]
        return np.concatenate([r, uu[:, 0], t, np.array([qq[0] for qq in q])])

    want = np.zeros(olat.q)
    for k in range(olat.q):
        fc = f.astype(np.complex128)
        fc[k] += 1e-30j
        want[k] = np.sum(bar * moments(fc).imag) / 1e-30
    fb = np.zeros(olat.q)
    getattr(host, mfn)(_ptr(f[idx] - d.w), d.c, _ptr(bar), fb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    got = np.empty_like(fb)
    got[idx] = fb
    assert np.abs(got - want).max() < 1e-11 * max(1.0, np.abs(want).max())
