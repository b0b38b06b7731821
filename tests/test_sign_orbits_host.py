"""The sign-orbit tables of the CUDA path's velocity sets (csrc/lattices.cuh), compiled as host
code, against the sets' integer vectors as the oracle states them. The projection and the
rebuild of the D3Q39 / D3Q103 kernels sum per orbit: for a member v = s (.) a of an orbit (v the
pair's +e or -e, positive on the orbit's first nonzero axis), v^gamma = a^gamma (-1)^popcount(b & c)
with b the member's sign bits and c the slot's transform entry. Checked here for every member
and every slot up to order 4, together with the labelling itself. Runs on the CPU (nvcc needed)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import lattice as OL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "orbits_host.cu")
OUT = os.path.join(ROOT, "paper_2401_11086_gb300", "_build", "orbits_host_test.so")


@pytest.fixture(scope="module")
def host():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    deps = [SRC] + [os.path.join(ROOT, "paper_2401_11086_gb300", "csrc", n) for n in ("core.cuh", "lattices.cuh")]
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < max(os.path.getmtime(d) for d in deps):
        subprocess.run([nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-shared",
                        "-Xcompiler", "-fPIC", SRC, "-o", OUT], check=True)
    return ctypes.CDLL(OUT)


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


@pytest.mark.parametrize("name,N", [("D3Q39", 3), ("D3Q103", 4)])
def test_sign_orbits_label_every_pair_and_factor_every_monomial(host, name, N):
    tag = name.lower()
    e = np.zeros((60, 3), dtype=np.int32)
    npairs = getattr(host, f"vectors_{tag}")(_ip(e))
    e = e[:npairs].astype(int)
    # the compile-time pairs are the oracle's velocity set, each +-e once
    olat = OL.by_name(name)
    want = {tuple(int(x) for x in v) for v in olat.e}
    got = {(0, 0, 0)} | {tuple(v) for v in e} | {tuple(-v) for v in e}
    assert got == want and 2 * npairs + 1 == olat.q

    tab = np.zeros(15 * npairs, dtype=np.int32)
    norb = getattr(host, f"orbits_{tag}")(_ip(tab))
    tab = tab[:15 * norb].reshape(norb, 15)
    M = (N + 1) * (N + 2) * (N + 3) // 6
    mono = np.zeros(norb * M, dtype=np.int32)
    cls = np.zeros(norb * M, dtype=np.int32)
    getattr(host, f"classes_{tag}")(N, _ip(mono), _ip(cls))
    mono, cls = mono.reshape(norb, M), cls.reshape(norb, M)
    comp = np.zeros(3 * M, dtype=np.int32)
    host.slot_components(N, _ip(comp))
    comp = comp.reshape(M, 3)
    # slots: every multi-index of order <= N once, ordered by order
    assert sorted(map(tuple, comp)) == sorted((i, j, n - i - j) for n in range(N + 1)
                                               for i in range(n + 1) for j in range(n + 1 - i))
    assert list(comp.sum(1)) == sorted(comp.sum(1))

    seen = []
    for o in range(norb):
        k, ax, a = tab[o, 0], tab[o, 1:4], tab[o, 4:7]
        pairs, flips = tab[o, 7:11], tab[o, 11:15]
        axes = [d for d in range(3) if a[d] != 0]
        assert k == len(axes) and list(ax[:k]) == axes
        for b in range(1 << (k - 1)):
            p = int(pairs[b])
            seen.append(p)
            v = -e[p] if flips[b] else e[p]
            assert list(np.abs(v)) == list(a) and v[ax[0]] > 0
            bits = sum(1 << (t - 1) for t in range(1, k) if v[ax[t]] < 0)
            assert bits == b
            for g in range(M):
                direct = int(np.prod([int(v[d]) ** int(comp[g, d]) for d in range(3)]))
                sign = -1 if bin(b & int(cls[o, g])).count("1") % 2 else 1
                assert direct == mono[o, g] * sign, (o, b, g)
    assert sorted(seen) == list(range(npairs))
