"""The Appendix B convergence study on the GPU (lb_hermite_convergence) against the oracle.

The reported order is an integer decided by comparing a floating-point integral with the
tolerance: it must equal the oracle's except where the oracle's own error at either order sits
within 1e-6 (relative) of the tolerance; the errors agree to 1e-7 relative.
"""
import numpy as np
import pytest

from oracle import convergence as CV

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2401_11086_gb300 as P  # noqa: E402


def test_study_grid_matches_oracle():
    """The paper's axes (theta in [0.1, 2], u in [0, 4]) on a 10 x 9 grid, tol = 0.01, N <= 99."""
    th = np.linspace(0.1, 1.9, 10)
    uu = np.linspace(0.0, 4.0, 9)
    T, U = np.meshgrid(th, uu, indexing="ij")
    order, err = P.lb_hermite_convergence(torch.from_numpy(T.ravel()).cuda(), torch.from_numpy(U.ravel()).cuda())
    order, err = order.cpu().numpy(), err.cpu().numpy()
    for p, (t, u) in enumerate(zip(T.ravel(), U.ravel())):
        e = CV.errors(float(u), float(t), 99)
        n_or = int(np.nonzero(e < 0.01)[0][0]) if (e < 0.01).any() else 100
        if order[p] != n_or:
            lo = min(order[p], n_or)
            assert abs(e[lo] - 0.01) < 1e-6 * 0.01, (t, u, order[p], n_or)
        ref = e[min(order[p], 99)]
        assert abs(err[p] - ref) < 1e-7 * max(ref, 1e-3), (t, u, err[p], ref)


def test_edge_cases():
    """The exact case (order 0), the theta = 2 boundary (no convergence), an invalid point,
    an empty call and bad arguments."""
    t = torch.tensor([1.0, 2.0, -1.0], dtype=torch.float64, device="cuda")
    u = torch.tensor([0.0, 0.0, 0.5], dtype=torch.float64, device="cuda")
    order, err = P.lb_hermite_convergence(t, u, tol=0.01, nmax=60)
    assert order.tolist() == [0, 61, -1]
    assert err[0].item() < 1e-12 and err[1].item() >= 0.01 and np.isnan(err[2].item())
    e0 = torch.empty(0, dtype=torch.float64, device="cuda")
    assert P.lb_hermite_convergence(e0, e0)[0].numel() == 0
    with pytest.raises(P.SmrtError):
        P.lb_hermite_convergence(t, u, nmax=500)
