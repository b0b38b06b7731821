"""lb_step_adjoint_noalloc -- the adjoint step for callers that cannot allocate device memory
(stream capture, pool-owned memory, fixed budgets) -- called through the C ABI twice in a row
and compared with lb_step_adjoint on the same inputs. Collected last on purpose: it shares a
process-wide device array with every other call of this entry point."""
import ctypes

import numpy as np
import pytest

import synthetic
from oracle import lattice as OL
from oracle import shock as OK
from _lb import lib_from_oracle, upload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2401_11086_gb300 as P  # noqa: E402
from paper_2401_11086_gb300 import _ffi  # noqa: E402


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_adjoint_matches_allocating_entry_point():
    olat = OL.d3q103()
    d = P.lb_lattice_named("D3Q103")
    idx = lib_from_oracle(olat, d)
    nx = 300
    case = OK.shock_case(olat, 4, 2.0, nx)
    st = case.states
    h0 = OK.initial_state(case, *[synthetic.tanh_blend(nx, 6.0, st[k + "1"], st[k + "2"])
                                  for k in ("rho", "u", "theta")])
    left, right = P.lb_rankine_hugoniot(2.0, theta1=case.theta1)
    ctx = P.lb_init_lattice(P.LatticeDesc(d.e, d.w, d.c, d.degree, (case.k, 0, 0)), nx, N=4,
                            precision="f64", bc_x=1)
    taus = [case.model.tau_star[k] * case.model.tau_ref for k in
            [(2, 0), (2, 1), (3, 0), (3, 1), (4, 0), (4, 1), (4, 2)]]
    P.lb_set_relaxation(ctx, taus, True, 1.0, left, right)
    lib = _ffi.lib()
    rng = np.random.default_rng(5)
    for call in range(2):                       # two calls in a row, different inputs
        h = h0 * (1 + 0.02 * rng.standard_normal(h0.shape))
        f = upload(ctx, h, idx)
        lam_next = torch.from_numpy(rng.standard_normal(ctx.state_elems)).cuda()
        ref_lam = torch.zeros_like(lam_next)
        ref_dtau = torch.zeros(len(taus), dtype=torch.float64, device="cuda")
        assert lib.lb_step_adjoint(ctx.handle, _vp(f), _vp(lam_next), _vp(ref_lam), _vp(ref_dtau)) == 0
        got_lam = torch.full_like(lam_next, np.nan)
        got_dtau = torch.zeros(len(taus), dtype=torch.float64, device="cuda")
        assert lib.lb_step_adjoint_noalloc(ctx.handle, _vp(f), _vp(lam_next), _vp(got_lam), _vp(got_dtau)) == 0
        torch.cuda.synchronize()
        planes = lambda t: t.view(ctx.lattice.q, ctx.plane_stride)[:, : ctx.cells]  # noqa: E731
        np.testing.assert_allclose(planes(got_lam).cpu().numpy(), planes(ref_lam).cpu().numpy(),
                                   rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(got_dtau.cpu().numpy(), ref_dtau.cpu().numpy(), rtol=1e-12, atol=0)
    assert P.lb_poll_status(ctx)[0] == 0
    ctx.close()


def test_noalloc_adjoint_rejects_grids_beyond_its_array():
    """A line context scheduled at 32-cell tiles with more tiles (8438) than the fixed array has
    slots (8192) is refused with LB_ERR_INVALID before any launch: lam_t and dtau keep their
    contents. At 128-cell tiles (2110 tiles) the same context is accepted."""
    d = P.lb_lattice_named("D3Q39")
    nx = 270000
    ctx = P.lb_init_lattice(P.LatticeDesc(d.e, d.w, d.c, d.degree, (1, 0, 0)), nx, N=3, precision="f64",
                            bc_x=1)
    left, right = P.lb_rankine_hugoniot(1.2, theta1=1.0)
    P.lb_set_relaxation(ctx, [2.4, 2.4, 1.6, 3.6], True, 1.0, left, right)
    lib = _ffi.lib()
    f = ctx.new_state()
    lam_next = torch.ones(ctx.state_elems, dtype=torch.float64, device="cuda")
    lam_t = torch.full_like(lam_next, 7.0)
    dtau = torch.full((4,), 3.0, dtype=torch.float64, device="cuda")
    P.lb_set_schedule(ctx, 32, 0, 0)
    assert lib.lb_step_adjoint_noalloc(ctx.handle, _vp(f), _vp(lam_next), _vp(lam_t), _vp(dtau)) == 1
    torch.cuda.synchronize()
    assert bool((lam_t == 7.0).all()) and bool((dtau == 3.0).all())
    P.lb_set_schedule(ctx, 128, 0, 0)
    assert lib.lb_step_adjoint_noalloc(ctx.handle, _vp(f), _vp(lam_next), _vp(lam_t), _vp(dtau)) == 0
    torch.cuda.synchronize()
    assert P.lb_poll_status(ctx)[0] == 0
    ctx.close()
