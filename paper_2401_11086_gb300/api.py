"""Python binding of libsmrt with the C ABI's names (include/smrt.h).

Argument marshalling only: PyTorch provides device memory and the CUDA stream; every step of
the method runs in libsmrt's kernels. Errors raise ``SmrtError`` carrying the lb_status.
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_int, c_int8, c_uint, c_void_p
from dataclasses import dataclass

import numpy as np

from . import _ffi
from ._ffi import (LB_F32, LB_F32_CONS64, LB_F64, LB_MOM_D, LB_MOM_Q, LB_MOM_RHO, LB_MOM_SIGMA,  # noqa: F401
                   LB_MODEL_ES_BGK, LB_MODEL_SMRT, LB_MOM_THETA, LB_MOM_U, LbGridDesc, LbLatticeDesc,
                   LbSchedule, LbState)

PRECISIONS = {"f64": LB_F64, "f32": LB_F32, "f32c64": LB_F32_CONS64}


class SmrtError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _ffi.lib().lb_error_string(status).decode()
        super().__init__(f"{where}: {msg} (lb_status {status})")
        self.status = status


def _check(status: int, where: str):
    if status != _ffi.LB_OK:
        raise SmrtError(status, where)


@dataclass
class LatticeDesc:
    """Velocity set: integer vectors e (q, 3), weights w (q,), scale c, degree, shift k."""
    e: np.ndarray
    w: np.ndarray
    c: float
    degree: int
    shift: tuple = (0, 0, 0)
    name: str = ""

    @property
    def q(self) -> int:
        return int(self.e.shape[0])


def lb_lattice_named(name: str) -> LatticeDesc:
    cap = 4913
    e = (c_int8 * (3 * cap))()
    w = (c_double * cap)()
    c, q, deg = c_double(), c_int(), c_int()
    _check(_ffi.lib().lb_lattice_named(name.encode(), e, w, byref(c), byref(q), byref(deg), cap),
           "lb_lattice_named")
    n = q.value
    return LatticeDesc(e=np.frombuffer(e, dtype=np.int8, count=3 * n).reshape(n, 3).copy(),
                       w=np.frombuffer(w, dtype=np.float64, count=n).copy(), c=c.value,
                       degree=deg.value, name=name)


def lb_rankine_hugoniot(Ma: float, gamma: float = 5.0 / 3.0, rho1: float = 1.0, theta1: float = 1.0):
    left, right = LbState(), LbState()
    _check(_ffi.lib().lb_rankine_hugoniot(Ma, gamma, rho1, theta1, byref(left), byref(right)),
           "lb_rankine_hugoniot")
    as_dict = lambda s: {"rho": s.rho, "u": (s.u[0], s.u[1], s.u[2]), "theta": s.theta}  # noqa: E731
    return as_dict(left), as_dict(right)


def lb_shock_frame(Ma: float, c: float, gamma: float = 5.0 / 3.0, theta2_max: float = 1.2):
    """(theta1, kx): reference temperature and frame shift of a normal shock."""
    t1, k = c_double(), c_int()
    _check(_ffi.lib().lb_shock_frame(Ma, gamma, c, theta2_max, byref(t1), byref(k)), "lb_shock_frame")
    return t1.value, k.value


def lb_shock_shift(Ma: float, c: float, theta1: float, gamma: float = 5.0 / 3.0) -> int:
    """kx: frame shift of a normal shock for a given upstream temperature."""
    k = c_int()
    _check(_ffi.lib().lb_shock_shift(Ma, gamma, c, theta1, byref(k)), "lb_shock_shift")
    return k.value


def lb_error_string(status: int) -> str:
    return _ffi.lib().lb_error_string(status).decode()


def _state(s) -> LbState:
    if s is None:
        return None
    u = s["u"] if isinstance(s, dict) else s[1]
    u = tuple(u) + (0.0,) * (3 - len(tuple(u)))
    rho = s["rho"] if isinstance(s, dict) else s[0]
    th = s["theta"] if isinstance(s, dict) else s[2]
    return LbState(float(rho), (c_double * 3)(*map(float, u)), float(th))


class Context:
    """An lb_ctx plus the Python objects it was made from."""

    def __init__(self, handle, lattice: LatticeDesc, N: int, precision: int, stream, device):
        self.handle = handle
        self.lattice = lattice
        self.N = N
        self.precision = precision
        self.stream = stream
        self.device = device
        lib = _ffi.lib()
        self.cells = int(lib.lb_cells(handle))
        self.plane_stride = int(lib.lb_plane_stride(handle))
        self.state_elems = int(lib.lb_state_elems(handle))

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == LB_F64 else torch.float32

    def new_state(self):
        import torch
        return torch.zeros(self.state_elems, dtype=self.dtype, device=self.device)

    def planes(self, f):
        """(q, cells) view of a state tensor (drops the alignment padding of each plane).
        A state stores deviations df_i = f_i - w_i (see include/smrt.h)."""
        return f.view(self.lattice.q, self.plane_stride)[:, : self.cells]

    @property
    def weights(self):
        """w_i in the caller's velocity order (add to a state's planes to get f_i)."""
        return np.asarray(self.lattice.w, dtype=np.float64)

    def close(self):
        if self.handle:
            _ffi.lib().lb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lb_init_lattice(lattice: LatticeDesc, nx: int, ny: int = 1, nz: int = 1, N: int = 3,
                    precision: str | int = "f32", bc_x: int = 0, nx_per_instance=None,
                    stream=None, device=None) -> Context:
    import torch
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    e = np.ascontiguousarray(lattice.e, dtype=np.int8)
    w = np.ascontiguousarray(lattice.w, dtype=np.float64)
    desc = LbLatticeDesc(int(lattice.q), e.ctypes.data_as(ctypes.POINTER(c_int8)),
                         w.ctypes.data_as(ctypes.POINTER(c_double)), float(lattice.c),
                         int(lattice.degree), (c_int * 3)(*map(int, lattice.shift)))
    if nx_per_instance is not None:
        lens = (c_int * len(nx_per_instance))(*map(int, nx_per_instance))
        grid = LbGridDesc(0, 1, 1, len(nx_per_instance), lens, bc_x)
    else:
        grid = LbGridDesc(nx, ny, nz, 1, None, bc_x)
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if stream is None:
        stream = torch.cuda.current_stream(device)
    h = c_void_p()
    _check(_ffi.lib().lb_init_lattice(byref(h), byref(desc), byref(grid), int(N), prec,
                                      c_void_p(stream.cuda_stream)), "lb_init_lattice")
    return Context(h, lattice, N, prec, stream, device)


def lb_set_relaxation(ctx: Context, tau, maxwell_molecule_law: bool = True, rho_ref: float = 1.0,
                      left=None, right=None, instance: int = -1):
    t = np.ascontiguousarray(tau, dtype=np.float64)
    ctx.relax_args = dict(maxwell_molecule_law=maxwell_molecule_law, rho_ref=rho_ref, left=left,
                          right=right, instance=instance)
    L, R = _state(left), _state(right)
    _check(_ffi.lib().lb_set_relaxation(ctx.handle, t.ctypes.data_as(ctypes.POINTER(c_double)),
                                        int(bool(maxwell_molecule_law)), float(rho_ref),
                                        byref(L) if L is not None else None,
                                        byref(R) if R is not None else None, int(instance)),
           "lb_set_relaxation")


def lb_set_frame_shift(ctx: Context, instance: int, kx: int):
    _check(_ffi.lib().lb_set_frame_shift(ctx.handle, int(instance), int(kx)), "lb_set_frame_shift")


def lb_hermite_convergence(theta, u, tol: float = 0.01, nmax: int = 99, stream=None):
    """Appendix B study on the GPU: (order int32, err float64) tensors for the points
    (theta[p], u[p]) given as float64 CUDA tensors of one shape."""
    import torch
    th = theta.contiguous().to(torch.float64)
    uu = u.contiguous().to(torch.float64)
    if th.shape != uu.shape or th.device.type != "cuda" or uu.device != th.device:
        raise ValueError("theta and u must be CUDA tensors of one shape")
    order = torch.empty(th.shape, dtype=torch.int32, device=th.device)
    err = torch.empty(th.shape, dtype=torch.float64, device=th.device)
    stream = torch.cuda.current_stream(th.device) if stream is None else stream
    _check(_ffi.lib().lb_hermite_convergence(c_void_p(th.data_ptr()), c_void_p(uu.data_ptr()), int(th.numel()),
                                             float(tol), int(nmax), c_void_p(order.data_ptr()),
                                             c_void_p(err.data_ptr()), c_void_p(stream.cuda_stream)),
           "lb_hermite_convergence")
    return order, err


def lb_set_collision_model(ctx: Context, instance: int, model: int, b: float = 0.0):
    _check(_ffi.lib().lb_set_collision_model(ctx.handle, int(instance), int(model), float(b)),
           "lb_set_collision_model")


def _ptr(t, dtype=None):
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return c_void_p(t.data_ptr())


def lb_fill_equilibrium(ctx: Context, f, rho, u, theta):
    import torch
    _check(_ffi.lib().lb_fill_equilibrium(ctx.handle, _ptr(f, ctx.dtype), _ptr(rho, torch.float64),
                                          _ptr(u, torch.float64), _ptr(theta, torch.float64)),
           "lb_fill_equilibrium")
    return f


def lb_step(ctx: Context, f_a, f_b, nsteps: int = 1):
    """Advance nsteps steps; returns whichever of f_a / f_b holds the newest state."""
    if f_a.numel() < ctx.state_elems or f_b.numel() < ctx.state_elems:
        raise ValueError("state tensors are smaller than lb_state_elems")
    _check(_ffi.lib().lb_step(ctx.handle, _ptr(f_a, ctx.dtype), _ptr(f_b, ctx.dtype), int(nsteps)), "lb_step")
    return f_b if nsteps % 2 == 1 else f_a


def lb_num_moment_rows(ctx: Context, mask: int) -> int:
    return int(_ffi.lib().lb_num_moment_rows(ctx.handle, c_uint(mask)))


def lb_moments(ctx: Context, f, mask: int = LB_MOM_RHO | LB_MOM_U | LB_MOM_THETA, out=None):
    import torch
    rows = lb_num_moment_rows(ctx, mask)
    if out is None:
        out = torch.empty((rows, ctx.cells), dtype=torch.float64, device=ctx.device)
    _check(_ffi.lib().lb_moments(ctx.handle, _ptr(f, ctx.dtype), _ptr(out, torch.float64), c_uint(mask)),
           "lb_moments")
    return out


def lb_step_adjoint(ctx: Context, f_t, lam_next, lam_t, dtau):
    """lam_t = adjoint of one step at forward state f_t applied to lam_next; dtau += gradient."""
    import torch
    _check(_ffi.lib().lb_step_adjoint(ctx.handle, _ptr(f_t, ctx.dtype), _ptr(lam_next, torch.float64),
                                      _ptr(lam_t, torch.float64), _ptr(dtau, torch.float64)),
           "lb_step_adjoint")
    return lam_t


def lb_moments_adjoint(ctx: Context, f, gbar, mask: int, lam):
    import torch
    _check(_ffi.lib().lb_moments_adjoint(ctx.handle, _ptr(f, ctx.dtype), _ptr(gbar, torch.float64),
                                         c_uint(mask), _ptr(lam, torch.float64)), "lb_moments_adjoint")
    return lam


def _sched_dict(s: LbSchedule) -> dict:
    return {"tile_width": s.tile_width, "blocks_per_sm": s.blocks_per_sm,
            "persistent": s.persistent, "tensor_cores": s.tensor_cores, "ms_per_step": s.ms_per_step}


def lb_set_schedule(ctx: Context, tile_width: int = 128, blocks_per_sm: int = 0, persistent: int = 0,
                    tensor_cores: int = 0):
    s = LbSchedule(int(tile_width), int(blocks_per_sm), int(persistent), int(tensor_cores), 0.0)
    _check(_ffi.lib().lb_set_schedule(ctx.handle, byref(s)), "lb_set_schedule")


def lb_get_schedule(ctx: Context) -> dict:
    s = LbSchedule()
    _check(_ffi.lib().lb_get_schedule(ctx.handle, byref(s)), "lb_get_schedule")
    return _sched_dict(s)


def lb_autotune(ctx: Context, f_a, f_b, trial_steps: int = 20) -> dict:
    """Time the candidate schedules on f_a/f_b (advanced in place), keep and return the best."""
    s = LbSchedule()
    _check(_ffi.lib().lb_autotune(ctx.handle, _ptr(f_a, ctx.dtype), _ptr(f_b, ctx.dtype), int(trial_steps),
                                  byref(s)), "lb_autotune")
    return _sched_dict(s)


def lb_step_graph(ctx: Context, f_a, f_b, nsteps: int):
    _check(_ffi.lib().lb_step_graph(ctx.handle, _ptr(f_a, ctx.dtype), _ptr(f_b, ctx.dtype), int(nsteps)),
           "lb_step_graph")
    return f_b if nsteps % 2 == 1 else f_a


def lb_test_barrier_timeout(ctx: Context, f_a, f_b):
    _check(_ffi.lib().lb_test_barrier_timeout(ctx.handle, _ptr(f_a, ctx.dtype), _ptr(f_b, ctx.dtype)),
           "lb_test_barrier_timeout")


def lb_poll_status(ctx: Context):
    flags = c_uint()
    st = _ffi.lib().lb_poll_status(ctx.handle, byref(flags))
    return st, flags.value


def lb_destroy(ctx: Context):
    ctx.close()
