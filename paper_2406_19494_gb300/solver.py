"""Python binding of the C ABI: the same entry points, taking torch CUDA tensors.

Argument marshalling only -- every step of the computation runs in the CUDA kernels of
libfluid.so.  PyTorch supplies device memory and the current stream.
"""
import ctypes

import numpy as np
import torch

from . import native


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One solve on the current CUDA device, configured from a case dict (see workloads.py)."""

    def __init__(self, case, precision="fp64", adjoint=False):
        if not torch.cuda.is_available():
            raise RuntimeError("the fluid solver needs a CUDA device")
        self.lib = native.lib()
        self.case = case
        self.cfg = native.config_from_case(case, precision, adjoint)
        h = ctypes.c_void_p()
        st = self.lib.fluid_create(ctypes.byref(self.cfg), ctypes.byref(h))
        if st != native.FLUID_OK:
            raise native.FluidError(st, self.lib.fluid_last_error(None).decode())
        self.handle = h
        p = (ctypes.c_int32 * 3)()
        self.lib.fluid_padded_dims(self.handle, p)
        self.padded = (p[0], p[1], p[2])
        self.shape = (5, p[2], p[1], p[0])

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self.lib.fluid_destroy(h)
            self.handle = None

    def close(self):
        self.__del__()

    def _check(self, st):
        if st != native.FLUID_OK:
            raise native.FluidError(st, self.lib.fluid_last_error(self.handle).decode())

    def _state(self, U, name="U"):
        if not (isinstance(U, torch.Tensor) and U.is_cuda and U.dtype == torch.float64
                and U.is_contiguous() and tuple(U.shape) == self.shape):
            raise ValueError("%s must be a contiguous float64 CUDA tensor of shape %s" % (name, self.shape))
        return ctypes.c_void_p(U.data_ptr())

    # -- geometry ------------------------------------------------------------------------------
    def grid(self, axis):
        """(xc, dx) of axis over the padded range, as numpy arrays."""
        p = self.padded[axis]
        xc = np.zeros(p)
        dx = np.zeros(p)
        self._check(self.lib.fluid_get_grid(self.handle, axis, xc.ctypes.data_as(ctypes.c_void_p),
                                            dx.ctypes.data_as(ctypes.c_void_p)))
        return xc, dx

    def new_state(self):
        return torch.zeros(self.shape, dtype=torch.float64, device="cuda")

    # -- entry points --------------------------------------------------------------------------
    def prim_to_cons(self, W, U=None, stream=None):
        U = self.new_state() if U is None else U
        self._check(self.lib.fluid_prim_to_cons(self.handle, self._state(W, "W"), self._state(U),
                                                _stream(stream)))
        return U

    def rhs(self, U, R=None, stream=None):
        R = torch.zeros_like(U) if R is None else R
        self._check(self.lib.fluid_rhs(self.handle, self._state(U), self._state(R, "R"), _stream(stream)))
        return R

    def compute_dt(self, U, out=None, stream=None):
        out = torch.zeros(1, dtype=torch.float64, device="cuda") if out is None else out
        self._check(self.lib.fluid_compute_dt(self.handle, self._state(U), ctypes.c_void_p(out.data_ptr()),
                                              _stream(stream)))
        return out

    def step(self, U, nsteps=1, t_end=0.0, stream=None):
        self._check(self.lib.fluid_step(self.handle, self._state(U), int(nsteps), float(t_end),
                                        _stream(stream)))
        return U

    def rk3_stage(self, stage, Un, Us, Ud, dt, stream=None):
        """One RK3 stage with the given dt (fluid_rk3_stage); Ud may be Us or Un."""
        self._check(self.lib.fluid_rk3_stage(self.handle, int(stage), self._state(Un, "Un"),
                                             self._state(Us, "Us"), self._state(Ud, "Ud"),
                                             float(dt), _stream(stream)))
        return Ud

    def halo_count(self, axis):
        n = ctypes.c_size_t()
        self._check(self.lib.fluid_halo_count(self.handle, int(axis), ctypes.byref(n)))
        return n.value

    def pack_halo(self, U, axis, side, buf=None, stream=None):
        """The three interior layers of U next to face (axis, side) packed into buf (fluid_pack_halo)."""
        if buf is None:
            buf = torch.empty(self.halo_count(axis), dtype=torch.float64, device=U.device)
        elif buf.numel() != self.halo_count(axis):
            raise ValueError("halo buffer of axis %d must hold %d doubles" % (axis, self.halo_count(axis)))
        self._check(self.lib.fluid_pack_halo(self.handle, self._state(U), int(axis), int(side),
                                             _ptr(buf), _stream(stream)))
        return buf

    def unpack_halo(self, U, axis, side, buf, stream=None):
        """buf (a neighbour's packed layers) into the halo layers of U at face (axis, side)."""
        if buf.numel() != self.halo_count(axis):
            raise ValueError("halo buffer of axis %d must hold %d doubles" % (axis, self.halo_count(axis)))
        self._check(self.lib.fluid_unpack_halo(self.handle, self._state(U), int(axis), int(side),
                                               _ptr(buf), _stream(stream)))
        return U

    def step_stages(self, U, U1, U2, stream=None):
        self._check(self.lib.fluid_step_stages(self.handle, self._state(U), self._state(U1, "U1"),
                                               self._state(U2, "U2"), _stream(stream)))

    def adjoint_rhs(self, U, mu, gU=None, gphi=None, stream=None):
        gU = torch.zeros_like(U) if gU is None else gU
        self._check(self.lib.fluid_adjoint_rhs(self.handle, self._state(U), self._state(mu, "mu"),
                                               self._state(gU, "gU"), _ptr(gphi), _stream(stream)))
        return gU

    def adjoint_step(self, Un, lam, gphi=None, U1=None, U2=None, stream=None):
        self._check(self.lib.fluid_adjoint_step(
            self.handle, self._state(Un), None if U1 is None else self._state(U1, "U1"),
            None if U2 is None else self._state(U2, "U2"), self._state(lam, "lam"), _ptr(gphi),
            _stream(stream)))
        return lam

    def wall_heat_loss(self, U, axis, side, grad=False, stream=None):
        J = torch.zeros(1, dtype=torch.float64, device="cuda")
        dJ = torch.zeros_like(U) if grad else None
        self._check(self.lib.fluid_wall_heat_loss(self.handle, self._state(U), int(axis), int(side),
                                                  ctypes.c_void_p(J.data_ptr()), _ptr(dJ), _stream(stream)))
        return (J, dJ) if grad else J

    def wall_fluxes(self, U, axis, side, stream=None):
        """(q_w, tau_w) per wall cell of the isothermal or porous face (axis, side), shaped
        [n_t2, n_t1] (fluid_wall_fluxes)."""
        t1 = 1 if axis == 0 else 0
        t2 = 3 - axis - t1
        n = self.case["n"]
        qw = torch.zeros((n[t2], n[t1]), dtype=torch.float64, device="cuda")
        tw = torch.zeros_like(qw)
        self._check(self.lib.fluid_wall_fluxes(self.handle, self._state(U), int(axis), int(side),
                                               _ptr(qw), _ptr(tw), _stream(stream)))
        return qw, tw

    def time(self, stream=None):
        t, dt = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.fluid_get_time(self.handle, ctypes.byref(t), ctypes.byref(dt), _stream(stream)))
        return t.value, dt.value

    def set_time(self, t, stream=None):
        self._check(self.lib.fluid_set_time(self.handle, float(t), _stream(stream)))

    def check(self, stream=None):
        self._check(self.lib.fluid_check(self.handle, _stream(stream)))

    def tune_faces(self, block=0, seg=0):
        self._check(self.lib.fluid_tune_faces(self.handle, int(block), int(seg)))

    def autotune_faces(self, U, stream=None):
        """Time the FP64 face kernels' segment lengths on state U and keep the fastest per axis
        (fluid_autotune_faces); the result of every later call is unchanged."""
        self._check(self.lib.fluid_autotune_faces(self.handle, self._state(U), _stream(stream)))

    def profile(self, enable=True):
        self._check(self.lib.fluid_profile_enable(self.handle, 1 if enable else 0))

    def profile_read(self, reset=True):
        """{kernel class: (total ms, launches)} of the launches bracketed since the last reset."""
        out = {}
        for k, name in enumerate(native.KERNELS):
            ms, n = ctypes.c_double(), ctypes.c_int64()
            self._check(self.lib.fluid_profile_read(self.handle, k, ctypes.byref(ms), ctypes.byref(n), 0))
            out[name] = (ms.value, n.value)
        if reset:
            self._check(self.lib.fluid_profile_read(self.handle, 0, None, None, 1))
        return out

    def set_wall_params(self, phi, stream=None):
        if not (phi.is_cuda and phi.dtype == torch.float64 and phi.is_contiguous()):
            raise ValueError("phi must be a contiguous float64 CUDA tensor")
        self._check(self.lib.fluid_set_wall_params(self.handle, ctypes.c_void_p(phi.data_ptr()),
                                                   int(phi.numel()), _stream(stream)))

    def set_inflow(self, axis, side, W, stream=None):
        if not (W.is_cuda and W.dtype == torch.float64 and W.is_contiguous()):
            raise ValueError("W must be a contiguous float64 CUDA tensor")
        self._check(self.lib.fluid_set_inflow(self.handle, int(axis), int(side), ctypes.c_void_p(W.data_ptr()),
                                              int(W.numel()), _stream(stream)))
