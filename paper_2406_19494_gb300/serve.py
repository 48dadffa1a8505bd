"""Python binding of the serving loop (fluid_serve_* in include/fluid.h): argument marshalling.

The scheduler runs natively in the library; this wrapper keeps the host arrays of the requests
alive until their results have been polled.
"""
import ctypes

import numpy as np

from . import native


class Server:
    """Continuous-batching server for independent solves on one GPU."""

    def __init__(self, budget_bytes=150e9, max_active=16, chunk_steps=20, graphs=True, autotune=True,
                 device=0, batch=True):
        self.lib = native.lib()
        c = native.FluidServeConfig(struct_size=ctypes.sizeof(native.FluidServeConfig), device=device,
                                    max_active=max_active, chunk_steps=chunk_steps,
                                    use_graphs=1 if graphs else 0, autotune=1 if autotune else 0,
                                    hbm_budget_bytes=int(budget_bytes), batch=1 if batch else 0)
        h = ctypes.c_void_p()
        st = self.lib.fluid_serve_create(ctypes.byref(c), ctypes.byref(h))
        if st != native.FLUID_OK:
            raise native.FluidError(st, "fluid_serve_create failed")
        self.handle = h
        self._keep = {}

    def footprint(self, case, precision="fp64"):
        cfg = native.config_from_case(case, precision)
        return int(self.lib.fluid_serve_footprint(ctypes.byref(cfg)))

    def submit(self, case, U0, nsteps, precision="fp64", t_end=0.0):
        """Queue a solve from the padded initial state U0 (numpy float64); returns its ticket."""
        U0 = np.ascontiguousarray(U0, dtype=np.float64)
        out = np.empty_like(U0)
        req = native.FluidRequest(struct_size=ctypes.sizeof(native.FluidRequest), nsteps=int(nsteps),
                                  cfg=native.config_from_case(case, precision),
                                  U0_host=U0.ctypes.data, U_out_host=out.ctypes.data, t_end=float(t_end))
        t = ctypes.c_uint64()
        st = self.lib.fluid_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t))
        if st != native.FLUID_OK:
            raise native.FluidError(st, "fluid_serve_submit failed")
        self._keep[t.value] = out
        return t.value

    def poll(self, ticket, timeout_ms=0):
        """(result dict, final state) when ready; None on timeout."""
        r = native.FluidResult()
        st = self.lib.fluid_serve_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(r), int(timeout_ms))
        if st == native.FLUID_ETIMEOUT:
            return None
        if st != native.FLUID_OK:
            raise native.FluidError(st, "fluid_serve_poll failed")
        out = self._keep.pop(ticket)
        res = {k: getattr(r, k) for k, _ in native.FluidResult._fields_}
        return res, out

    def stats(self):
        s = native.FluidServeStats()
        self.lib.fluid_serve_stats(self.handle, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in native.FluidServeStats._fields_}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.fluid_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()
