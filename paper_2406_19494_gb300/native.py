"""ctypes view of the C ABI in include/fluid.h (argument marshalling only).

The shared library is loaded from this package's _build/ directory.  There is no fallback: if the
library is missing or fails to load, every call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfluid.so")

FLUID_OK, FLUID_EINVAL, FLUID_ENOMEM, FLUID_ECUDA, FLUID_ENONFINITE = 0, 1, 2, 3, 4
FLUID_ETIMEOUT, FLUID_EBUSY, FLUID_EBUDGET, FLUID_ENOTSUP = 5, 6, 7, 8
STATUS_NAMES = {0: "FLUID_OK", 1: "FLUID_EINVAL", 2: "FLUID_ENOMEM", 3: "FLUID_ECUDA",
                4: "FLUID_ENONFINITE", 5: "FLUID_ETIMEOUT", 6: "FLUID_EBUSY", 7: "FLUID_EBUDGET",
                8: "FLUID_ENOTSUP"}

BC = {"periodic": 0, "zero_gradient": 1, "wall": 2, "adiabatic": 3, "porous": 4, "inflow": 5,
      "exchange": 6}
STRETCH = {"uniform": 0, "tanh2": 1, "tanh1": 2}
VISC = {"none": 0, "constant": 1, "power": 2, "sutherland": 3}
WENO = {"js": 0, "z": 1, "teno6a": 2}
PRECISION = {"fp64": 0, "mixed": 1}
KERNELS = ("prim_bc", "grad", "face_x", "face_y", "face_z", "stage", "dt", "source", "adj_face", "adj_cell")

# every symbol the header declares, with (restype, argtypes)
_vp, _i, _d, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
SIGNATURES = {
    "fluid_create": (_i, [_vp, ctypes.POINTER(_vp)]),
    "fluid_destroy": (None, [_vp]),
    "fluid_last_error": (ctypes.c_char_p, [_vp]),
    "fluid_padded_dims": (_i, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "fluid_get_grid": (_i, [_vp, _i, _vp, _vp]),
    "fluid_set_wall_params": (_i, [_vp, _vp, _i, _vp]),
    "fluid_set_inflow": (_i, [_vp, _i, _i, _vp, _sz, _vp]),
    "fluid_prim_to_cons": (_i, [_vp, _vp, _vp, _vp]),
    "fluid_rhs": (_i, [_vp, _vp, _vp, _vp]),
    "fluid_compute_dt": (_i, [_vp, _vp, _vp, _vp]),
    "fluid_step": (_i, [_vp, _vp, _i, _d, _vp]),
    "fluid_step_stages": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "fluid_adjoint_rhs": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "fluid_adjoint_step": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fluid_wall_heat_loss": (_i, [_vp, _vp, _i, _i, _vp, _vp, _vp]),
    "fluid_wall_fluxes": (_i, [_vp, _vp, _i, _i, _vp, _vp, _vp]),
    "fluid_halo_count": (_i, [_vp, _i, ctypes.POINTER(_sz)]),
    "fluid_pack_halo": (_i, [_vp, _vp, _i, _i, _vp, _vp]),
    "fluid_unpack_halo": (_i, [_vp, _vp, _i, _i, _vp, _vp]),
    "fluid_rk3_stage": (_i, [_vp, _i, _vp, _vp, _vp, _d, _vp]),
    "fluid_get_time": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(_d), _vp]),
    "fluid_set_time": (_i, [_vp, _d, _vp]),
    "fluid_check": (_i, [_vp, _vp]),
    "fluid_tune_faces": (_i, [_vp, _i, _i]),
    "fluid_autotune_faces": (_i, [_vp, _vp, _vp]),
    "fluid_profile_enable": (_i, [_vp, _i]),
    "fluid_profile_read": (_i, [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(ctypes.c_int64), _i]),
    "fluid_measure_peak": (_i, [_i, ctypes.POINTER(_d), _vp]),
    "fluid_rhs_noalloc": (_i, [_vp, _vp, _vp, _vp, ctypes.c_char_p, _sz]),
    "fluid_check_rcp": (_i, [_vp, _vp, _vp, _i, _vp]),
    "fluid_check_widen": (_i, [_vp, _vp, _vp, _i, _vp]),
    "fluid_check_bulk_staging": (_i, [_vp, _vp, _i, _i, _vp, _vp]),
    "fluid_check_sqrt": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "fluid_check_pow": (_i, [_vp, _vp, _vp, _i, _d, _vp]),
    "fluid_serve_create": (_i, [_vp, ctypes.POINTER(_vp)]),
    "fluid_serve_destroy": (None, [_vp]),
    "fluid_serve_submit": (_i, [_vp, _vp, ctypes.POINTER(ctypes.c_uint64)]),
    "fluid_serve_poll": (_i, [_vp, ctypes.c_uint64, _vp, _i]),
    "fluid_serve_stats": (_i, [_vp, _vp]),
    "fluid_serve_footprint": (_sz, [_vp]),
    "fluid_abi_version": (_i, []),
    "fluid_config_size": (_sz, []),
}


class FluidConfig(ctypes.Structure):
    """Mirror of struct fluid_config."""
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("ndim", ctypes.c_int32),
        ("n", ctypes.c_int32 * 3),
        ("stretch", ctypes.c_int32 * 3),
        ("bc", (ctypes.c_int32 * 2) * 3),
        ("visc_law", ctypes.c_int32),
        ("weno", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("porous_axis", ctypes.c_int32),
        ("porous_side", ctypes.c_int32),
        ("porous_begin", ctypes.c_int32),
        ("porous_count", ctypes.c_int32),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("beta", ctypes.c_double * 3),
        ("t_wall", (ctypes.c_double * 2) * 3),
        ("gamma", ctypes.c_double),
        ("gas_R", ctypes.c_double),
        ("prandtl", ctypes.c_double),
        ("mu_ref", ctypes.c_double),
        ("T_ref", ctypes.c_double),
        ("visc_exp", ctypes.c_double),
        ("suth_S", ctypes.c_double),
        ("weno_eps", ctypes.c_double),
        ("body_force", ctypes.c_double * 3),
        ("cfl", ctypes.c_double),
        ("dt_fixed", ctypes.c_double),
        ("porous_A", ctypes.c_double),
        ("porous_kappa", ctypes.c_double),
        ("porous_phi0", ctypes.c_double),
        ("adjoint", ctypes.c_int32),
        ("visc_order", ctypes.c_int32),
        ("global_n", ctypes.c_int32 * 3),
        ("offset", ctypes.c_int32 * 3),
    ]


class FluidServeConfig(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("device", ctypes.c_int32),
                ("max_active", ctypes.c_int32), ("chunk_steps", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_uint64), ("batch", ctypes.c_int32), ("pad", ctypes.c_int32)]


class FluidRequest(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("nsteps", ctypes.c_int32),
                ("cfg", FluidConfig), ("U0_host", ctypes.c_void_p), ("U_out_host", ctypes.c_void_p),
                ("t_end", ctypes.c_double)]


class FluidResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps_done", ctypes.c_int32), ("t_final", ctypes.c_double),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double), ("finish_s", ctypes.c_double)]


class FluidServeStats(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_int64), ("active", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("bytes_in_use", ctypes.c_uint64),
                ("peak_bytes", ctypes.c_uint64), ("cell_updates", ctypes.c_double),
                ("elapsed_s", ctypes.c_double)]


def config_from_case(case, precision="fp64", adjoint=False):
    """Fill a FluidConfig from a case dict (the schema of workloads.py)."""
    c = FluidConfig()
    c.struct_size = ctypes.sizeof(FluidConfig)
    c.ndim = int(case["ndim"])
    for a in range(3):
        c.n[a] = int(case["n"][a])
        c.stretch[a] = STRETCH[case.get("stretch", ("uniform",) * 3)[a]]
        c.lo[a] = float(case["lo"][a])
        c.hi[a] = float(case["hi"][a])
        c.beta[a] = float(case.get("beta", (0, 0, 0))[a])
        for s in range(2):
            c.bc[a][s] = BC[case["bc"][a][s]]
            c.t_wall[a][s] = float(case.get("t_wall", ((0, 0),) * 3)[a][s])
        c.body_force[a] = float(case.get("body_force", (0, 0, 0))[a])
    c.gamma = float(case["gamma"])
    c.gas_R = float(case["R"])
    c.prandtl = float(case.get("Pr", 0.72))
    c.visc_law = VISC[case.get("visc", "none")]
    c.mu_ref = float(case.get("mu_ref", 0.0))
    c.T_ref = float(case.get("T_ref", 1.0))
    c.visc_exp = float(case.get("visc_exp", 0.7))
    c.suth_S = float(case.get("suth_S", 0.0))
    c.weno = WENO[case.get("weno", "z")]
    eps = case.get("weno_eps", None)
    c.weno_eps = float(eps) if eps is not None else 0.0
    c.cfl = float(case.get("cfl", 0.5))
    c.dt_fixed = float(case.get("dt_fixed", 0.0))
    c.precision = PRECISION[precision]
    c.adjoint = 1 if adjoint else 0
    c.visc_order = int(case.get("visc_order", 4))
    for a in range(3):
        c.global_n[a] = int(case.get("global_n", (0, 0, 0))[a])
        c.offset[a] = int(case.get("offset", (0, 0, 0))[a])
    pz = case.get("porous", None)
    if pz:
        c.porous_axis, c.porous_side = int(pz["axis"]), int(pz["side"])
        c.porous_begin, c.porous_count = int(pz["begin"]), int(pz["count"])
        c.porous_A, c.porous_kappa, c.porous_phi0 = float(pz["A"]), float(pz["kappa"]), float(pz["phi0"])
    else:
        c.porous_axis = -1
    return c


_lib = None


def lib():
    """The loaded library (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfluid.so is not built (%s); run paper_2406_19494_gb300.build.build()"
                           % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    if L.fluid_config_size() != ctypes.sizeof(FluidConfig):
        raise RuntimeError("fluid_config layout mismatch between the library and the binding")
    _lib = L
    return L


class FluidError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status
