"""CPU checks of the C ABI: the library builds, loads, exports every symbol include/fluid.h
declares, agrees with the binding on struct layout, and rejects bad configurations before touching
the GPU."""
import ctypes
import os
import re

import pytest

from conftest import ROOT
from paper_2406_19494_gb300 import build as B
from paper_2406_19494_gb300 import native
from paper_2406_19494_gb300 import workloads as wl


@pytest.fixture(scope="module")
def lib():
    B.build()
    return native.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fluid.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fluid_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree_on_symbols():
    assert declared_symbols() == sorted(native.SIGNATURES)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_config_layout(lib):
    assert lib.fluid_abi_version() == 1
    assert lib.fluid_config_size() == ctypes.sizeof(native.FluidConfig)


def _create(lib, cfg):
    h = ctypes.c_void_p()
    st = lib.fluid_create(ctypes.byref(cfg), ctypes.byref(h))
    return st, lib.fluid_last_error(None).decode()


@pytest.mark.parametrize("mutate,needle", [
    (lambda c: setattr(c, "ndim", 4), "ndim"),
    (lambda c: c.n.__setitem__(0, 2), "3 <= n"),
    (lambda c: c.n.__setitem__(0, 0), "3 <= n"),
    (lambda c: c.n.__setitem__(2, 5), "inactive"),
    (lambda c: c.bc[0].__setitem__(1, native.BC["wall"]), "periodic boundaries must pair"),
    (lambda c: setattr(c, "gamma", 1.0), "gamma"),
    (lambda c: setattr(c, "struct_size", 8), "struct_size"),
    (lambda c: setattr(c, "precision", 7), "precision"),
    (lambda c: setattr(c, "weno", 9), "reconstruction"),
    (lambda c: setattr(c, "visc_order", 5), "visc_order"),
    (lambda c: (setattr(c, "weno", 2), setattr(c, "precision", 1)), "FP64 only"),
    (lambda c: (setattr(c, "visc_order", 6), setattr(c, "adjoint", 1)), "adjoint"),
    (lambda c: (setattr(c, "cfl", 0.0), setattr(c, "dt_fixed", 0.0)), "cfl"),
    (lambda c: c.n.__setitem__(0, (1 << 20) + 1), "3 <= n"),
    (lambda c: (c.n.__setitem__(0, 20000), c.n.__setitem__(1, 20000)), "32-bit"),
    (lambda c: (c.n.__setitem__(0, 14000), c.n.__setitem__(1, 14000), setattr(c, "precision", 1)), "mixed path"),
    (lambda c: (c.n.__setitem__(0, 8000), c.n.__setitem__(1, 8000), setattr(c, "adjoint", 1)), "adjoint (36"),
    (lambda c: c.global_n.__setitem__(0, 4), "inside the global grid"),
    (lambda c: (c.global_n.__setitem__(0, 20), c.offset.__setitem__(0, 13)), "inside the global grid"),
    (lambda c: c.offset.__setitem__(1, 2), "offset needs global_n"),
    (lambda c: c.global_n.__setitem__(2, 1), "inactive axes cannot be split"),
    (lambda c: (c.bc[0].__setitem__(0, native.BC["exchange"]), c.bc[0].__setitem__(1, native.BC["exchange"]),
                setattr(c, "adjoint", 1)), "exchange"),
    (lambda c: c.bc[1].__setitem__(0, 7), "unknown boundary kind"),
])
def test_invalid_configs_are_rejected_before_any_gpu_call(lib, mutate, needle):
    cfg = native.config_from_case(wl.random_box(2, (8, 8, 1)))
    mutate(cfg)
    st, msg = _create(lib, cfg)
    assert st == native.FLUID_EINVAL and needle in msg, (st, msg)


def test_porous_strip_must_fit(lib):
    c = wl.porous_bl_case(nx=16, ny=8)
    c["porous"] = dict(c["porous"], begin=10, count=10)
    st, msg = _create(lib, native.config_from_case(c))
    assert st == native.FLUID_EINVAL and "porous" in msg


def test_null_out_pointer(lib):
    cfg = native.config_from_case(wl.sod_case(16))
    assert lib.fluid_create(ctypes.byref(cfg), None) == native.FLUID_EINVAL


def test_serve_config_rejected_before_any_gpu_call(lib):
    c = native.FluidServeConfig(struct_size=4, device=0, max_active=1, chunk_steps=1, use_graphs=1,
                                autotune=0, hbm_budget_bytes=1 << 30)
    h = ctypes.c_void_p()
    assert lib.fluid_serve_create(ctypes.byref(c), ctypes.byref(h)) == native.FLUID_EINVAL
    c.struct_size = ctypes.sizeof(native.FluidServeConfig)
    c.max_active = 0
    assert lib.fluid_serve_create(ctypes.byref(c), ctypes.byref(h)) == native.FLUID_EINVAL


def test_serve_footprint_grows_with_the_grid(lib):
    small = native.config_from_case(wl.tgv_case(32))
    big = native.config_from_case(wl.tgv_case(64))
    fs, fb = lib.fluid_serve_footprint(ctypes.byref(small)), lib.fluid_serve_footprint(ctypes.byref(big))
    assert 0 < fs < fb and fb > 8 * 38 ** 3 * 30


def test_product_path_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: without the built library the binding raises instead of computing."""
    monkeypatch.setattr(native, "LIB_PATH", str(tmp_path / "missing" / "libfluid.so"))
    monkeypatch.setattr(native, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        native.lib()


def test_solver_needs_a_cuda_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2406_19494_gb300.solver import Solver
    with pytest.raises(RuntimeError, match="CUDA device"):
        Solver(wl.random_box(2, (8, 8, 1)))
