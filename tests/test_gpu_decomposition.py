"""Block decomposition in the product (Section 2.2: the domain is split into blocks, one per device,
and every right-hand side first exchanges N_h = 3 halo layers with the neighbouring blocks).

Each case splits a solve into blocks that run as sub-domain solvers of the library
(FLUID_BC_EXCHANGE faces, global grid placement), with fluid_pack_halo / fluid_unpack_halo before
every RK3 stage and the CFL time step minimised over the blocks, and advances them with
fluid_rk3_stage.  After several steps every block's interior equals the single-domain fluid_step's
bitwise: the exchange reproduces exactly the halo values the single domain builds (including the
edges and corners that the dissipative cross-derivatives read between diagonal blocks), every face
flux depends only on its stencil, and the metrics are those of the global grid.

The first tests hold all blocks in one process (several solvers on one GPU, exchanged through
device buffers).  The last runs two processes on the GPU, each owning one block, exchanging through
host tensors over a gloo process group: the path a multi-GPU run takes with NCCL in place of gloo.
"""
import os
import socket

import numpy as np
import pytest

from helpers import padded_state
from paper_2406_19494_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = ("periodic", "periodic")
WALL = ("wall", "wall")
ZG = ("zero_gradient", "zero_gradient")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build
    build.build()


CASES = {
    # z-slabs of a periodic box (the Taylor-Green layout), two and three blocks
    "tgv_z2": (lambda: wl.tgv_case(16) | dict(n=(16, 12, 14)), (1, 1, 2), "fp64"),
    "periodic_z3_js": (lambda: wl.random_box(3, (12, 10, 15), weno="js", visc="constant"), (1, 1, 3), "fp64"),
    # y-slabs of a channel: isothermal walls on the outer blocks, tanh-stretched y, body force
    "channel_y2": (lambda: wl.random_box(3, (12, 20, 10), bc=(P, WALL, P),
                                         stretch=("uniform", "tanh2", "uniform"), beta=(0.0, 2.0, 0.0),
                                         body_force=(0.05, 0.0, 0.0), t_wall=((1, 1), (2.5, 2.2), (1, 1))),
                   (1, 2, 1), "fp64"),
    # 2 x 2 blocks in x and y: corners between diagonal blocks; walls on y, zero gradient on x
    "blocks_xy_walls": (lambda: wl.random_box(3, (14, 13, 8), bc=(ZG, WALL, P), visc="sutherland",
                                              stretch=("tanh1", "tanh2", "uniform"), beta=(1.2, 1.7, 0.0)),
                        (2, 2, 1), "fp64"),
    # 2 x 2 x 2 blocks of a periodic box
    "blocks_xyz": (lambda: wl.random_box(3, (12, 12, 12)), (2, 2, 2), "fp64"),
    # the mixed-precision path and the paper's channel scheme on slabs
    "mixed_z2": (lambda: wl.random_box(3, (16, 12, 18)), (1, 1, 2), "mixed"),
    "teno6a_visc6_y2": (lambda: wl.random_box(3, (12, 18, 10), bc=(P, WALL, P), weno="teno6a",
                                              visc_order=6, stretch=("uniform", "tanh2", "uniform"),
                                              beta=(0.0, 1.5, 0.0), t_wall=((1, 1), (1.4, 1.2), (1, 1))),
                        (1, 2, 1), "fp64"),
    # 2-D porous boundary layer split along the wall: the inflow block, the porous strip cut in two
    "porous_bl_x3": (lambda: wl.porous_bl_case(nx=36, ny=16, porous_count=14), (3, 1, 1), "fp64"),
}


def _setup(name):
    from paper_2406_19494_gb300.solver import Solver
    make, splits, prec = CASES[name]
    c = make()
    case, grid, U0 = _initial(c)
    extra = {}
    if c.get("porous"):
        extra["phi"] = wl.porous_phi(c, seed=1)
    for a in range(case.ndim):
        for s in range(2):
            if case.bc[a][s] == "inflow":
                extra[(a, s)] = wl.porous_bl_inflow(c, grid.axes[1].xc)
    glob = Solver(c, prec)
    _configure(glob, extra, None)
    return c, splits, prec, U0, glob, extra


def _initial(c):
    """Seeded random state; the boundary layer starts from its inflow profile (a random state of
    order one is far from the Ma 6 gas and would mirror to negative wall ghost temperatures)."""
    if c.get("porous"):
        from oracle import ns_fv as nf
        case = nf.Case(c)
        grid = nf.Grid(case)
        xc = grid.axes[0].xc[3:3 + case.n[0]]
        yc = grid.axes[1].xc[3:3 + case.n[1]]
        return padded_state(c, prims=wl.porous_bl_prims(c, xc, yc))
    return padded_state(c, seed=5)


def _configure(solver, extra, layout):
    for key, val in extra.items():
        if key == "phi":
            phi = val if layout is None else layout.phi_slice(val)
            if phi is not None:
                solver.set_wall_params(torch.tensor(np.ascontiguousarray(phi), device="cuda"))
        else:
            prof = val if layout is None else layout.inflow_slice(key[0], val)
            if solver.case["bc"][key[0]][key[1]] == "inflow":
                solver.set_inflow(key[0], key[1], torch.tensor(np.ascontiguousarray(prof), device="cuda"))


def _block_state(layout, U0):
    """The block's padded state cut from the global padded state (halos are refreshed anyway)."""
    nd = int(layout.case["ndim"])
    sl = [slice(None)]
    for a in (2, 1, 0):
        h = 3 if a < nd else 0
        sl.append(slice(layout.offset[a], layout.offset[a] + layout.n[a] + 2 * h))
    return torch.tensor(np.ascontiguousarray(U0[tuple(sl)]), device="cuda")


@pytest.mark.parametrize("name", sorted(CASES))
def test_blocks_equal_single_domain_bitwise(name):
    from paper_2406_19494_gb300 import decomp
    c, splits, prec, U0, glob, extra = _setup(name)
    nsteps = 3
    Ug = torch.tensor(U0, device="cuda")
    glob.step(Ug, nsteps)
    t_glob, _ = glob.time()

    hub = decomp.LocalComm()
    size = splits[0] * splits[1] * splits[2]
    blocks, Us = [], []
    for r in range(size):
        b = decomp.BlockSolver(c, splits, r, hub.endpoint(r), prec)
        _configure(b.solver, extra, b.layout)
        blocks.append(b)
        Us.append(_block_state(b.layout, U0))
    dts = decomp.run_local_blocks(blocks, Us, nsteps)
    torch.cuda.synchronize()
    t = 0.0
    for d in dts:                            # the solver's own order of additions (no compensation)
        t += d
    assert t == t_glob                       # the same dt every step: the same bits
    Ugh = Ug.cpu().numpy()
    for b, U in zip(blocks, Us):
        got = U.cpu().numpy()[(slice(None),) + b.layout.interior()]
        ref = Ugh[(slice(None),) + b.layout.interior_of_global()]
        assert np.array_equal(got, ref), (name, b.layout.rank, np.max(np.abs(got - ref)))


def test_sub_domain_rejections():
    """Entry points that run several right-hand sides in one call cannot refresh the exchange
    halos; the allocation-free entry point and the adjoint do not cover blocks."""
    from paper_2406_19494_gb300 import decomp, native
    from paper_2406_19494_gb300.solver import Solver
    c = wl.random_box(3, (12, 10, 12))
    lc = decomp.Layout(c, (1, 1, 2), 0).local_case()
    s = Solver(lc)
    U = s.new_state()
    with pytest.raises(native.FluidError, match="fluid_rk3_stage"):
        s.step(U, 1)
    with pytest.raises(native.FluidError):
        Solver(lc, adjoint=True)
    with pytest.raises(native.FluidError):
        s.rk3_stage(2, U, U, U, 0.0)
    with pytest.raises(native.FluidError):
        s.rk3_stage(1, U, s.new_state(), U, 0.1)
    import ctypes
    cfg = native.config_from_case(lc)
    err = ctypes.create_string_buffer(256)
    st = native.lib().fluid_rhs_noalloc(ctypes.byref(cfg), ctypes.c_void_p(U.data_ptr()),
                                        ctypes.c_void_p(s.new_state().data_ptr()), None, err, 256)
    assert st == native.FLUID_ENOTSUP, err.value
    bad = dict(lc, offset=(0, 0, 7))                      # block outside the global grid
    with pytest.raises(native.FluidError, match="inside the global grid"):
        Solver(bad)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, name, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2406_19494_gb300 import decomp
        make, splits, prec = CASES[name]
        c = make()
        _, _, U0 = _initial(c)
        b = decomp.BlockSolver(c, splits, rank, decomp.TorchComm(), prec)
        U = _block_state(b.layout, U0)
        b.step(U, 3)
        torch.cuda.synchronize()
        np.save(os.path.join(out_dir, "block%d.npy" % rank),
                U.cpu().numpy()[(slice(None),) + b.layout.interior()])
    finally:
        dist.destroy_process_group()


def test_two_processes_over_gloo_equal_single_domain(tmp_path):
    """Two ranks, one block each, both on GPU 0, halos through host tensors over gloo: the same
    bits as the single-domain step."""
    import torch.multiprocessing as mp
    from paper_2406_19494_gb300 import decomp
    name = "channel_y2"
    c, splits, prec, U0, glob, extra = _setup(name)
    Ug = torch.tensor(U0, device="cuda")
    glob.step(Ug, 3)
    ref = Ug.cpu().numpy()
    mp.spawn(_rank_main, args=(2, _free_port(), name, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        lay = decomp.Layout(c, splits, r)
        got = np.load(os.path.join(str(tmp_path), "block%d.npy" % r))
        assert np.array_equal(got, ref[(slice(None),) + lay.interior_of_global()])
