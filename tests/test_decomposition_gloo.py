"""Block decomposition with a halo exchange per right-hand side (Sec. 2.2: single-program
multiple-data over devices, each exchanging data with exactly one neighbour per permutation),
emulated with two gloo ranks on the CPU.

This test checks the decomposition on the oracle (the library's own blocks are checked in
test_gpu_decomposition.py and test_decomposition_host.py).  Two ranks hold z-slabs of a periodic
Taylor-Green box.  At
every right-hand side a rank fills its x and y halos locally, then receives its z halos from the
neighbouring rank: the three boundary layers over the whole x-y plane (halos included), which is
what the single-domain z pass reads.  The time step is the minimum over ranks of the local CFL
bounds.  After one RK3 step every slab equals the single-domain step bitwise."""
import copy
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

N = (10, 8, 12)          # interior cells (x, y, z); z is split over the ranks
WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _global():
    from oracle import ns_fv as nf
    from paper_2406_19494_gb300 import workloads as wl
    c = wl.tgv_case(8)
    c["n"] = N
    case = nf.Case(c)
    grid = nf.Grid(case)
    cen = [grid.axes[a].xc[case.h[a]:case.h[a] + case.n[a]] for a in range(3)]
    W = np.pad(wl.tgv_prims(c, *cen), [(0, 0)] + [(3, 3)] * 3, mode="edge")
    return c, case, grid, nf.prim_to_cons(W, case)


def _slab(c, case, grid, U, rank):
    """The rank's slab: interior z cells [rank nz, (rank + 1) nz) with h halo layers on each side,
    its case and grid (z metrics cut from the single-domain axis)."""
    from oracle import ns_fv as nf
    h, nz = case.h[2], case.n[2] // WORLD
    lc = dict(c, n=(N[0], N[1], nz), lo=(c["lo"][0], c["lo"][1], c["lo"][2] + rank * math.pi),
              hi=(c["hi"][0], c["hi"][1], c["lo"][2] + (rank + 1) * math.pi))
    lcase = nf.Case(lc)
    lgrid = nf.Grid(lcase)
    z0 = rank * nz                                      # padded z index of the slab's first layer
    lgrid.axes[2] = copy.copy(grid.axes[2])
    for name in ("xc", "dx", "mc", "mf"):
        setattr(lgrid.axes[2], name, getattr(grid.axes[2], name)[z0:z0 + nz + 2 * h])
    return lcase, lgrid, U[:, z0:z0 + nz + 2 * h].copy()


def _rank(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from oracle import ns_fv as nf
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    c, case, grid, U = _global()
    h, nz = case.h[2], case.n[2] // WORLD
    lcase, lgrid, U = _slab(c, case, grid, U, rank)
    lo_nb, hi_nb = (rank - 1) % WORLD, (rank + 1) % WORLD

    def exchange(V):
        # the lowest and highest h interior layers over the whole x-y plane go to the neighbours
        mine = torch.from_numpy(np.stack([V[:, h:2 * h], V[:, nz:nz + h]]).copy())
        got = [torch.empty_like(mine) for _ in range(WORLD)]
        dist.all_gather(got, mine)
        V[:, 0:h] = got[lo_nb][1].numpy()              # the lower neighbour's highest layers
        V[:, nz + h:nz + 2 * h] = got[hi_nb][0].numpy()  # the upper neighbour's lowest layers

    def L(V):
        nf.fill_halos(V, lcase, lgrid)                 # x and y passes (the z pass is replaced)
        exchange(V)
        return nf.rhs_filled(V, lcase, lgrid)

    dt = torch.tensor([nf.cfl_dt(U, lcase, lgrid)], dtype=torch.float64)
    dist.all_reduce(dt, op=dist.ReduceOp.MIN)
    U1 = nf.rk3(U, float(dt[0]), L, (slice(None),) + lcase.interior())
    out[rank] = (float(dt[0]), U1[(slice(None),) + lcase.interior()])
    dist.barrier()
    dist.destroy_process_group()


def test_two_slabs_equal_the_single_domain_step_bitwise():
    from oracle import ns_fv as nf
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(_free_port(), out), nprocs=WORLD, join=True, start_method="spawn")
        res = dict(out)
    c, case, grid, U = _global()
    dt = nf.cfl_dt(U, case, grid)
    ref = nf.rk3_step(U, dt, case, grid)[(slice(None),) + case.interior()]
    nz = case.n[2] // WORLD
    for r in range(WORLD):
        assert res[r][0] == dt
        assert np.array_equal(res[r][1], ref[:, r * nz:(r + 1) * nz]), r
    # the exchange is what makes them equal: a slab that wraps around on its own differs
    lcase, lgrid, Us = _slab(c, case, grid, U, 0)
    alone = nf.rk3_step(Us, dt, lcase, lgrid)[(slice(None),) + lcase.interior()]
    assert not np.array_equal(alone[:, 0], ref[:, 0])
