"""CPU checks of the block decomposition's host logic (paper_2406_19494_gb300/decomp.py): block
placement, neighbours, the configuration of a block, and the halo-exchange schedule over gloo ranks.

The exchange test runs decomp.exchange itself on gloo ranks (world sizes 2 and 4) with stand-ins
for the library's pack / unpack that follow the buffer layout include/fluid.h documents
([5][layer][t2][t1], the other axes over the padded range below the exchange axis and the interior
range above it).  Each rank starts with its interior cells of one global field and garbage in its
halos; after the exchange every cell that is interior or an exchange halo on every axis holds the
global field's value there, corners between diagonal blocks included."""
import os
import socket

import numpy as np
import pytest

from paper_2406_19494_gb300 import decomp
from paper_2406_19494_gb300 import workloads as wl

torch = pytest.importorskip("torch")

P = ("periodic", "periodic")
WALL = ("wall", "wall")


def test_block_ranges_tile_the_axis():
    for n, parts in ((12, 2), (13, 3), (128, 8), (7, 2)):
        got = [decomp.block_range(n, parts, k) for k in range(parts)]
        assert got[0][0] == 0 and sum(c for _, c in got) == n
        for (o0, c0), (o1, _) in zip(got, got[1:]):
            assert o1 == o0 + c0
        assert max(c for _, c in got) - min(c for _, c in got) <= 1


def test_neighbours_and_block_configuration():
    c = wl.random_box(3, (12, 20, 10), bc=(P, WALL, P), stretch=("uniform", "tanh2", "uniform"),
                      beta=(0.0, 2.0, 0.0))
    lays = [decomp.Layout(c, (2, 2, 1), r) for r in range(4)]
    # x periodic with two blocks: both x faces face the other x block
    assert [l.neighbour(0, 0) for l in lays] == [1, 0, 3, 2]
    assert [l.neighbour(0, 1) for l in lays] == [1, 0, 3, 2]
    # y walls: the outer faces keep the wall, the shared face is an exchange face
    assert [l.neighbour(1, 0) for l in lays] == [None, None, 0, 1]
    assert [l.neighbour(1, 1) for l in lays] == [2, 3, None, None]
    assert all(l.neighbour(2, s) is None for l in lays for s in (0, 1))
    lc = lays[2].local_case()
    assert lc["bc"] == (("exchange", "exchange"), ("exchange", "wall"), P)
    assert lc["n"] == (6, 10, 10) and lc["global_n"] == (12, 20, 0) and lc["offset"] == (0, 10, 0)


def test_porous_strip_and_inflow_are_cut_per_block():
    c = wl.porous_bl_case(nx=36, ny=16, porous_count=14)          # strip on cells 11 .. 24
    lays = [decomp.Layout(c, (3, 1, 1), r) for r in range(3)]
    cases = [l.local_case() for l in lays]
    assert [lc["bc"][0] for lc in cases] == [("inflow", "exchange"), ("exchange", "exchange"),
                                             ("exchange", "zero_gradient")]
    # each block's strip covers its wall cells and the neighbours' wall cells in its exchange
    # halos (3 on each exchange side): global cells 11..14, 11..24 and 21..24
    assert [(lc["porous"]["begin"], lc["porous"]["count"]) for lc in cases] == [(11, 4), (-1, 14), (-3, 4)]
    phi = np.arange(14.0)
    assert [l.phi_slice(phi).tolist() for l in lays] == [phi[0:4].tolist(), phi.tolist(), phi[10:14].tolist()]
    c2 = dict(c, porous=dict(c["porous"], begin=2, count=6))          # strip inside block 0 only
    l1 = decomp.Layout(c2, (3, 1, 1), 1)
    assert l1.local_case()["bc"][1] == ("wall", "zero_gradient") and l1.local_case()["porous"] is None
    prof = np.random.default_rng(0).uniform(size=(5, 1, 22))
    assert np.array_equal(lays[0].inflow_slice(0, prof), prof)


def test_layout_rejects_thin_blocks():
    with pytest.raises(ValueError):
        decomp.Layout(wl.random_box(3, (8, 8, 5)), (1, 1, 2), 0)


# ---------------------------------------------------------------------------------------------
# the exchange schedule on gloo ranks
# ---------------------------------------------------------------------------------------------
def _shape(lay):
    nd = int(lay.case["ndim"])
    return (5,) + tuple(lay.n[a] + (6 if a < nd else 0) for a in (2, 1, 0))


def _sel(lay, a, layers):
    """Index tuple of the buffer region of axis a: `layers` along a, padded below, interior above."""
    nd = int(lay.case["ndim"])
    sl = [slice(None)] * 4
    for b in range(3):
        h = 3 if b < nd else 0
        if b == a:
            sl[3 - b] = layers
        elif b < a:
            sl[3 - b] = slice(None)
        else:
            sl[3 - b] = slice(h, h + lay.n[b])
    return tuple(sl)


def _pack(lay):
    def pack(U, a, side):
        n = lay.n[a]
        layers = slice(3, 6) if side == 0 else slice(n, n + 3)
        return U[_sel(lay, a, layers)].contiguous().reshape(-1)
    return pack


def _unpack(lay):
    def unpack(U, a, side, buf):
        n = lay.n[a]
        layers = slice(0, 3) if side == 0 else slice(n + 3, n + 6)
        region = U[_sel(lay, a, layers)]
        U[_sel(lay, a, layers)] = buf.reshape(region.shape)
    return unpack


def _global_value(case, idx):
    """A field whose value encodes the global (wrapped) cell index and the variable."""
    v, k, j, i = idx
    n = case["n"]
    return v * 1e6 + (k % n[2]) * 1e4 + (j % n[1]) * 1e2 + (i % n[0])


def _rank(rank, world, port, splits, which, grouped=False):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = _cases()[which]
        lay = decomp.Layout(c, splits, rank)
        shp = _shape(lay)
        U = torch.full(shp, -7.0, dtype=torch.float64)
        vv, kk, jj, ii = np.meshgrid(*[np.arange(s) for s in shp], indexing="ij")
        gk, gj, gi = kk - 3 + lay.offset[2], jj - 3 + lay.offset[1], ii - 3 + lay.offset[0]
        field = torch.tensor(_global_value(c, (vv, gk, gj, gi)))
        inner = (slice(None),) + lay.interior()
        U[inner] = field[inner]
        decomp.exchange(U, lay, _pack(lay), _unpack(lay), decomp.TorchComm(grouped=grouped))
        # cells interior or in an exchange halo along every axis hold the global value
        ok = np.ones(shp[1:], dtype=bool)
        for a, g in ((2, kk[0]), (1, jj[0]), (0, ii[0])):
            n = lay.n[a]
            inside = (g >= 3) & (g < 3 + n)
            lo = (g < 3) & (lay.neighbour(a, 0) is not None)
            hi = (g >= 3 + n) & (lay.neighbour(a, 1) is not None)
            ok &= inside | lo | hi
        assert ok.sum() > np.prod([lay.n[a] for a in range(3)])
        got = U.numpy()[:, ok]
        want = field.numpy()[:, ok]
        assert np.array_equal(got, want), (rank, np.argwhere(got != want)[:5])
    finally:
        dist.destroy_process_group()


def _cases():
    return {
        "slabs": wl.random_box(3, (6, 5, 8), bc=(P, WALL, P)),
        "blocks": wl.random_box(3, (7, 8, 6), bc=(P, WALL, P)),
        "blocks3": wl.random_box(3, (6, 6, 7)),
    }


def _port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


@pytest.mark.parametrize("which,splits", [("slabs", (1, 1, 2)), ("blocks", (2, 2, 1)),
                                          ("blocks3", (2, 1, 2))])
def test_exchange_fills_every_exchange_halo_over_gloo(which, splits):
    import torch.multiprocessing as mp
    world = splits[0] * splits[1] * splits[2]
    mp.spawn(_rank, args=(world, _port(), splits, which), nprocs=world, join=True)


@pytest.mark.parametrize("which,splits", [("blocks", (2, 2, 1)), ("slabs", (1, 1, 2))])
def test_grouped_exchange_over_gloo(which, splits):
    """The same exchange with each axis's sends and receives posted as one batch_isend_irecv group
    (what TorchComm does over NCCL, where separately enqueued sends would wait on each other):
    every exchange halo holds the global value, including two blocks on a periodic axis, where both
    faces swap with the same peer."""
    import torch.multiprocessing as mp
    world = splits[0] * splits[1] * splits[2]
    mp.spawn(_rank, args=(world, _port(), splits, which, True), nprocs=world, join=True)
