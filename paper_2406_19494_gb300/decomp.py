"""Block decomposition of one solve over several ranks (Section 2.2 of the paper: the padded domain
is split into S_x x S_y x S_z blocks, one per device, and every right-hand side first exchanges the
N_h = 3 halo layers with the neighbouring blocks; the time step is a minimum over the blocks).

Host logic only.  Layout says which cells a rank owns, who its neighbours are and what its block's
configuration is (FLUID_BC_EXCHANGE on the faces it shares, the global grid placement so that the
block's metrics are the global ones).  exchange() runs the halo passes x -> y -> z with caller-given
pack / unpack functions (the library's fluid_pack_halo / fluid_unpack_halo on the GPU) over a
torch.distributed process group: NCCL sends the device buffers, gloo goes through host copies.
BlockSolver advances one block with fluid_rk3_stage; with the same dt its result is bitwise the
single-domain fluid_step's on the same cells.
"""
import copy
import math

HALO = 3


def block_range(n, parts, k):
    """(offset, count) of block k when n cells are split into `parts` near-equal blocks (the first
    n % parts blocks get one cell more)."""
    base, extra = divmod(n, parts)
    return k * base + min(k, extra), base + (1 if k < extra else 0)


class Layout:
    """Placement of rank `rank` in a block decomposition of `case` (a workloads.py case dict) into
    splits = (S_x, S_y, S_z) blocks; ranks are numbered x fastest."""

    def __init__(self, case, splits, rank):
        self.case = case
        self.splits = tuple(int(s) for s in splits) + (1,) * (3 - len(splits))
        nd = int(case["ndim"])
        for a in range(3):
            if self.splits[a] < 1 or (a >= nd and self.splits[a] != 1):
                raise ValueError("splits must be >= 1 and 1 on inactive axes")
        self.size = self.splits[0] * self.splits[1] * self.splits[2]
        if not 0 <= rank < self.size:
            raise ValueError("rank outside the decomposition")
        self.rank = rank
        r = rank
        self.coords = []
        for a in range(3):
            self.coords.append(r % self.splits[a])
            r //= self.splits[a]
        self.offset, self.n = [], []
        for a in range(3):
            o, c = block_range(int(case["n"][a]), self.splits[a], self.coords[a])
            if self.splits[a] > 1 and int(case["n"][a]) // self.splits[a] < HALO:
                raise ValueError("every block needs at least %d cells on a split axis" % HALO)
            self.offset.append(o)
            self.n.append(c)

    def rank_of(self, coords):
        return coords[0] + self.splits[0] * (coords[1] + self.splits[1] * coords[2])

    def neighbour(self, axis, side):
        """Rank across face (axis, side), or None where the face is a physical boundary (or the
        axis is not split)."""
        S = self.splits[axis]
        if S == 1:
            return None
        c = list(self.coords)
        c[axis] += 1 if side == 1 else -1
        if c[axis] < 0 or c[axis] >= S:
            if self.case["bc"][axis][0] != "periodic":
                return None
            c[axis] %= S
        return self.rank_of(c)

    def local_case(self):
        """The case dict of this block: local sizes, exchange faces, global placement, the porous
        strip restricted to the block's wall cells."""
        c = copy.deepcopy(self.case)
        c["n"] = tuple(self.n)
        bc = [list(p) for p in self.case["bc"]]
        for a in range(3):
            for s in range(2):
                if self.neighbour(a, s) is not None:
                    bc[a][s] = "exchange"
        c["global_n"] = tuple(int(self.case["n"][a]) if self.splits[a] > 1 else 0 for a in range(3))
        c["offset"] = tuple(self.offset[a] if self.splits[a] > 1 else 0 for a in range(3))
        pz = self.case.get("porous")
        if pz:
            A, side = int(pz["axis"]), int(pz["side"])
            if bc[A][side] != "porous":
                c["porous"] = None                       # this block does not touch the wall
            else:
                # the wall cells of the block and of its exchange halos along the wall: the corner
                # ghost cells next to an exchange face mirror the neighbour's wall cells
                t1 = 1 if A == 0 else 0
                lo, hi = self._strip(t1, bc)
                if hi <= lo:
                    bc[A][side] = "wall"                 # no porous cell here: v_w = 0 everywhere
                    c["porous"] = None
                else:
                    c["porous"] = dict(pz, begin=lo - self.offset[t1], count=hi - lo)
        c["bc"] = tuple(tuple(p) for p in bc)
        return c

    def _strip(self, t1, bc):
        """Global cell range [lo, hi) of the porous strip on this block's wall, its exchange halos
        along the wall included."""
        pz = self.case["porous"]
        ext_lo = HALO if bc[t1][0] == "exchange" else 0
        ext_hi = HALO if bc[t1][1] == "exchange" else 0
        lo = max(int(pz["begin"]), self.offset[t1] - ext_lo)
        hi = min(int(pz["begin"]) + int(pz["count"]), self.offset[t1] + self.n[t1] + ext_hi)
        return lo, hi

    def phi_slice(self, phi):
        """The block's part of the global porous parameters (its strip, halos included; None when
        it has no porous cell)."""
        pz = self.case.get("porous")
        loc = self.local_case().get("porous")
        if not pz or not loc:
            return None
        t1 = 1 if int(pz["axis"]) == 0 else 0
        b = loc["begin"] + self.offset[t1] - int(pz["begin"])
        return phi[b:b + loc["count"]]

    def inflow_slice(self, axis, prof):
        """The block's part of a global inflow profile [5][T2][T1] over padded tangential ranges."""
        t1 = 1 if axis == 0 else 0
        t2 = 1 if axis == 2 else 2
        nd = int(self.case["ndim"])
        p = lambda b: self.n[b] + (2 * HALO if b < nd else 0)
        return prof[:, self.offset[t2]:self.offset[t2] + p(t2), self.offset[t1]:self.offset[t1] + p(t1)]

    def interior_of_global(self):
        """Index tuple (z, y, x) of this block's interior cells within a global padded field."""
        nd = int(self.case["ndim"])
        sl = []
        for a in (2, 1, 0):
            h = HALO if a < nd else 0
            sl.append(slice(h + self.offset[a], h + self.offset[a] + self.n[a]))
        return tuple(sl)

    def interior(self):
        nd = int(self.case["ndim"])
        return tuple(slice(HALO if a < nd else 0, (HALO if a < nd else 0) + self.n[a])
                     for a in (2, 1, 0))


def plan_axis(layout, a, U, pack):
    """The swaps of one axis: (ops, sides) with ops a list of ("send", peer, tag, buffer) and
    ("recv", peer, tag, count) and sides the halo face of each receive, in order.  A buffer sent
    across the high face lands in the neighbour's low halo and vice versa; the tag names the
    sender's side, so both faces may face the same peer (two blocks on a periodic axis), and the
    order (high send, low receive, low send, high receive) pairs the messages of a peer pair in
    posting order for transports without tags."""
    lo, hi = layout.neighbour(a, 0), layout.neighbour(a, 1)
    ops, sides = [], []
    if hi is not None:
        buf = pack(U, a, 1)
        count = buf.numel()
        ops.append(("send", hi, 2 * a + 1, buf))
    if lo is not None:
        buf0 = pack(U, a, 0)
        count = buf0.numel()
        ops.append(("recv", lo, 2 * a + 1, count))
        sides.append(0)
        ops.append(("send", lo, 2 * a, buf0))
    if hi is not None:
        ops.append(("recv", hi, 2 * a, count))
        sides.append(1)
    return ops, sides


def exchange(U, layout, pack, unpack, comm):
    """Refresh the exchange halos of U: for each axis in the order x, y, z, pack both faces, swap
    the buffers with the neighbours (comm.swap) and unpack what arrived.  pack(U, axis, side)
    returns a buffer, unpack(U, axis, side, buf) writes one.  Later axes carry the halos the
    earlier ones filled, which fills the edges and corners between diagonal blocks."""
    for a in range(int(layout.case["ndim"])):
        ops, sides = plan_axis(layout, a, U, pack)
        if not ops:
            continue
        for side, buf in zip(sides, comm.swap(ops)):
            unpack(U, a, side, buf)


class TorchComm:
    """Point-to-point swaps over a torch.distributed process group.  NCCL moves device tensors;
    gloo (CPU) stages them through host memory.  Buffers may be torch tensors of any device."""

    def __init__(self, group=None, grouped=None):
        """grouped: post each swap as one batch_isend_irecv group (default: with NCCL only)."""
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.backend = dist.get_backend(group)
        self.grouped = (self.backend == "nccl") if grouped is None else bool(grouped)

    def swap(self, ops):
        """Post every send and receive of one axis, then wait for all.  With NCCL they go as one
        group (batch_isend_irecv): a rank's sends and receives then progress together, where
        separately enqueued NCCL sends would each wait for a receive that the peer has queued
        behind its own send (every rank sends to its high neighbour first); NCCL ignores tags and
        matches a peer pair's messages in posting order, which plan_axis's order pairs up."""
        import torch
        dist = self.dist
        host = self.backend != "nccl"
        reqs, recvs, like, p2p = [], [], None, []
        for kind, peer, tag, x in ops:
            if kind == "send":
                like = x
                t = x.cpu() if host else x.contiguous()
                if self.grouped:
                    p2p.append(dist.P2POp(dist.isend, t, peer, group=self.group, tag=tag))
                else:
                    reqs.append(dist.isend(t, peer, group=self.group, tag=tag))
            else:
                dev = "cpu" if host else x_device(ops)
                r = torch.empty(x, dtype=torch.float64, device=dev)
                if self.grouped:
                    p2p.append(dist.P2POp(dist.irecv, r, peer, group=self.group, tag=tag))
                else:
                    reqs.append(dist.irecv(r, peer, group=self.group, tag=tag))
                recvs.append(r)
        if p2p:
            reqs.extend(dist.batch_isend_irecv(p2p))
        for q in reqs:
            q.wait()
        if host and like is not None and like.device.type != "cpu":
            return [r.to(like.device) for r in recvs]
        return recvs

    def min(self, x):
        """Minimum of a host float over the group."""
        import torch
        dist = self.dist
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=self.group)
        return float(t.item())


def x_device(ops):
    for kind, _, _, x in ops:
        if kind == "send":
            return x.device
    raise ValueError("a swap needs at least one send")


class LocalComm:
    """Swaps between blocks held by one process (several solvers on one device): buffers are
    posted per (sender, receiver, tag) and collected by the receiving block."""

    def __init__(self):
        self.box = {}

    def endpoint(self, rank):
        return _LocalEnd(self, rank)


class _LocalEnd:
    def __init__(self, hub, rank):
        self.hub, self.rank = hub, rank

    def post(self, ops):
        for kind, peer, tag, buf in ops:
            if kind == "send":
                self.hub.box[(self.rank, peer, tag)] = buf.clone()

    def collect(self, ops):
        return [self.hub.box.pop((peer, self.rank, tag)) for kind, peer, tag, _ in ops if kind == "recv"]


class BlockSolver:
    """One block of a decomposed solve on the current CUDA device: a sub-domain Solver, its halo
    exchange and the RK3 step through fluid_rk3_stage."""

    def __init__(self, case, splits, rank, comm, precision="fp64"):
        import torch
        from .solver import Solver
        self.layout = Layout(case, splits, rank)
        self.comm = comm
        self.solver = Solver(self.layout.local_case(), precision)
        self.S = torch.zeros(self.solver.shape, dtype=torch.float64, device="cuda")
        self.t = 0.0

    def pack(self, U, a, side):
        return self.solver.pack_halo(U, a, side)

    def unpack(self, U, a, side, buf):
        self.solver.unpack_halo(U, a, side, buf)

    def exchange(self, U):
        exchange(U, self.layout, self.pack, self.unpack, self.comm)

    def local_dt(self, U):
        return float(self.solver.compute_dt(U).item())

    def step(self, U, nsteps=1, dt=None):
        """nsteps RK3 steps of U (this block's padded state, halos refreshed here); dt=None takes
        the CFL time step of each step's initial state, minimised over the blocks."""
        for _ in range(nsteps):
            self.exchange(U)
            d = dt if dt is not None else self.comm.min(self.local_dt(U))
            if not (d > 0 and math.isfinite(d)):
                raise RuntimeError("non-positive or non-finite time step %r" % (d,))
            self.solver.rk3_stage(1, U, U, self.S, d)
            self.exchange(self.S)
            self.solver.rk3_stage(2, U, self.S, self.S, d)
            self.exchange(self.S)
            self.solver.rk3_stage(3, U, self.S, U, d)
            self.t += d
        return U


def run_local_blocks(blocks, Us, nsteps=1):
    """Advance blocks that one process holds (LocalComm endpoints) in lock step: every exchange
    posts all blocks' buffers before any block collects.  Returns the dt of each step."""
    dts = []

    def exchange_all(states):
        for a in range(int(blocks[0].layout.case["ndim"])):
            plans = []
            for b, U in zip(blocks, states):
                ops, sides = plan_axis(b.layout, a, U, b.pack)
                b.comm.post(ops)
                plans.append((ops, sides))
            for b, U, (ops, sides) in zip(blocks, states, plans):
                for side, buf in zip(sides, b.comm.collect(ops)):
                    b.unpack(U, a, side, buf)

    for _ in range(nsteps):
        exchange_all(Us)
        d = min(b.local_dt(U) for b, U in zip(blocks, Us))
        for b, U in zip(blocks, Us):
            b.solver.rk3_stage(1, U, U, b.S, d)
        exchange_all([b.S for b in blocks])
        for b, U in zip(blocks, Us):
            b.solver.rk3_stage(2, U, b.S, b.S, d)
        exchange_all([b.S for b in blocks])
        for b, U in zip(blocks, Us):
            b.solver.rk3_stage(3, U, b.S, U, d)
            b.t += d
        dts.append(d)
    return dts
