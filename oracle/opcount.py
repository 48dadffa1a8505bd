"""Operation counts of the discretisation, measured on the oracle with a counting scalar.

TEST INFRASTRUCTURE (part of the oracle package): it runs the oracle's own functions on numpy object
arrays of `Counted` scalars.  Every arithmetic operation on a Counted value creates a node of an
operation graph (its class, its operands, and the phase of the computation it belongs to).  Only
the nodes reachable from the results are counted, so what the oracle evaluates and then discards
(the unselected branches of the HLLC solver, evaluated for all faces and picked with np.where; the
fluxes of halo rows that no cell uses) is not counted, and a value the oracle forms once and reuses
is counted once.  A selection (np.where, np.minimum, the TENO keep flags) is a node of no cost whose
operands are the value it picked and the operands of the comparisons that decided it, so the work
of a decision counts exactly when the value it selected is used, and a branch test that the
definition never reaches (np.where nests them) does not count.  The result is the work of the
definition evaluated face by face and cell by cell, with nothing shared between neighbouring faces.

Classes: add (additions and subtractions), mul, div, sqrt, pow (non-integer powers; an integer
power counts the multiplications of binary exponentiation), misc (abs, floor), neg (sign changes).
flops = add + mul + div + sqrt + pow.

Phases: prim (conservative -> primitive), recon (WENO5 / TENO6-A with its limiter), riemann (HLLC),
visc (the dissipative face flux), grad (centre velocity derivatives), div (combining the convective
and dissipative face fluxes, the flux difference, its scaling by the width, accumulation), stage
(RK3 combination), cfl (the time step's rates).

`python -m oracle.opcount` writes profiles/oracle_op_counts.json (the per-unit counts the
benchmark's rooflines use); tests/test_oracle_opcount.py pins the counter and checks that the file
is current.
"""
import json
import math
import os
import sys

import numpy as np

from . import ns_fv as nf
from . import teno as tn

CLASSES = ("add", "mul", "div", "sqrt", "pow", "misc", "neg")
_phase = ["other"]
_roots = []


class Decision:
    """The outcome of a comparison with the values it compared."""
    __slots__ = ("b", "ops")

    def __init__(self, b, ops):
        self.b = bool(b)
        self.ops = ops

    def __bool__(self):
        return self.b

    def __or__(self, o):
        return Decision(self.b or bool(o), self.ops + (o.ops if isinstance(o, Decision) else ()))

    __ror__ = __or__

    def _sel(self, x):
        return Counted(float(x) * self.b, "sel", self.ops)

    def __mul__(self, x):
        return self._sel(x)

    __rmul__ = __mul__


class Counted:
    """A float that records the operation graph of everything computed from it."""
    __slots__ = ("v", "op", "a", "phase")

    def __init__(self, v, op=None, a=()):
        self.v = float(v)
        self.op = op
        self.a = a
        self.phase = _phase[0]

    @staticmethod
    def _val(x):
        return x.v if isinstance(x, Counted) else float(x)

    def _bin(self, other, op, f, swap=False):
        if isinstance(other, Decision):
            other = other._sel(1.0)
        ov = Counted._val(other)
        v = f(ov, self.v) if swap else f(self.v, ov)
        o = other if isinstance(other, Counted) else None
        return Counted(v, op, (o, self) if swap else (self, o))

    def __add__(self, o):
        return self._bin(o, "add", lambda x, y: x + y)

    def __radd__(self, o):
        return self._bin(o, "add", lambda x, y: x + y, swap=True)

    def __sub__(self, o):
        return self._bin(o, "add", lambda x, y: x - y)

    def __rsub__(self, o):
        return self._bin(o, "add", lambda x, y: x - y, swap=True)

    def __mul__(self, o):
        return self._bin(o, "mul", lambda x, y: x * y)

    def __rmul__(self, o):
        return self._bin(o, "mul", lambda x, y: x * y, swap=True)

    def __truediv__(self, o):
        return self._bin(o, "div", lambda x, y: x / y)

    def __rtruediv__(self, o):
        return self._bin(o, "div", lambda x, y: x / y, swap=True)

    def __pow__(self, e):
        ev = Counted._val(e)
        if not isinstance(e, Counted) and ev == int(ev) and 2 <= ev <= 64:
            # binary exponentiation: bit_length - 1 squarings, popcount - 1 multiplications
            n = int(ev)
            muls = n.bit_length() - 1 + bin(n).count("1") - 1
            node = self
            for _ in range(muls - 1):
                node = Counted(node.v, "mul", (node,))
            return Counted(self.v ** n, "mul", (node,))
        return Counted(self.v ** ev, "pow", (self, e if isinstance(e, Counted) else None))

    def __rpow__(self, base):
        return Counted(float(base) ** self.v, "pow", (self,))

    def floor(self):
        return Counted(math.floor(self.v), "misc", (self,))

    def __neg__(self):
        return Counted(-self.v, "neg", (self,))

    def __pos__(self):
        return self

    def __abs__(self):
        return Counted(abs(self.v), "misc", (self,))

    def sqrt(self):
        return Counted(math.sqrt(self.v), "sqrt", (self,))

    def _cmp(self, o, f):
        return Decision(f(self.v, Counted._val(o)), (self, o) if isinstance(o, Counted) else (self,))

    def __lt__(self, o):
        return self._cmp(o, lambda x, y: x < y)

    def __le__(self, o):
        return self._cmp(o, lambda x, y: x <= y)

    def __gt__(self, o):
        return self._cmp(o, lambda x, y: x > y)

    def __ge__(self, o):
        return self._cmp(o, lambda x, y: x >= y)

    def __hash__(self):
        return id(self)

    def __float__(self):
        return self.v


class _NumpyProxy:
    """numpy for the oracle's modules while counting: selections become zero-cost nodes linked to
    the comparisons that decided them; everything else is numpy."""

    def __getattr__(self, k):
        f = getattr(np, k)
        if not callable(f) or isinstance(f, type):
            return f

        def keep(x):
            if isinstance(x, np.ndarray) and x.dtype == object and not isinstance(x, CountedArray):
                return x.view(CountedArray)
            if isinstance(x, (list, tuple)):
                return type(x)(keep(y) for y in x)
            return x

        return lambda *a, **kw: keep(f(*a, **kw))

    @staticmethod
    def _pick(c, a, b):
        v = a if c else b
        if isinstance(c, Decision):
            base = v if isinstance(v, Counted) else None
            return Counted(Counted._val(v), "sel", ((base,) if base is not None else ()) + c.ops)
        return v

    def where(self, cond, a, b):
        cond, a, b = np.broadcast_arrays(np.asarray(cond, dtype=object), np.asarray(a, dtype=object),
                                         np.asarray(b, dtype=object))
        out = np.empty(cond.shape, dtype=object)
        for i in np.ndindex(cond.shape):
            out[i] = self._pick(cond[i], a[i], b[i])
        return out.view(CountedArray)

    def minimum(self, a, b):
        a, b = np.broadcast_arrays(np.asarray(a, dtype=object), np.asarray(b, dtype=object))
        out = np.empty(a.shape, dtype=object)
        for i in np.ndindex(a.shape):
            x, y = a[i], b[i]
            xv, yv = Counted._val(x), Counted._val(y)
            pick = x if xv <= yv else y
            ops = tuple(z for z in (x, y) if isinstance(z, Counted))
            out[i] = Counted(Counted._val(pick), "sel", ops)
        return out.view(CountedArray)

    def logical_not(self, a):
        a = np.asarray(a, dtype=object)
        out = np.empty(a.shape, dtype=object)
        for i in np.ndindex(a.shape):
            d = a[i]
            out[i] = Decision(not bool(d), d.ops if isinstance(d, Decision) else ())
        return out.view(CountedArray)

    def min(self, a, *args, **kw):
        arr = np.asarray(a, dtype=object).reshape(-1)
        _roots.extend(x for x in arr if isinstance(x, Counted))
        return min(arr, key=Counted._val)


_cmp_obj = {name: np.frompyfunc(f, 2, 1) for name, f in (
    ("lt", lambda x, y: x < y), ("le", lambda x, y: x <= y),
    ("gt", lambda x, y: x > y), ("ge", lambda x, y: x >= y))}


class CountedArray(np.ndarray):
    """Object arrays whose comparisons keep each element's Decision (numpy's own comparison of
    object arrays converts the results to plain booleans); results of numpy operations on them
    stay of this type."""

    def _cmp(self, o, name):
        return _cmp_obj[name](np.asarray(self), np.asarray(o, dtype=object)).view(CountedArray)

    def __lt__(self, o):
        return self._cmp(o, "lt")

    def __le__(self, o):
        return self._cmp(o, "le")

    def __gt__(self, o):
        return self._cmp(o, "gt")

    def __ge__(self, o):
        return self._cmp(o, "ge")


def counted_array(x):
    """An object array of Counted leaves with the values of x."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty(x.shape, dtype=object)
    flat = out.reshape(-1)
    for i, v in enumerate(x.reshape(-1)):
        flat[i] = Counted(v)
    return out.view(CountedArray)


def tally(roots):
    """Per phase and class: the nodes reachable from roots, each counted once (selections free)."""
    seen = set()
    stack = [r for r in roots if isinstance(r, Counted)]
    counts = {}
    while stack:
        n = stack.pop()
        if id(n) in seen:
            continue
        seen.add(id(n))
        if n.op is not None:
            if n.op != "sel":
                ph = counts.setdefault(n.phase, dict.fromkeys(CLASSES, 0))
                ph[n.op] += 1
            for p in n.a:
                if isinstance(p, Counted):
                    stack.append(p)
    return counts


class _Phase:
    def __init__(self, name):
        self.name = name

    def __enter__(self):
        self.prev = _phase[0]
        _phase[0] = self.name

    def __exit__(self, *a):
        _phase[0] = self.prev


def _tagged(f, phase):
    def g(*args, **kw):
        with _Phase(phase):
            return f(*args, **kw)
    return g


def _counting(fn):
    """Run fn with the oracle's building blocks tagged by phase and numpy's selections linked to
    their decisions."""
    tags = [(nf, "cons_to_prim", "prim"), (nf, "weno5", "recon"), (nf, "hllc_flux", "riemann"),
            (nf, "viscous_face_flux", "visc"), (nf, "_centre_derivative", "grad"),
            (tn, "teno6a", "recon"), (tn, "limit_states", "recon")]
    saved = [(m, name, getattr(m, name)) for m, name, _ in tags]
    saved_np = [(m, m.np) for m in (nf, tn)]
    try:
        for m, name, ph in tags:
            setattr(m, name, _tagged(getattr(m, name), ph))
        for m in (nf, tn):
            m.np = _NumpyProxy()
        return fn()
    finally:
        for m, name, f in saved:
            setattr(m, name, f)
        for m, orig in saved_np:
            m.np = orig


def _flops(c):
    return c["add"] + c["mul"] + c["div"] + c["sqrt"] + c["pow"]


def _state(case_dict, seed=0, amp=0.3):
    """A smooth subsonic state on the case's grid (every HLLC face takes a star branch, as in the
    benchmark flows), padded."""
    case = nf.Case(case_dict)
    grid = nf.Grid(case)
    z, y, x = np.meshgrid(grid.axes[2].xc, grid.axes[1].xc, grid.axes[0].xc, indexing="ij")
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * math.pi, 8)
    rho = 1.0 + 0.1 * np.sin(x + ph[0]) * np.cos(y + ph[1])
    u = amp * np.sin(x + ph[2]) * np.cos(z + ph[3])
    v = amp * np.cos(y + ph[4]) * np.sin(x + ph[5])
    w = amp * np.sin(z + ph[6]) * np.cos(y + ph[7])
    p = 1.0 + 0.05 * np.cos(x + y + z)
    return case, grid, nf.prim_to_cons(np.stack([rho, u, v, w, p]), case)


def count_rhs(case_dict):
    """Per unit of one right-hand side on a periodic box: per face (recon, riemann, visc), per cell
    and axis (div), per cell (grad; prim on a one-cell array, every output used)."""
    case, grid, U = _state(case_dict)
    Uc = counted_array(U)
    inner = (slice(None),) + case.interior()
    R = _counting(lambda: nf.rhs_filled(Uc, case, grid))
    t = tally(list(R[inner].reshape(-1)))
    ncell = case.n[0] * case.n[1] * case.n[2]
    nface = sum((case.n[d] + 1) * (ncell // case.n[d]) for d in range(case.ndim))
    zero = dict.fromkeys(CLASSES, 0)
    per = {}
    for ph, unit in (("recon", nface), ("riemann", nface), ("visc", nface),
                     ("other", ncell * case.ndim), ("grad", ncell)):
        src = t.get(ph, zero)
        per["div" if ph == "other" else ph] = {k: src[k] / unit for k in CLASSES}
    one = counted_array(U[:, :1, :1, :1])
    W1, T1 = _counting(lambda: nf.cons_to_prim(one, case))
    per["prim"] = dict(tally(list(W1.reshape(-1)) + list(T1.reshape(-1))).get("prim", zero))
    return per


def count_stage_and_cfl(case_dict):
    """The RK3 combination per cell over one step (a right-hand side returning leaves), and the
    time step's rates per cell (cfl_dt; the primitives it converts are the right-hand side's)."""
    case, grid, U = _state(case_dict)
    inner = (slice(None),) + case.interior()
    ncell = case.n[0] * case.n[1] * case.n[2]
    Un1 = nf.rk3(counted_array(U), 0.01, lambda V: counted_array(np.ones(V.shape)), inner)
    st = tally(list(Un1[inner].reshape(-1))).get("other", dict.fromkeys(CLASSES, 0))
    stage = {k: v / ncell for k, v in st.items()}
    del _roots[:]
    _counting(lambda: nf.cfl_dt(counted_array(U), case, grid))
    cf = tally(list(_roots))
    cfl = {k: sum(ph[k] for name, ph in cf.items() if name != "prim") / ncell for k in CLASSES}
    return stage, cfl


def counts_for(case_dict):
    per = count_rhs(case_dict)
    stage, cfl = count_stage_and_cfl(case_dict)
    nd = int(case_dict["ndim"])
    face = {k: per["recon"][k] + per["riemann"][k] + per["visc"][k] for k in CLASSES}
    cell_axis = {k: face[k] + per["div"][k] for k in CLASSES}
    update = {k: 3 * (nd * cell_axis[k] + per["prim"][k] + per["grad"][k]) + stage[k] + cfl[k]
              for k in CLASSES}
    out = {ph: dict(v, flops=_flops(v)) for ph, v in per.items()}
    out["stage_per_step"] = dict(stage, flops=_flops(stage))
    out["cfl"] = dict(cfl, flops=_flops(cfl))
    out["face"] = dict(face, flops=_flops(face))
    out["cell_axis"] = dict(cell_axis, flops=_flops(cell_axis))
    out["cell_update"] = dict(update, flops=_flops(update))
    return out


def workloads_to_count():
    from paper_2406_19494_gb300 import workloads as wl
    P = ("periodic", "periodic")
    box = lambda **kw: wl.random_box(3, (6, 5, 4), bc=(P, P, P), lo=(0, 0, 0),      # noqa: E731
                                     hi=(2 * math.pi,) * 3, **kw)
    return {
        "weno5z_power": box(visc="power", weno="z"),          # the Taylor-Green / channel scheme
        "weno5js_power": box(visc="power", weno="js"),
        "weno5z_sutherland": box(visc="sutherland", weno="z"),
        "weno5z_euler": box(visc="none", weno="z"),
        "teno6a_power_visc6": box(visc="power", weno="teno6a", visc_order=6),
    }


def main(path=None):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = path or os.path.join(root, "profiles", "oracle_op_counts.json")
    out = {"how": "python -m oracle.opcount: the oracle's right-hand side, RK3 combination and CFL "
                  "rates on counting scalars (3-D periodic 6x5x4 box, smooth subsonic state: every "
                  "HLLC face takes a star branch); operations reachable from the results, per unit",
           "classes": list(CLASSES), "flops": "add + mul + div + sqrt + pow",
           "workloads": {k: counts_for(v) for k, v in workloads_to_count().items()}}
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    return out


if __name__ == "__main__":
    res = main(sys.argv[1] if len(sys.argv) > 1 else None)
    for k, v in res["workloads"].items():
        print(k, "cell_axis", round(v["cell_axis"]["flops"], 2), "face", round(v["face"]["flops"], 2),
              "recon/face", round(v["recon"]["flops"], 1), "riemann", round(v["riemann"]["flops"], 1),
              "visc", round(v["visc"]["flops"], 1), "update", round(v["cell_update"]["flops"], 1))
