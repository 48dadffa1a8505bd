"""Shared test helpers: build oracle cases and seeded padded states from the workload generators."""
import numpy as np

from oracle import ns_fv as nf
from paper_2406_19494_gb300 import workloads as wl


def centres(case, grid):
    return [grid.axes[a].xc[case.h[a]:case.h[a] + case.n[a]] for a in range(3)]


def padded_state(case_dict, prims=None, seed=0, uniform=None, **kw):
    """(case, grid, U) with the interior of U set from `prims` (5, nz, ny, nx) or a random field;
    halo cells hold a harmless copy of the nearest interior value (they are overwritten by BCs)."""
    case = nf.Case(case_dict)
    grid = nf.Grid(case)
    xc, yc, zc = centres(case, grid)
    if uniform is not None:
        W = np.broadcast_to(np.asarray(uniform, dtype=np.float64)[:, None, None, None],
                            (5, case.n[2], case.n[1], case.n[0])).copy()
    elif prims is not None:
        W = np.asarray(prims, dtype=np.float64)
    else:
        W = wl.random_prims(xc, yc, zc, seed=seed, **kw)
    Wp = np.pad(W, [(0, 0)] + [(case.h[a], case.h[a]) for a in (2, 1, 0)], mode="edge")
    return case, grid, nf.prim_to_cons(Wp, case)


def rel_err(x, ref):
    """Per-variable max |x - ref| / max |ref| (ref nonzero), as a list."""
    out = []
    for v in range(x.shape[0]):
        m = np.max(np.abs(ref[v]))
        d = np.max(np.abs(x[v] - ref[v]))
        out.append(d / m if m > 0 else d)
    return out
