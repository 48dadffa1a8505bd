"""Invariants of the GPU right-hand side that hold whatever the oracle says, for the three face
schemes (WENO5-Z and WENO5-JS in FP64, the paper's TENO6-A with sixth-order dissipative fluxes, and
the mixed FP32-flux / FP64-state form):

* free stream: a uniform state on a grid stretched along two axes gives R = 0 exactly, since every
  face then computes bitwise the same flux (Eq. ODE is a difference of face fluxes);
* conservation: on a periodic box the cell-volume-weighted sum of R vanishes to rounding for every
  variable, each face flux entering its two cells with opposite signs;
* axis exchange: exchanging x and y in a cubic periodic state (and the u, v momenta with them)
  exchanges R the same way, to rounding (the face kernels of different axes add their
  contributions in a different order)."""
import math

import numpy as np
import pytest

from helpers import padded_state
from paper_2406_19494_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = ("periodic", "periodic")
ZG = ("zero_gradient", "zero_gradient")

SCHEMES = {
    "fp64_wenoz": (dict(), "fp64"),
    "fp64_wenojs": (dict(weno="js"), "fp64"),
    "fp64_teno6a_visc6": (dict(weno="teno6a", visc_order=6), "fp64"),
    "mixed_wenoz": (dict(), "mixed"),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build
    build.build()


def _rhs(c, U, precision):
    from paper_2406_19494_gb300.solver import Solver
    s = Solver(c, precision=precision)
    R = s.rhs(torch.from_numpy(U).cuda())
    s.check()
    return s, R.cpu().numpy()


@pytest.mark.parametrize("name", list(SCHEMES))
def test_free_stream_gives_zero_rhs_exactly(name):
    extra, precision = SCHEMES[name]
    c = wl.random_box(3, (21, 17, 13), bc=(ZG, ZG, P), stretch=("tanh1", "tanh2", "uniform"),
                      beta=(1.3, 2.0, 0.0), visc="sutherland", **extra)
    case, grid, U = padded_state(c, uniform=(1.2, 0.3, -0.2, 0.1, 0.9))
    _, R = _rhs(c, U, precision)
    inner = (slice(None),) + case.interior()
    assert np.count_nonzero(R[inner]) == 0


@pytest.mark.parametrize("name", list(SCHEMES))
def test_periodic_box_conserves_every_variable(name):
    extra, precision = SCHEMES[name]
    c = wl.random_box(3, (19, 16, 14), stretch=("uniform", "tanh2", "uniform"), beta=(0.0, 1.5, 0.0),
                      **extra)
    case, grid, U = padded_state(c, seed=12)
    s, R = _rhs(c, U, precision)
    h = case.h
    dx = [s.grid(a)[1][h[a]:h[a] + case.n[a]] for a in range(3)]
    vol = dx[2][:, None, None] * dx[1][None, :, None] * dx[0][None, None, :]
    inner = (slice(None),) + case.interior()
    Ri = R[inner]
    for v in range(5):
        terms = (Ri[v] * vol).ravel()
        total = math.fsum(terms)
        scale = math.fsum(np.abs(terms))
        assert abs(total) <= 1e-13 * scale, (v, total, scale)


@pytest.mark.parametrize("name", list(SCHEMES))
def test_exchanging_x_and_y_exchanges_the_rhs(name):
    extra, precision = SCHEMES[name]
    n = 14
    c = wl.random_box(3, (n, n, 10), lo=(0.0, 0.0, 0.0), hi=(1.5, 1.5, 1.0), **extra)
    case, grid, U = padded_state(c, seed=21)
    _, R = _rhs(c, U, precision)
    # x <-> y: U'[v](z, y, x) = U[sigma v](z, x, y) with the x and y momenta exchanged
    sigma = [0, 2, 1, 3, 4]
    Us = np.ascontiguousarray(np.swapaxes(U, 2, 3)[sigma])
    _, Rs = _rhs(c, Us, precision)
    back = np.swapaxes(Rs, 2, 3)[sigma]
    inner = (slice(None),) + case.interior()
    tol = 1e-13 if precision == "fp64" else 1e-6
    for v in range(5):
        m = np.max(np.abs(R[inner][v]))
        assert np.max(np.abs(back[inner][v] - R[inner][v])) <= tol * m, v
