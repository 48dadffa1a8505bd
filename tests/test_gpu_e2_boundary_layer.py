"""Section 3.2's validation of the laminar boundary layer (the wall disturbance switched off): Ma 2.25,
Pr 0.72, Re per unit length 1e4, [1, 1.5] x [0, 0.4] on 300 x 200 cells (uniform in x, tanh
beta = 2.2 towards the wall in y), Sutherland viscosity, adiabatic no-slip wall, zero gradient at
north and east, the compressible similarity solution imposed at the inlet.  The paper compares
u / u_e and T / T_e at the outlet x = 1.5 with the similarity solution over eta.

From the self-similar field, FP64 WENO5-Z + HLLC + fourth-order dissipative fluxes, to t = 2 (two
flow-through times of the free stream; the profile is then within about 0.003 of its steady
state, reached near t = 5): at the last cell column, with eta formed from the computed density
(eta = int rho dy / sqrt(2 x / Re)), the velocity and temperature differ from the similarity
solution by at most 2.5 % of the edge values over eta <= 8 (measured 1.6 % at t = 2 and 1.9 % for
u, 2.0 % for T at t = 5), and the wall temperature is the similarity solution's adiabatic wall
temperature within 0.5 % (measured 0.2 %)."""
import numpy as np
import pytest

from paper_2406_19494_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build
    build.build()


def outlet_profile(c, sim, s, U):
    """(eta, u, T) at the last interior column from the state U (numpy, padded)."""
    xc, _ = s.grid(0)
    _, dy = s.grid(1)
    rho = U[0, 0, 3:-3, -4]
    u = U[1, 0, 3:-3, -4] / rho
    v = U[2, 0, 3:-3, -4] / rho
    p = (c["gamma"] - 1.0) * (U[4, 0, 3:-3, -4] - 0.5 * rho * (u * u + v * v))
    T = p / (rho * c["R"])
    d = dy[3:-3]
    eta = (np.cumsum(rho * d) - 0.5 * rho * d) / np.sqrt(2.0 * xc[-4] * c["mu_ref"])
    return eta, u, T


def test_outlet_profile_matches_the_similarity_solution():
    from paper_2406_19494_gb300.solver import Solver
    c = wl.e2_case()
    sim = wl.e2_similarity(c)
    s = Solver(c)
    xc, _ = s.grid(0)
    yc, _ = s.grid(1)
    W = wl.similarity_field(c, sim, xc[3:-3], yc[3:-3])
    Wp = np.pad(W, [(0, 0), (0, 0), (3, 3), (3, 3)], mode="edge")
    U = s.prim_to_cons(torch.from_numpy(np.ascontiguousarray(Wp)).cuda())
    s.set_inflow(0, 0, torch.from_numpy(wl.e2_inflow(c, sim, yc)).cuda())
    t = 0.0
    while t < 2.0:
        s.step(U, 4000, 2.0)
        t, _ = s.time()
    s.check()
    eta, u, T = outlet_profile(c, sim, s, U.cpu().numpy())
    fp = np.interp(eta, sim["eta"], sim["fp"], right=1.0)
    g = np.interp(eta, sim["eta"], sim["g"], right=1.0)
    sel = eta <= 8.0
    assert sel.sum() > 100                          # the layer is resolved by the stretched grid
    assert np.max(np.abs(u - fp)[sel]) < 0.025
    assert np.max(np.abs(T - g)[sel]) < 0.025
    assert abs(T[0] / sim["g"][0] - 1.0) < 0.005
    assert np.all(np.diff(u[sel]) > -1e-3)           # monotone velocity profile (no overshoot)
