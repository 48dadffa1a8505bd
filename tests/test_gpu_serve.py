"""Serving loop: continuous batching of uneven solves on one GPU.

Every solve in the mix must give exactly (bitwise) what the same solve gives alone through
fluid_step: the kernels have no atomics and no shape-dependent arithmetic, so the tolerance stated
for serving is zero.  Admission must respect the HBM budget; polls time out on the host."""
import numpy as np
import pytest

from paper_2406_19494_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build
    build.build()


def _initial(req):
    from paper_2406_19494_gb300.solver import Solver

    def centres_of(case):
        s = Solver(case)
        out = [s.grid(a)[0] for a in range(3)]
        h = [3 if a < case["ndim"] else 0 for a in range(3)]
        return [out[a][h[a]:len(out[a]) - h[a]] for a in range(3)]

    case, W = wl.serving_case_and_prims(req, centres_of)
    pad = [(0, 0)] + [(3 if a < case["ndim"] else 0,) * 2 for a in (2, 1, 0)]
    Wp = np.pad(W, pad, mode="edge")
    s = Solver(case)
    U = s.prim_to_cons(torch.from_numpy(np.ascontiguousarray(Wp)).cuda()).cpu().numpy()
    return case, U


def _alone(case, U0, nsteps, precision):
    from paper_2406_19494_gb300.solver import Solver
    s = Solver(case, precision=precision)
    U = torch.from_numpy(U0.copy()).cuda()
    s.step(U, nsteps)
    s.check()
    return U.cpu().numpy()


def _mix():
    reqs = [dict(kind="vortex", n=48, nsteps=23, seed=1), dict(kind="riemann", n=40, nsteps=31, seed=2),
            dict(kind="tgv", n=16, nsteps=12, seed=3), dict(kind="vortex", n=64, nsteps=45, seed=4),
            dict(kind="riemann", n=56, nsteps=17, seed=5), dict(kind="tgv", n=20, nsteps=9, seed=6),
            dict(kind="riemann", n=40, nsteps=31, seed=7), dict(kind="vortex", n=32, nsteps=60, seed=8)]
    return [(r,) + _initial(r) for r in reqs]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_results_equal_alone_and_in_the_mix(precision):
    from paper_2406_19494_gb300.serve import Server
    mix = _mix()
    srv = Server(budget_bytes=8e9, max_active=5, chunk_steps=7, graphs=True, autotune=True)
    tickets = []
    for i, (r, case, U0) in enumerate(mix):
        tickets.append(srv.submit(case, U0, r["nsteps"], precision=precision))
    outs = [srv.poll(t, timeout_ms=120000) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(mix)
    for (r, case, U0), (res, U) in zip(mix, outs):
        assert res["status"] == 0 and res["steps_done"] == r["nsteps"]
        assert res["submit_s"] <= res["start_s"] <= res["finish_s"]
        ref = _alone(case, U0, r["nsteps"], precision)
        assert np.array_equal(U, ref), (r, np.max(np.abs(U - ref)))


def test_channel_scheme_requests_equal_alone_and_in_the_mix():
    """Requests with the paper's channel scheme (TENO6-A, sixth-order dissipative fluxes, FP64) in
    a mix with WENO5 requests: each result equals the same solve alone."""
    from paper_2406_19494_gb300.serve import Server
    mix = _mix()[:4]
    teno = []
    for r, case, U0 in mix:
        if case["visc"] == "none":
            case = dict(case, weno="teno6a")
        else:
            case = dict(case, weno="teno6a", visc_order=6)
        teno.append((r, case, U0))
    jobs = mix[:2] + teno
    srv = Server(budget_bytes=8e9, max_active=4, chunk_steps=5, graphs=True, autotune=True)
    tickets = [srv.submit(case, U0, r["nsteps"], precision="fp64") for r, case, U0 in jobs]
    outs = [srv.poll(t, timeout_ms=120000) for t in tickets]
    srv.close()
    for (r, case, U0), (res, U) in zip(jobs, outs):
        assert res["status"] == 0 and res["steps_done"] == r["nsteps"]
        assert np.array_equal(U, _alone(case, U0, r["nsteps"], "fp64")), r


def test_admission_respects_the_budget():
    from paper_2406_19494_gb300.serve import Server
    mix = _mix()
    srv = Server(budget_bytes=1, max_active=4)
    biggest = max(srv.footprint(case) for _, case, _ in mix)
    srv.close()
    budget = int(2.2 * biggest)
    srv = Server(budget_bytes=budget, max_active=8, chunk_steps=5)
    tickets = [srv.submit(case, U0, r["nsteps"]) for r, case, U0 in mix]
    for t in tickets:
        res, _ = srv.poll(t, timeout_ms=120000)
        assert res["status"] == 0
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(mix)
    assert 0 < st["peak_bytes"] <= budget


def test_over_budget_request_and_poll_timeout():
    from paper_2406_19494_gb300 import native
    from paper_2406_19494_gb300.serve import Server
    r, case, U0 = _mix()[3]
    srv = Server(budget_bytes=srv_budget(case), max_active=2, chunk_steps=1, graphs=False, autotune=False)
    big = wl.tgv_case(128)
    with pytest.raises(native.FluidError) as ei:
        srv.submit(big, np.zeros((5, 134, 134, 134)), 10)
    assert ei.value.status == native.FLUID_EBUDGET
    t = srv.submit(case, U0, 3000)
    assert srv.poll(t, timeout_ms=0) is None          # still running: host-side timeout
    assert srv.poll(t, timeout_ms=1) is None
    res, _ = srv.poll(t, timeout_ms=300000)
    srv.close()
    assert res["status"] == 0 and res["steps_done"] == 3000


def srv_budget(case):
    from paper_2406_19494_gb300.serve import Server
    s = Server(budget_bytes=1)
    b = s.footprint(case)
    s.close()
    return 2 * b
