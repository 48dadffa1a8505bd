"""Serving loop: continuous batching of uneven solves on one GPU.

Every solve in the mix gives exactly (bitwise) what the same request gives when it is served
alone: no kernel has atomics or arithmetic that depends on the other solves or on the launch
shape.  Solves that run alone in the server (their own stream and graph) also equal fluid_step
bitwise.  Batched solves run the same kernel bodies compiled into the batched launches, where the
compiler may fuse a few multiply-adds differently, so they equal fluid_step within the parity
tolerance (1e-12 of each variable's magnitude; observed at most 1e-13).  Admission must respect
the HBM budget; polls time out on the host."""
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


def _served_alone(case, U0, nsteps, precision, batch=True, chunk=7):
    """The request served on its own (a bucket of one when batched)."""
    from paper_2406_19494_gb300.serve import Server
    srv = Server(budget_bytes=8e9, max_active=2, chunk_steps=chunk, graphs=True, batch=batch)
    res, U = srv.poll(srv.submit(case, U0, nsteps, precision=precision), timeout_ms=120000)
    srv.close()
    assert res["status"] == 0
    return U


TOL = 1e-12


def _close(U, ref):
    for v in range(5):
        m = np.max(np.abs(ref[v]))
        if np.max(np.abs(U[v] - ref[v])) > TOL * m:
            return False
    return True


def _mix():
    reqs = [dict(kind="vortex", n=48, nsteps=23, seed=1), dict(kind="riemann", n=40, nsteps=31, seed=2),
            dict(kind="tgv", n=16, nsteps=12, seed=3), dict(kind="vortex", n=64, nsteps=45, seed=4),
            dict(kind="riemann", n=56, nsteps=17, seed=5), dict(kind="tgv", n=20, nsteps=9, seed=6),
            dict(kind="riemann", n=40, nsteps=31, seed=7), dict(kind="vortex", n=32, nsteps=60, seed=8)]
    return [(r,) + _initial(r) for r in reqs]


@pytest.mark.parametrize("precision,batch", [("fp64", True), ("mixed", True), ("fp64", False),
                                             ("mixed", False)])
def test_results_equal_alone_and_in_the_mix(precision, batch):
    """Batched (one launch per kernel over a bucket of 2-D and 3-D solves of different sizes, graph
    per bucket) and unbatched (a stream and graph per solve): both bitwise equal to fluid_step."""
    from paper_2406_19494_gb300.serve import Server
    mix = _mix()
    srv = Server(budget_bytes=8e9, max_active=5, chunk_steps=7, graphs=True, autotune=True, batch=batch)
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
        if batch:
            # the same bits as the request served alone, and fluid_step's result to rounding
            assert np.array_equal(U, _served_alone(case, U0, r["nsteps"], precision)), r
            assert _close(U, ref), (r, np.max(np.abs(U - ref)))
        else:
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
        ref = _alone(case, U0, r["nsteps"], "fp64")
        if case["weno"] == "teno6a":
            assert np.array_equal(U, ref), r                 # runs alone in the server
        else:
            assert np.array_equal(U, _served_alone(case, U0, r["nsteps"], "fp64", chunk=5)), r
            assert _close(U, ref), r


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


def test_late_arrivals_join_a_running_bucket():
    """Requests submitted while a bucket is advancing join it between chunks (continuous
    batching): 16 solves of uneven sizes and step counts, the second half submitted after the
    first results are out; every result equals the solve alone."""
    import time
    from paper_2406_19494_gb300.serve import Server
    reqs = []
    for i in range(16):
        kind = ("vortex", "riemann", "tgv")[i % 3]
        n = (24 + 7 * i) if kind != "tgv" else 12 + 2 * (i % 4)
        reqs.append(dict(kind=kind, n=n, nsteps=5 + 11 * (i % 5), seed=100 + i))
    mix = [(r,) + _initial(r) for r in reqs]
    srv = Server(budget_bytes=8e9, max_active=12, chunk_steps=4, graphs=True)
    first = [srv.submit(case, U0, r["nsteps"]) for r, case, U0 in mix[:8]]
    got = {0: srv.poll(first[0], timeout_ms=120000)}
    st_mid = srv.stats()
    late = [srv.submit(case, U0, r["nsteps"]) for r, case, U0 in mix[8:]]
    tickets = first + late
    for i, t in enumerate(tickets):
        if i not in got:
            got[i] = srv.poll(t, timeout_ms=120000)
    srv.close()
    assert st_mid["completed"] >= 1
    for i, (r, case, U0) in enumerate(mix):
        res, U = got[i]
        assert res["status"] == 0 and res["steps_done"] == r["nsteps"]
        assert np.array_equal(U, _served_alone(case, U0, r["nsteps"], "fp64", chunk=4)), r
        assert _close(U, _alone(case, U0, r["nsteps"], "fp64")), r


def test_served_solve_matches_the_oracle():
    """A member of a batched mix against the CPU oracle's own steps (FP64, CFL time step each
    step): per variable within 1e-12 of the state's magnitude, as the parity tests."""
    from oracle import ns_fv as nf
    from paper_2406_19494_gb300.serve import Server
    mix = _mix()
    r, case, U0 = mix[0]                       # the 48^2 isentropic vortex
    nsteps = 6
    srv = Server(budget_bytes=8e9, max_active=8, chunk_steps=4, graphs=True)
    tickets = [srv.submit(c, U, rr["nsteps"] if i else nsteps) for i, (rr, c, U) in enumerate(mix)]
    res, U = srv.poll(tickets[0], timeout_ms=120000)
    for t in tickets[1:]:
        srv.poll(t, timeout_ms=120000)
    srv.close()
    oc = nf.Case(case)
    og = nf.Grid(oc)
    ref, t_ref, taken = nf.advance(U0.copy(), oc, og, nsteps)
    assert taken == nsteps and res["t_final"] == pytest.approx(t_ref, rel=1e-12)
    inner = (slice(None),) + oc.interior()
    for v in range(5):
        m = np.max(np.abs(ref[inner][v]))
        assert np.max(np.abs(U[inner][v] - ref[inner][v])) <= 1e-12 * m, v
