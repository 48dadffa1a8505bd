"""The face kernels' launch shape (fluid_tune_faces: threads per block, cells per marching
segment, the mixed path's tile or register-window kernels) is a performance choice only: the
right-hand side is the same to rounding for every shape.  The mixed path's y / z tiles of either
size compute each face with the same code from the same cell differences, so they agree bitwise;
its register-window kernels compile the same face arithmetic in another kernel, where the compiler
may fuse a different pair of FP32 operations into one multiply-add, so they agree to FP32
rounding.  The FP64 marches (WENO5-JS, WENO5-Z, TENO6-A) start every segment with the terms the
march would have carried there, formed by the march's own operations, so every segment length
gives bitwise the same right-hand side."""
import numpy as np
import pytest

from helpers import padded_state, rel_err
from paper_2406_19494_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = ("periodic", "periodic")
WALL = ("wall", "wall")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build
    build.build()


def _rhs(c, U, precision, block, seg):
    from paper_2406_19494_gb300.solver import Solver
    s = Solver(c, precision=precision)
    s.tune_faces(block, seg)
    R = s.rhs(torch.from_numpy(U).cuda())
    s.check()
    return R.cpu().numpy()


CASE = lambda: wl.random_box(3, (37, 29, 21), bc=(P, WALL, P), stretch=("uniform", "tanh2", "uniform"),
                             beta=(0.0, 2.0, 0.0), t_wall=((1, 1), (2.5, 2.2), (1, 1)))


@pytest.mark.parametrize("scheme", [dict(), dict(weno="js"), dict(weno="teno6a", visc_order=6)])
def test_fp64_shapes_agree_bitwise(scheme):
    c = dict(CASE(), **scheme)
    case, grid, U = padded_state(c, seed=8)
    inner = (slice(None),) + case.interior()
    base = _rhs(c, U, "fp64", 0, 0)[inner]
    for block, seg in ((64, 8), (96, 5), (128, 64), (32, 3), (128, 1)):
        R = _rhs(c, U, "fp64", block, seg)[inner]
        assert np.array_equal(R, base), (block, seg)


def test_mixed_shapes_agree():
    c = CASE()
    case, grid, U = padded_state(c, seed=9)
    inner = (slice(None),) + case.interior()
    base = _rhs(c, U, "mixed", 0, 0)[inner]
    for block, seg in ((64, 0), (128, 0)):
        R = _rhs(c, U, "mixed", block, seg)[inner]
        assert np.array_equal(R, base), (block, seg)
    for block, seg in ((64, -8), (128, -5), (32, -3)):
        R = _rhs(c, U, "mixed", block, seg)[inner]
        assert max(rel_err(R, base)) <= 1e-6, (block, seg)


@pytest.mark.parametrize("scheme", [dict(), dict(weno="teno6a", visc_order=6)])
def test_autotuned_shapes_agree_bitwise(scheme):
    """fluid_autotune_faces picks a segment length per axis by timing; whatever it picks, the
    right-hand side and a step are bitwise those of the automatic shape, and the state it was
    timed on is untouched."""
    from paper_2406_19494_gb300.solver import Solver
    c = dict(CASE(), **scheme)
    case, grid, U = padded_state(c, seed=10)
    inner = (slice(None),) + case.interior()
    Ud = torch.from_numpy(U).cuda()
    ref, tuned = Solver(c), Solver(c)
    U0 = Ud.clone()
    tuned.autotune_faces(Ud)
    assert torch.equal(Ud, U0)
    assert np.array_equal(tuned.rhs(Ud).cpu().numpy()[inner], ref.rhs(Ud).cpu().numpy()[inner])
    Ua, Ub = Ud.clone(), Ud.clone()
    ref.step(Ua, 2)
    tuned.step(Ub, 2)
    assert torch.equal(Ua, Ub)


def test_autotune_mixed_is_a_no_op():
    from paper_2406_19494_gb300.solver import Solver
    c = CASE()
    case, grid, U = padded_state(c, seed=11)
    s = Solver(c, precision="mixed")
    Ud = torch.from_numpy(U).cuda()
    before = s.rhs(Ud).cpu().numpy()
    s.autotune_faces(Ud)
    assert np.array_equal(s.rhs(Ud).cpu().numpy(), before)


def test_profiler_counts_kernels():
    """The profiler's launch count is the number of kernels: a face call with segment seams is two
    kernels (the face kernel and its seam kernel), one without (segments shorter than the seam
    buffer's minimum of 4 cells run without it)."""
    from paper_2406_19494_gb300.solver import Solver
    c = CASE()
    case, grid, U = padded_state(c, seed=12)
    s = Solver(c)
    Ud = torch.from_numpy(U).cuda()
    for seg, per_call in ((4, 2), (3, 1)):
        s.tune_faces(128, seg)
        s.profile(True)
        s.profile_read(True)
        s.rhs(Ud)
        p = s.profile_read(True)
        s.profile(False)
        for axis in ("face_x", "face_y", "face_z"):
            assert p[axis][1] == per_call, (seg, axis, p[axis])
        assert p["prim_bc"][1] == 1 and p["grad"][1] == 1, p


@pytest.mark.parametrize("scheme", [dict(), dict(weno="js"), dict(visc="none")])
def test_mixed_bulk_staged_tiles_agree_bitwise(scheme):
    """seg = 1 stages each y / z tile's (hi, lo) rows by cp.async.bulk and forms the cell
    differences from shared memory in the order the plain tiles form them from global memory, so
    the right-hand side is bitwise the same, on a 3-D box with walls and a 2-D grid of odd size."""
    for c in (dict(CASE(), **scheme),
              dict(wl.random_box(2, (45, 23, 1), bc=(P, WALL, P), stretch=("uniform", "tanh1", "uniform"),
                                 beta=(0.0, 2.0, 0.0), t_wall=((1, 1), (1.5, 1.2), (1, 1))), **scheme)):
        case, grid, U = padded_state(c, seed=11)
        inner = (slice(None),) + case.interior()
        base = _rhs(c, U, "mixed", 0, 0)[inner]
        R = _rhs(c, U, "mixed", 0, 1)[inner]
        assert np.array_equal(R, base)


def test_mixed_bulk_staged_steps_agree_bitwise():
    """A mixed fluid_step folds the stage into the last axis's tile kernel; with bulk-staged tiles
    (seg = 1) the stepped state is bitwise that of the plain tiles."""
    from paper_2406_19494_gb300.solver import Solver
    c = CASE()
    case, grid, U = padded_state(c, seed=12)
    out = []
    for seg in (0, 1):
        s = Solver(c, precision="mixed")
        s.tune_faces(0, seg)
        Ud = torch.from_numpy(U).cuda()
        s.step(Ud, 3)
        s.check()
        out.append(Ud.cpu().numpy())
    assert np.array_equal(out[0], out[1])
