"""Host logic of the benchmark's multi-GPU mode: every rank advances one z-slab of a solve that is
the workload extended N times along z (weak scaling), the job time is the slowest rank's and the
rate counts every rank's cells.  Checked here with two gloo ranks on the CPU; the slabs' halo
exchange itself is covered by test_decomposition_host.py (gloo) and test_gpu_decomposition.py."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
    job_ms = bench.max_over_ranks(ms, "cpu")
    out[rank] = (ws, r, local, job_ms, bench.whole_job_rate(1000, 4, ws, job_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank_and_count_all_cells():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][:3] == (2, 0, 0) and res[1][:3] == (2, 1, 1)
    assert res[0][3] == res[1][3] == 15.0
    assert res[0][4] == res[1][4] == pytest.approx(1000 * 4 * 2 / 15e-3)


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, "cpu") == 12.5
    assert bench.whole_job_rate(100, 10, 1, 1000.0) == pytest.approx(1000.0)


def test_slab_case_extends_the_workload_along_z():
    import bench
    from paper_2406_19494_gb300 import decomp
    base = bench.WORKLOADS["tgv64"]()
    c = bench.slab_case(base, 4)
    assert c["n"] == (64, 64, 256) and c["hi"][2] == pytest.approx(4 * base["hi"][2])
    for r in range(4):
        lay = decomp.Layout(c, (1, 1, 4), r)
        assert lay.n == [64, 64, 64] and lay.offset[2] == 64 * r
        assert lay.local_case()["bc"][2] == ("exchange", "exchange")
