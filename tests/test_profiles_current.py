"""The bench's measured-counter fields come from committed ncu captures that carry a hash of the
kernel sources they were taken on (profiles/k_face_traffic.json for the FP64 face kernels'
DRAM traffic, profiles/mixed_step_counters.json for the mixed path's whole-step floors).  They
must match the sources as committed, so that the bench line reports them instead of null, and
the floors they give must be the ones the profile summary states."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CELLS = 128 ** 3


def test_fp64_face_traffic_capture_is_current():
    t = bench.face_traffic(CELLS)
    assert t is not None
    info = json.load(open(os.path.join(ROOT, "profiles", "k_face_traffic.json")))
    assert len(info["dram_bytes_per_launch"]) == 3
    # the x, y and z launches move between the compulsory 120-160 B and 300 B per cell
    for b in info["dram_bytes_per_launch"]:
        assert 100 * CELLS < b < 300 * CELLS


def test_mixed_step_counters_are_current_and_consistent():
    r = bench.mixed_step_roofline(2.0, CELLS)
    assert r is not None
    info = json.load(open(os.path.join(ROOT, "profiles", "mixed_step_counters.json")))
    kinds = [l["kernel"].split("<")[0] for l in info["launches"]]
    # one single-step call: primitives, CFL partials, and per stage gradients + x, y, z faces
    # (the last with the stage), with the halo pass after the first two stages
    assert kinds.count("k_face_mixed_x") == 3 and kinds.count("k_face_mixed_ts") == 3
    assert kinds.count("k_prim_bc") == 1 and kinds.count("k_halo_prim") == 2
    floors = r["floors_ms"]
    assert r["bound"] == max(floors, key=floors.get) and r["floor_ms"] == floors[r["bound"]]
    assert abs(r["frac"] - r["floor_ms"] / 2.0) < 1e-12
    # the summary states the same floors (two decimals)
    md = open(os.path.join(ROOT, "profiles", "k_face_mixed_tgv128_step.md")).read()
    assert info["source_sha256_16"] in md
    for k in ("fp64_pipe", "issue", "hbm"):
        assert "%.2f ms" % floors[k] in md.replace("\n", " ")


def test_roofline_is_none_when_a_capture_is_stale(tmp_path, monkeypatch):
    src = json.load(open(os.path.join(ROOT, "profiles", "mixed_step_counters.json")))
    src["source_sha256_16"] = "0" * 16
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "mixed_step_counters.json").write_text(json.dumps(src))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the kernel sources are read from ROOT as well: point them at the real tree
    csrc = os.path.join(ROOT, "paper_2406_19494_gb300")
    os.symlink(csrc, tmp_path / "paper_2406_19494_gb300")
    assert bench.mixed_step_roofline(2.0, CELLS) is None
