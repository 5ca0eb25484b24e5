"""Host logic of bench.py (no GPU): the algorithmic byte model, the roofline
arithmetic and kernel choice, the traffic lookup and the reference arm's
JSON line."""
import json
import subprocess
import sys

import pytest

import bench

C2E5, F2E5 = 205379, 1584871   # the 59^3 jittered-lattice Voronoi mesh


@pytest.mark.parametrize("w,expected", [(4, {"k_grad": 621, "k_flux": 933, "k_gather": 684, "k_chem": 360}),
                                        (8, {"k_grad": 1115, "k_flux": 1804, "k_gather": 1007, "k_chem": 312})])
def test_algorithmic_bytes_per_cell(w, expected):
    """Per cell at F/C = 7.717, B = 3: the compulsory traffic of each kernel
    (mixed w = 4, FP64 w = 8): the per-cell compulsory traffic of each
    kernel, worked out by hand from the arrays it reads and writes."""
    for k, per_cell in expected.items():
        assert bench.algorithmic_bytes(k, C2E5, F2E5, 3, w) / C2E5 == pytest.approx(per_cell, abs=0.5), k


def _res(prof):
    return dict(C=C2E5, F=F2E5, prof=prof)


def test_roofline_chemistry_against_fp64_peak():
    """The chemistry on top: an `alu` line, FLOP per attempt x attempts per
    launch over the mean launch time, against 152 x 2 x 2 x 2.07e9 FLOP/s;
    beside it the largest memory kernel against the HBM peak."""
    prof = {"k_chem": (13.4, 200), "k_grad": (11.0, 200), "k_flux": (11.6, 200), "k_gather": (9.0, 200)}
    line, kern, mem = bench.roofline(_res(prof), "mixed", {"hbm_gbs": 6777.3}, "measured", attempts=float(C2E5))
    assert line["kernel"] == "k_chem" and line["bound"] == "alu" and line["unit"] == "TFLOP/s"
    per_launch = 13.4e-3 / 200
    assert line["achieved"] == pytest.approx(176.0 * C2E5 / per_launch / 1e12, rel=1e-3)
    assert line["peak"] == pytest.approx(1.25856, rel=1e-4)
    assert line["frac"] == pytest.approx(line["achieved"] / line["peak"], rel=1e-3)
    assert mem["kernel"] == "k_flux" and mem["bound"] == "hbm"
    gbs = bench.algorithmic_bytes("k_flux", C2E5, F2E5, 3, 4) / (11.6e-3 / 200) / 1e9
    assert mem["achieved"] == pytest.approx(gbs, rel=1e-3)
    assert mem["frac"] == pytest.approx(gbs / 6777.3, rel=1e-3)
    assert kern["k_chem"]["share"] == pytest.approx(13.4 / 45.0, abs=1e-4)


def test_roofline_memory_kernel_on_top_and_unlaunched_classes():
    """A memory kernel on top gives an `hbm` line; kernel classes with no
    launch are left out."""
    prof = {"k_chem": (5.0, 200), "k_grad": (11.0, 200), "k_flux": (12.0, 200), "k_gather": (9.0, 200),
            "k_unused": (0.0, 0)}
    line, kern, _ = bench.roofline(_res(prof), "mixed", {"hbm_gbs": 6777.3}, "measured", attempts=float(C2E5))
    assert line["kernel"] == "k_flux" and line["bound"] == "hbm"
    assert "k_unused" not in kern


def test_roofline_fp64_path_is_alu_bound():
    """In the FP64 path every kernel has an FP64 FLOP count; the top one is
    reported against the FP64 peak."""
    prof = {"k_chem": (66.0, 200), "k_grad": (180.0, 200), "k_flux": (295.0, 200), "k_gather": (23.0, 200)}
    line, kern, _ = bench.roofline(_res(prof), "fp64", {"hbm_gbs": 6777.3}, "measured", attempts=float(C2E5))
    assert line["kernel"] == "k_flux" and line["bound"] == "alu"
    f, unit = bench.FP64_FLOP["fp64"]["k_flux"]
    assert unit == "cell"
    assert line["achieved"] == pytest.approx(f * C2E5 / (295.0e-3 / 200) / 1e12, rel=1e-3)
    assert all("fp64_frac" in kern[k] for k in prof)


def test_traffic_only_for_matching_sources_and_mesh(tmp_path):
    sha = bench.source_hash()
    p = tmp_path / "t.json"
    p.write_text(json.dumps({"mixed:k_flux": {"dram_bytes_per_launch": 123, "source_sha": sha, "cells": C2E5},
                             "mixed:k_grad": {"dram_bytes_per_launch": 456, "source_sha": "0" * 16, "cells": C2E5}}))
    assert bench.ncu_traffic("k_flux", "mixed", C2E5, path=str(p)) == 123
    assert bench.ncu_traffic("k_flux", "mixed", 2097152, path=str(p)) is None   # another mesh
    assert bench.ncu_traffic("k_grad", "mixed", C2E5, path=str(p)) is None      # stale sources
    assert bench.ncu_traffic("k_gather", "mixed", C2E5, path=str(p)) is None    # not captured
    assert bench.ncu_traffic("k_flux", "mixed", C2E5, path=str(tmp_path / "missing.json")) is None


def test_reference_arm_json_line():
    """`bench.py --impl reference` times the oracle on the host and prints
    one JSON line with the contract's keys."""
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_source_hash_ignores_comments(tmp_path):
    """The traffic summary is keyed by a hash of the subcycle kernels'
    sources without comments: a comment-only edit keeps it, a code edit
    changes it, and the units that define no subcycle kernel do not enter."""
    import shutil
    root = tmp_path / "r"
    shutil.copytree(bench.ROOT + "/paper_2404_17630_gb300/csrc", root / "paper_2404_17630_gb300" / "csrc")
    h0 = bench.source_hash(str(root))
    assert h0 == bench.source_hash()
    f = root / "paper_2404_17630_gb300" / "csrc" / "rt_kernels.cuh"
    f.write_text(f.read_text() + "\n/* a note */\n// another\n")
    assert bench.source_hash(str(root)) == h0
    g = root / "paper_2404_17630_gb300" / "csrc" / bench.NOT_SUBCYCLE[1]
    g.write_text(g.read_text() + "\nint rt_unused_symbol;\n")
    assert bench.source_hash(str(root)) == h0
    f.write_text(f.read_text() + "\nint rt_unused_symbol;\n")
    assert bench.source_hash(str(root)) != h0
    assert bench.code_text("a = 1; // x\n/* y\n z */ b = 2;\n\n") == "a = 1;\n  b = 2;"
