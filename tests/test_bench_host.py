"""Host logic of bench.py (no GPU): the algorithmic byte model, the roofline
arithmetic and kernel choice, the traffic lookup and the reference arm's
JSON line."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bench

C2E5, F2E5 = 205379, 1584871   # the 59^3 jittered-lattice Voronoi mesh


@pytest.mark.parametrize("w,total", [(4, (720, 180)), (8, (1176, 328))])
def test_survey_bytes_per_cell_update(w, total):
    """The contract's traffic model: 720 + 180 fbar bytes per cell-update
    mixed, 1176 + 328 fbar FP64, split over gradients, face fluxes and
    gather + chemistry as its rows state."""
    fbar = F2E5 / C2E5
    rows = {4: {"k_grad": (232, 40), "k_flux": (204, 84), "gather_chem": (284, 56)},
            8: {"k_grad": (460, 64), "k_flux": (408, 160), "gather_chem": (308, 104)}}[w]
    per = {k: bench.survey_bytes(k, C2E5, F2E5, w) / C2E5 for k in ("k_grad", "k_flux", "k_gather", "k_chem")}
    for k in ("k_grad", "k_flux"):
        assert per[k] == pytest.approx(rows[k][0] + rows[k][1] * fbar, abs=1e-6), k
    a, b = rows["gather_chem"]
    assert per["k_gather"] + per["k_chem"] == pytest.approx(a + b * fbar, abs=1e-6)
    assert per["k_chem"] == 104
    assert bench.survey_bytes_per_cell_update(C2E5, F2E5, w) == pytest.approx(total[0] + total[1] * fbar, abs=1e-6)


@pytest.mark.parametrize("w,expected", [(4, {"k_grad": 621, "k_flux": 933, "k_gather": 588, "k_chem": 264}),
                                        (8, {"k_grad": 1115, "k_flux": 1804, "k_gather": 1007, "k_chem": 312})])
def test_layout_bytes_per_cell(w, expected):
    """Per cell at F/C = 7.717, B = 3: the bytes each kernel moves in this
    implementation's layout (mixed w = 4, FP64 w = 8), worked out by hand
    from the arrays it reads and writes."""
    for k, per_cell in expected.items():
        assert bench.layout_bytes(k, C2E5, F2E5, 3, w) / C2E5 == pytest.approx(per_cell, abs=0.5), k


def _res(prof, ms=None):
    return dict(C=C2E5, F=F2E5, prof=prof, ms=ms)


PK = (1.2, "measured: test")


def test_roofline_chemistry_against_fp64_peak():
    """The chemistry on top: an `alu` line, FLOP per attempt x attempts per
    launch over the mean launch time, against the measured FP64 peak;
    beside it the largest memory kernel against the HBM peak on the
    contract's bytes, and the whole subcycle's line."""
    prof = {"k_chem": (13.4, 200), "k_grad": (11.0, 200), "k_flux": (11.6, 200), "k_gather": (9.0, 200)}
    line, kern, mem, sub = bench.roofline(_res(prof, ms=45.0), "mixed", {"hbm_gbs": 6777.3}, "measured", PK,
                                          attempts=float(C2E5), n_sub=200, steps=1)
    assert line["kernel"] == "k_chem" and line["bound"] == "alu" and line["unit"] == "TFLOP/s"
    per_launch = 13.4e-3 / 200
    assert line["achieved"] == pytest.approx(bench.FP64_FLOP["mixed"]["k_chem"][0] * C2E5 / per_launch / 1e12, rel=1e-3)
    assert line["peak"] == pytest.approx(1.2)
    assert line["frac"] == pytest.approx(line["achieved"] / line["peak"], rel=1e-3)
    assert mem["kernel"] == "k_flux" and mem["bound"] == "hbm"
    gbs = bench.survey_bytes("k_flux", C2E5, F2E5, 4) / (11.6e-3 / 200) / 1e9
    assert mem["achieved"] == pytest.approx(gbs, rel=1e-3)
    assert mem["frac"] == pytest.approx(gbs / 6777.3, rel=1e-3)
    lgbs = bench.layout_bytes("k_flux", C2E5, F2E5, 3, 4) / (11.6e-3 / 200) / 1e9
    assert mem["layout_frac"] == pytest.approx(lgbs / 6777.3, rel=1e-3)
    assert kern["k_chem"]["share"] == pytest.approx(13.4 / 45.0, abs=1e-4)
    bpc = 720 + 180 * F2E5 / C2E5
    assert sub["frac"] == pytest.approx(bpc * C2E5 * 200 / 45e-3 / 1e9 / 6777.3, rel=1e-3)
    gc = kern["k_gather+k_chem"]
    assert gc["ms_per_subcycle"] == pytest.approx((13.4 + 9.0) / 200)


def test_roofline_memory_kernel_on_top_and_unlaunched_classes():
    """A memory kernel on top gives an `hbm` line; kernel classes with no
    launch are left out."""
    prof = {"k_chem": (5.0, 200), "k_grad": (11.0, 200), "k_flux": (12.0, 200), "k_gather": (9.0, 200),
            "k_unused": (0.0, 0)}
    line, kern, _, sub = bench.roofline(_res(prof), "mixed", {"hbm_gbs": 6777.3}, "measured", PK,
                                        attempts=float(C2E5))
    assert line["kernel"] == "k_flux" and line["bound"] == "hbm"
    assert "k_unused" not in kern
    assert sub is None


def test_roofline_fp64_path_is_alu_bound():
    """In the FP64 path every kernel has an FP64 FLOP count; the top one is
    reported against the FP64 peak."""
    prof = {"k_chem": (66.0, 200), "k_grad": (180.0, 200), "k_flux": (295.0, 200), "k_gather": (23.0, 200)}
    line, kern, _, _ = bench.roofline(_res(prof), "fp64", {"hbm_gbs": 6777.3}, "measured", PK,
                                      attempts=float(C2E5))
    assert line["kernel"] == "k_flux" and line["bound"] == "alu"
    f, unit = bench.FP64_FLOP["fp64"]["k_flux"]
    assert unit == "cell"
    assert line["achieved"] == pytest.approx(f * C2E5 / (295.0e-3 / 200) / 1e12, rel=1e-3)
    assert all("fp64_frac" in kern[k] for k in prof)


def test_field_errors_per_cell():
    """Both error measures: a 1e-6 relative error in a cell whose value is
    1e-5 of the field's largest is invisible to max|a-b|/max|b| (1e-11) and
    shows in the per-cell measure."""
    b = {k: np.array([1.0, 1e-5, 0.5]) for k in ("N", "F", "x5", "T")}
    a = {k: v.copy() for k, v in b.items()}
    a["N"][1] *= 1 + 1e-6
    e = bench.field_errors(a, b)
    assert e["N"]["max_rel"] == pytest.approx(1e-11, rel=1e-3)
    assert e["N"]["cell_rel"] == pytest.approx(1e-6, rel=1e-3)
    assert e["T"]["cell_rel"] == 0.0


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
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["host_cores"] == os.cpu_count()
    from oracle import oracle_threads_available
    if oracle_threads_available():
        assert cb["cores"] == os.cpu_count()
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


def test_fp64_pipe_fraction():
    """The FP64-instruction rate of an `alu` kernel over the DFMA stream's
    instruction rate (peak FLOP / 2)."""
    prof = {"k_chem": (13.4, 200), "k_grad": (11.0, 200), "k_flux": (11.6, 200), "k_gather": (9.0, 200)}
    line, kern, _, _ = bench.roofline(_res(prof), "mixed", {"hbm_gbs": 6777.3}, "measured", PK, attempts=float(C2E5))
    rate = bench.FP64_INST["mixed"]["k_chem"][0] * C2E5 / (13.4e-3 / 200)
    assert line["fp64_pipe_frac"] == pytest.approx(rate / (1.2e12 / 2), rel=1e-3)
    assert line["fp64_pipe_frac"] > line["frac"]
