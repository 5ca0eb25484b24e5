"""Benchmark of the M1 RT subcycle on GB300: RT cell-updates/s per subcycle
(3 bins), mixed FP32/FP64 and FP64, with the HBM-roofline fraction of the
dominant kernel, an end-to-end number through the C ABI with host buffers,
and the FP64 CPU oracle timed on the host as a reported baseline.

Workload (one step = one rt_step of 200 subcycles): periodic Voronoi mesh of a
59^3 jittered lattice (205,379 cells, jitter 0.3 h, box 10 kpc), lognormal
n_H (median 1e-3 cm^-3, sigma_ln 1), neutral H+He gas (Y = 0.24) at 1e4 K,
16 sources with log10 Q ~ U(48, 51) split over the HI/HeI/HeII bins,
c_red = 0.01 c, CFL 0.3, full chemistry.  The simulation runs on from step to
step (warm-up steps included).  The working set is larger than the 129 MB L2.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
N > 1: one process per GPU (torchrun), independent replicas, max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RT cell-updates/s per subcycle (3 bins), FP64 vs mixed; % of HBM roofline"
UNIT = "cell-updates/s"
N_SUB = 200
LATTICE = 59
L_BOX = 10.0
L2_BYTES = 129e6


def thesan_like(n=128, seed=4, n_peaks=4096):
    """THESAN-like box (the recipe is synth.thesan_like): 128^3 jittered
    lattice, 3.58 Mpc, exp(GRF) density, 4096 peak sources, c_red = 0.2 c."""
    import synth
    return synth.thesan_like(n, seed, n_peaks)


def differentiable(n=64, seed=7, n_src=8):
    """Differentiable workload: n^3 jittered-lattice Voronoi mesh (box 10 kpc),
    lognormal n_H (sigma_ln 1), 8 sources with Q ~ U(1e49, 1e50) photons/s,
    full H+He network with thermal energy, FP64; loss = mass-weighted ionised
    fraction of the cells whose generators lie in the 16^3-lattice sub-cube
    centred on the first source."""
    import synth
    mesh = synth.voronoi_mesh(n, L_BOX, 0.3, seed=seed)
    C = mesh.n_cells
    nH = synth.lognormal_density(C, 1e-3, 1.0, seed + 1)
    srng = np.random.default_rng(seed + 2)
    cells = srng.choice(C, size=n_src, replace=False).astype(np.int64)
    Q = np.outer(srng.uniform(1e49, 1e50, n_src), synth.SPECTRAL_SPLIT_E4)
    x5 = np.zeros((5, C)); x5[0] = 1.0; x5[2] = 1.0
    cfg = dict(n_bins=3, c_red=0.01 * synth.C_LIGHT, unit_length_cm=synth.KPC_CM, box=L_BOX, cfl=0.3, chem_mode=2,
               chem_flags=15, limiter=1, lim_eps=1e-5, order=2, f_s=0.05, f_max=0.1, x_floor=1e-4,
               max_substeps=10000, y_he=synth.helium_ratio(0.24), sigma=synth.GREY_SIGMA, eps=synth.GREY_EPS)
    idx = np.arange(C)
    ijk = np.stack([idx % n, (idx // n) % n, idx // (n * n)], 1)
    d = (ijk - ijk[cells[0]] + n // 2) % n - n // 2      # periodic lattice offset from the first source
    region = np.all((d >= -8) & (d < 8), axis=1)
    state = dict(nH=nH, x5=x5, T=np.full(C, 1e4), N=np.zeros((3, C)), fr=np.zeros((3, 3, C)), cells=cells, Q=Q,
                 region=region)
    return mesh, cfg, state


def workload(n=LATTICE, seed=1, n_src=16):
    """Seeded inputs of the 2e5-cell Voronoi workload (see module doc)."""
    import synth
    mesh = synth.voronoi_mesh(n, L_BOX, 0.3, seed=seed)
    C = mesh.n_cells
    nH = synth.lognormal_density(C, 1e-3, 1.0, seed + 1)
    x5 = np.zeros((5, C)); x5[0] = 1.0; x5[2] = 1.0
    T = np.full(C, 1e4)
    srng = np.random.default_rng(seed + 2)
    cells = srng.choice(C, size=n_src, replace=False).astype(np.int64)
    Q = np.outer(10 ** srng.uniform(48, 51, n_src), synth.SPECTRAL_SPLIT_E4)
    cfg = dict(n_bins=3, c_red=0.01 * synth.C_LIGHT, unit_length_cm=synth.KPC_CM, box=L_BOX, cfl=0.3, chem_mode=2,
               chem_flags=15, limiter=1, lim_eps=1e-5, order=2, f_s=0.05, f_max=0.1, x_floor=1e-4,
               max_substeps=10000, y_he=synth.helium_ratio(0.24), sigma=synth.GREY_SIGMA, eps=synth.GREY_EPS)
    state = dict(nH=nH, x5=x5, T=T, N=np.zeros((3, C)), fr=np.zeros((3, 3, C)), cells=cells, Q=Q)
    return mesh, cfg, state


# ---------------------------------------------------------------------------
# algorithmic bytes per launch
# ---------------------------------------------------------------------------

def survey_bytes(kernel, C, F, w):
    """Compulsory bytes of one launch under the hot-path contract's traffic
    model (each array streamed once per kernel that needs it, neighbour
    re-reads hitting L2; per cell with fbar = F/C faces per cell; w = 8 FP64,
    4 mixed; CSR ids and face L/R int32):
      gradients  prim 12w + M^-1 6w + s 3w + G out 36w + CSR (4 + 8 fbar)
                 + faces (L/R 8 + w_f 3w + x_f 3w) fbar
      face flux  prim + G of the cells 48w + s 3w + faces (8 + (A, n, x_f) 7w)
                 fbar + flux out 12w fbar
      gather + chemistry  CSR (4 + 8 fbar) + flux in 12w fbar + 1/V 8
                 + radiation master r/w (FP64 192; mixed: N FP64 + F/c FP32
                 r/w 120 + FP32 shadow out 48) + chemistry state r/w 104
    Totals: FP64 1176 + 328 fbar, mixed 720 + 180 fbar per cell-update.  The
    gather and the chemistry are two kernels here: the chemistry gets its
    104 bytes of state, the flux application the rest of that row."""
    rad = 192 if w == 8 else 168
    if kernel == "k_grad":
        return (57 * w + 4) * C + (16 + 6 * w) * F
    if kernel == "k_flux":
        return 51 * w * C + (8 + 19 * w) * F
    if kernel == "k_gather":
        return (4 + 8 + rad) * C + (8 + 12 * w) * F
    if kernel == "k_chem":
        return 104 * C
    raise KeyError(kernel)


def survey_bytes_per_cell_update(C, F, w):
    """720 + 180 fbar (mixed) or 1176 + 328 fbar (FP64) bytes."""
    return sum(survey_bytes(k, C, F, w) for k in ("k_grad", "k_flux", "k_gather", "k_chem")) / C


def layout_bytes(kernel, C, F, B, w):
    """Bytes one launch moves in this implementation's data layout (each
    array it touches read or written once; w = bytes per word of the
    transport sweep, 8 FP64, 4 mixed).  Reported beside the contract's
    model: it counts the offsets x_f - s of both sides and the gradient
    records as laid out, so it is larger."""
    if kernel == "k_grad":
        # prim 4wBC, M^-1 6wC, offsets 4C, CSR 8F, face ids 8F, w_f 3wF,
        # x_f - s_L and x_f - s_R 6wF, gradients out 12wBC
        return (16 * w * B + 6 * w + 4) * C + (16 + 9 * w) * F
    if kernel == "k_flux":
        # face ids 8F, (n, A) 4wF, x_f - s 6wF, prim + gradients of the
        # cells 16wBC, fluxes out 4wBF
        return (8 + 10 * w + 4 * w * B) * F + 16 * w * B * C
    # radiation state r/w per (cell, bin): FP64 records 64 B; mixed: N in
    # FP64 16 B + the FP32 sweep record (N, F / c) 32 B
    rad = 64 if w == 8 else 48
    if kernel == "k_gather":
        # offsets 4C, CSR 8F, fluxes 4wBF, V (or 1/V) 8C, radiation state r/w
        return 4 * C + 8 * F + 4 * w * B * F + 8 * C + rad * B * C
    if kernel == "k_chem":
        # radiation state r/w, V 8C, source ids 4C, n_H 8C, abundances r/w
        # 80C, T r/w 16C, substep counts 4C
        return rad * B * C + 8 * C + 4 * C + 8 * C + 80 * C + 16 * C + 4 * C
    raise KeyError(kernel)


def code_text(src):
    """C/C++/CUDA source without its comments and blank lines (string
    literals, which hold no comment markers in these sources, are kept)."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


# Translation units that define no subcycle kernel (the allocation-free
# gradient entry point, the failure-path check and the FP64 peak
# measurement): they are left out of the hash that dates the counter
# summaries.
NOT_SUBCYCLE = ("rt_noalloc.cu", "rt_selftest.cu", "rt_peak.cu")


def source_hash(root=None):
    """Hash of the sources of the subcycle kernels and their launches
    (`csrc/` but the units in NOT_SUBCYCLE), comments excluded: a counter
    summary stays valid across comment-only edits and changes elsewhere."""
    root = root or ROOT
    h = hashlib.sha256()
    d = os.path.join(root, "paper_2404_17630_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")) and name not in NOT_SUBCYCLE:
            with open(os.path.join(d, name), encoding="utf-8") as f:
                h.update(code_text(f.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, precision, cells, path=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    from the current kernel sources on a mesh of this many cells; else None
    (traffic does not scale in proportion between meshes that do and do not
    fit in L2)."""
    path = path or os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    ent = d.get(f"{precision}:{kernel}")
    if not ent or ent.get("source_sha") != source_hash() or ent.get("cells") != cells:
        return None
    return ent.get("dram_bytes_per_launch")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0])); mx.append(float(p[1]))
            except ValueError:
                continue
            for k, v in zip(names, p[3:7]):
                if v.lower() == "active":
                    reasons.add(k)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def l2_flush(buf):
    buf.add_(1.0)


def max_over_ranks(ms, dist, device):
    """The timed region's length on the slowest rank (replicas: every rank
    times the same work on its own GPU; no data is exchanged)."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, cells, n_sub, steps, ms):
    """Whole-job cell-updates/s: the cells all ranks advanced over the
    slowest rank's time (weak scaling: each replica holds the whole mesh)."""
    return world * cells * n_sub * steps / (ms / 1e3)


def run_gpu(precision, mesh, cfg, state, steps, warmup, rank, world, dev, dist, clocks=None, gather_sum=1):
    import torch
    from paper_2404_17630_gb300 import RT, make_config
    from paper_2404_17630_gb300 import rt as rtb

    stream = torch.cuda.current_stream(dev)
    rt = RT(make_config(precision=precision, gather_sum=gather_sum, **cfg), mesh, stream=stream)
    rt.set_gas(state["nH"], state["x5"], state["T"])
    rt.set_radiation(state["N"], state["fr"] * cfg["c_red"])
    rt.set_sources(state["cells"], state["Q"])
    dt = rt.max_dt() * N_SUB
    flush = torch.empty(int(2 * L2_BYTES / 4), dtype=torch.float32, device=dev)
    for _ in range(warmup):
        rt.step(dt, N_SUB)
    rt.sync()
    l2_flush(flush)
    n0 = rtb.rt_launch_count(rt.ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ctx = clocks if clocks is not None else _Null()
    with ctx:
        ev0.record(stream)
        for _ in range(steps):
            rt.step(dt, N_SUB)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    rt.sync()
    ms = ev0.elapsed_time(ev1)
    launches = rtb.rt_launch_count(rt.ctx) - n0
    ms = max_over_ranks(ms, dist, dev)
    # per-kernel device times over the same number of steps (profiled pass)
    rtb.rt_profile_read(rt.ctx, reset=True)
    rtb.rt_profile_enable(rt.ctx, True)
    for _ in range(steps):
        rt.step(dt, N_SUB)
    prof = rtb.rt_profile_read(rt.ctx, reset=True)
    rtb.rt_profile_enable(rt.ctx, False)
    rt.sync()
    C, F, _ = rt.mesh_info()
    attempts = float(rt.fields()["nsub"].sum())  # chemistry attempts of the last subcycle
    return dict(ms=ms, C=C, F=F, launches=launches, prof=prof, rt=rt, attempts=attempts)


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def e2e_measure(precision, mesh, cfg, state, steps, warmup, dev):
    """The same metric through the C ABI with host buffers: every step copies
    the whole state in from pinned host memory, runs the 200 subcycles and
    copies all fields back into the same host buffers, so the run evolves as
    the device-resident one does (warm-up steps first)."""
    import torch
    from paper_2404_17630_gb300 import RT, make_config
    from paper_2404_17630_gb300 import rt as rtb

    stream = torch.cuda.current_stream(dev)
    rt = RT(make_config(precision=precision, gather_sum=1, **cfg), mesh, stream=stream)
    rt.set_sources(state["cells"], state["Q"])
    C, B = mesh.n_cells, 3
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
    hN, hF = pin(state["N"]), pin(state["fr"] * cfg["c_red"])
    hn, hx, hT = pin(state["nH"]), pin(state["x5"]), pin(state["T"])
    dt = rt.max_dt() * N_SUB
    mask = rtb.RT_FIELD_N | rtb.RT_FIELD_F | rtb.RT_FIELD_X | rtb.RT_FIELD_T

    def one():
        rtb.rt_set_radiation(rt.ctx, hN, hF)
        rtb.rt_set_gas(rt.ctx, hn, hx, hT)
        rtb.rt_step(rt.ctx, dt, N_SUB)
        rtb.rt_get_fields(rt.ctx, mask, [hN, hF, hx, hT])

    for _ in range(warmup):
        one()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize(dev)
    sec = time.perf_counter() - t0
    h2d = (hN.numel() + hF.numel() + hn.numel() + hx.numel() + hT.numel()) * 8
    d2h = (hN.numel() + hF.numel() + hx.numel() + hT.numel()) * 8
    return dict(value=C * N_SUB * steps / sec, unit=UNIT, h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                ms_per_step=1e3 * sec / steps)


# FP64 work of the kernels the FP64 unit bounds, from ncu on the 2e5-cell
# workload in steady state (FLOP = 2 x DFMA + DMUL + DADD thread
# instructions): per chemistry attempt for k_chem (one attempt per cell in
# steady state), per cell for the FP64 sweep kernels.  The unit counts behind
# the `alu` rooflines; re-measured after each change of these kernels.
FP64_FLOP = {
    "mixed": {"k_chem": (159.0, "attempt")},
    "fp64": {"k_chem": (1238.0, "attempt"), "k_grad": (2762.4, "cell"), "k_flux": (5673.8, "cell"),
             "k_gather": (439.4, "cell")},
}
# FP64-pipe instructions (thread instructions on the FP64 pipe, ncu
# sm__inst_executed_pipe_fp64 x 32) per unit, from the same captures.  A
# kernel's instruction mix holds DMUL and DADD beside DFMA, so its FLOP rate
# at a saturated FP64 pipe is below the DFMA-stream peak; the instruction
# rate against the stream's (peak FLOP / 2 per DFMA) is the pipe's use.
FP64_INST = {
    "mixed": {"k_chem": (109.1, "attempt")},
    "fp64": {"k_chem": (801.0, "attempt"), "k_grad": (1944.5, "cell"), "k_flux": (3803.6, "cell"),
             "k_gather": (282.0, "cell")},
}
# Fallback FP64 peak from unit counts and clock, used only when the
# measurement (rt_fp64_peak) is not available: 152 SMs x 2 FP64 FMA lanes per
# clock per SM (ncu: 16 cycles per warp instruction on the FP64 pipe) x 2 FLOP
# x 2.07 GHz = 1.259 TFLOP/s.
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.07e9 / 1e12


def fp64_peak(stream=None):
    """(TFLOP/s, source): the measured FMA-stream peak of this device
    (rt_fp64_peak, best of 5 launches of ~16 ms), else the derived figure."""
    try:
        from paper_2404_17630_gb300 import rt as rtb
        tf, ms = rtb.rt_fp64_peak(stream, 4096, 5)
        return tf, f"measured: rt_fp64_peak DFMA stream, best of 5 launches ({ms:.2f} ms each)"
    except Exception as e:  # noqa: BLE001 -- reported, then the derived figure
        return FP64_PEAK_DERIVED, f"derived (152 SMs x 2 FMA lanes/clk x 2 x 2.07 GHz); measurement failed: {e}"


def roofline(res, precision, peaks, peak_kind, fp64pk, attempts=None, n_sub=None, steps=None):
    """Per-kernel rooflines.  Bytes are the contract's traffic model
    (survey_bytes); this layout's own bytes are reported beside them
    (`layout_*`).  A kernel whose FP64 work is known (FP64_FLOP) is also
    reported against the measured FP64 peak (`alu`): the chemistry, and every
    kernel of the FP64 path.  Returns the line of the kernel with the largest
    time share (`alu` if it is FP64-bound, else `hbm`), the per-kernel table,
    the largest memory-bound kernel's `hbm` line and the whole subcycle's."""
    C, F, B = res["C"], res["F"], 3
    w = 4 if precision == "mixed" else 8
    prof = {k: v for k, v in res["prof"].items() if v[1] > 0}
    total = sum(v[0] for v in prof.values())
    shares = {k: (v[0] / total if total else 0.0) for k, v in prof.items()}
    peak = float(peaks["hbm_gbs"])
    fpk, fsrc = fp64pk
    kern = {}
    for k, v in prof.items():
        ms = v[0] / max(v[1], 1)
        sb, lb = survey_bytes(k, C, F, w), layout_bytes(k, C, F, B, w)
        kern[k] = {"ms_per_launch": ms, "launches": v[1], "share": round(shares[k], 4),
                   "alg_bytes_per_launch": sb, "GBs": sb / (ms / 1e3) / 1e9 if ms else None,
                   "layout_bytes_per_launch": lb, "layout_GBs": lb / (ms / 1e3) / 1e9 if ms else None}
        kern[k]["hbm_frac"] = round(kern[k]["GBs"] / peak, 4) if kern[k]["GBs"] else None
    units = {"cell": C, "attempt": attempts if attempts else C}
    flops = FP64_FLOP.get(precision, {})
    insts = FP64_INST.get(precision, {})
    for k in kern:
        if k in flops and kern[k]["ms_per_launch"] > 0:
            f, u = flops[k]
            tf = f * units[u] / (kern[k]["ms_per_launch"] / 1e3) / 1e12
            kern[k]["fp64_tflops"] = round(tf, 4)
            kern[k]["fp64_frac"] = round(tf / fpk, 4)
        if k in insts and kern[k]["ms_per_launch"] > 0:
            n, u = insts[k]
            rate = n * units[u] / (kern[k]["ms_per_launch"] / 1e3)     # FP64 thread instructions / s
            kern[k]["fp64_pipe_frac"] = round(rate / (fpk * 1e12 / 2), 4)
    parts = [k for k in ("k_gather", "k_chem") if k in prof]
    if "k_grad" in prof and parts:
        # the contract's gather + chemistry row over the time of the two
        # kernels that do it, per subcycle
        ms = sum(prof[k][0] for k in parts) / prof["k_grad"][1]
        sb = survey_bytes("k_gather", C, F, w) + survey_bytes("k_chem", C, F, w)
        kern["k_gather+k_chem"] = {"ms_per_subcycle": ms, "alg_bytes_per_launch": sb, "kernels": parts,
                                   "GBs": sb / (ms / 1e3) / 1e9, "hbm_frac": round(sb / (ms / 1e3) / 1e9 / peak, 4)}

    def hbm_line(k):
        return {"kernel": k, "bound": "hbm", "achieved": round(kern[k]["GBs"], 1), "peak": peak, "unit": "GB/s",
                "frac": kern[k]["hbm_frac"], "peak_source": f"hbm_gbs of {peak_kind}",
                "traffic": ncu_traffic(k, precision, C), "alg_bytes_per_launch": kern[k]["alg_bytes_per_launch"],
                "bytes_model": "contract (survey) traffic model",
                "layout_bytes_per_launch": kern[k]["layout_bytes_per_launch"],
                "layout_frac": round(kern[k]["layout_GBs"] / peak, 4)}

    top = max(prof, key=lambda k: prof[k][0])
    mem = [k for k in prof if k != "k_chem"]
    top_mem = max(mem, key=lambda k: prof[k][0])
    if top in flops:
        f, u = flops[top]
        line = {"kernel": top, "bound": "alu", "achieved": kern[top]["fp64_tflops"], "peak": round(fpk, 4),
                "unit": "TFLOP/s", "frac": kern[top]["fp64_frac"], "peak_source": fsrc,
                "fp64_pipe_frac": kern[top].get("fp64_pipe_frac"),
                "fp64_pipe_note": "FP64 instructions per second over the DFMA stream's (its mix of DMUL and DADD "
                                  "beside DFMA does fewer FLOP per instruction)",
                "traffic": ncu_traffic(top, precision, C), "alg_flop_per_launch": f * units[u], "flop_per_" + u: f,
                u + "s_per_launch": units[u], "alg_bytes_per_launch": kern[top]["alg_bytes_per_launch"],
                "hbm_frac_of_alg_bytes": kern[top]["hbm_frac"]}
    else:
        line = hbm_line(top)
    sub = None
    if n_sub and steps and res.get("ms"):
        bpc = survey_bytes_per_cell_update(C, F, w)
        gbs = bpc * C * n_sub * steps / (res["ms"] / 1e3) / 1e9
        sub = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
               "bytes_per_cell_update": round(bpc, 1), "faces_per_cell": round(F / C, 4),
               "bytes_model": "contract (survey): 720 + 180 fbar mixed, 1176 + 328 fbar FP64",
               "peak_source": f"hbm_gbs of {peak_kind}"}
    return line, kern, hbm_line(top_mem), sub


def _oracle_rate(mesh, cfg, state, threads, budget_s, max_sub=50):
    """Cell-updates/s of the FP64 oracle as it stands on the full mesh from
    the workload's initial state: subcycles until ~budget_s."""
    from oracle import Oracle, default_config
    o = Oracle(default_config(**cfg), mesh, threads=threads)
    o.set_radiation(state["N"], state["fr"])
    o.set_gas(state["nH"], state["x5"], state["T"])
    o.set_sources(state["cells"], state["Q"])
    dt = o.max_dt()
    t0 = time.perf_counter()
    n = 0
    while True:
        o.step(dt, 1)
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= max_sub:
            break
    sec = time.perf_counter() - t0
    return mesh.n_cells * n / sec, n, sec, o.threads


def cpu_baseline(mesh, cfg, state, budget_s=10.0):
    """The FP64 oracle as it stands on the host cores, on the same workload:
    all host cores (the OpenMP build of the same source, bitwise the same
    results) and one thread, each on subcycles of the full mesh until
    ~budget_s."""
    from oracle import oracle_threads_available
    host = os.cpu_count() or 1
    v1, n1, s1, _ = _oracle_rate(mesh, cfg, state, 1, budget_s)
    single = {"value": v1, "unit": UNIT, "cores": 1,
              "sample": f"{n1} subcycles of the full {mesh.n_cells}-cell workload from its initial state "
                        f"({s1:.1f} s, FP64, one thread)"}
    if host > 1 and oracle_threads_available():
        v, n, sec, th = _oracle_rate(mesh, cfg, state, 0, budget_s)
        return {"value": v, "unit": UNIT, "cores": th, "host_cores": host, "kind": "oracle",
                "sample": f"{n} subcycles of the full {mesh.n_cells}-cell workload from its initial state "
                          f"({sec:.1f} s, FP64, {th} threads: the OpenMP build of the oracle source)",
                "single_thread": single, "speedup_all_cores_over_one": round(v / v1, 2)}
    return dict(single, kind="oracle", host_cores=host)


def field_errors(a, b):
    """Per field (N, F, x5, T) of a against b: the largest |a - b| over the
    field's largest |b| (max_rel), and the largest per-cell relative error
    |a - b| / |b| over the cells where |b| > 1e-30 max|b| (cell_rel) and
    where |b| > 1e-6 max|b| (cell_rel_1e-6: beyond the light front a cell's
    photons are exponentially few, and its relative error measures nothing
    the transport decides)."""
    out = {}
    for k in ("N", "F", "x5", "T"):
        x, y = np.asarray(a[k], dtype=np.float64), np.asarray(b[k], dtype=np.float64)
        m = float(np.abs(y).max())
        d = np.abs(x - y)
        e = {"max_rel": float(d.max() / m) if m > 0 else float(d.max())}
        for key, th in (("cell_rel", 1e-30), ("cell_rel_1e-6", 1e-6)):
            sel = np.abs(y) > th * m
            e[key] = float((d[sel] / np.abs(y[sel])).max()) if sel.any() else 0.0
        out[k] = e
    return out


def measure_large(steps, warmup, dev, fp64pk, n_sub=100):
    """Mixed precision on the 2.1M-cell THESAN-like box, 100 subcycles/step;
    the FP64 path timed on one step of the same subcycles from the same
    initial state, and the per-field error of the mixed path against it."""
    t0 = time.perf_counter()
    mesh, cfg, state = thesan_like()
    build_s = time.perf_counter() - t0
    import torch
    from paper_2404_17630_gb300 import RT, make_config
    from paper_2404_17630_gb300 import rt as rtb
    stream = torch.cuda.current_stream(dev)

    def fresh(prec):
        r = RT(make_config(precision=prec, gather_sum=1, **cfg), mesh, stream=stream)
        r.set_gas(state["nH"], state["x5"], state["T"])
        r.set_radiation(state["N"], state["fr"] * cfg["c_red"])
        r.set_sources(state["cells"], state["Q"])
        return r

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_step(r, dt):
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        r.step(dt, n_sub)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        return ev0.elapsed_time(ev1)

    # first step of each precision from the initial state: the error of the
    # mixed path against the FP64 path, and the FP64 path's time
    fields, first_ms = {}, {}
    for prec in ("fp64", "mixed"):
        r2 = fresh(prec)
        dt = r2.max_dt() * n_sub
        r2.step(dt, n_sub)   # builds the step graph outside the timed step
        r2.sync()
        r2.set_gas(state["nH"], state["x5"], state["T"])     # back to the initial state
        r2.set_radiation(state["N"], state["fr"] * cfg["c_red"])
        first_ms[prec] = timed_step(r2, dt)
        r2.sync()
        fields[prec] = r2.fields()
        del r2
    # mixed: steady-state steps
    rt = fresh("mixed")
    dt = rt.max_dt() * n_sub
    for _ in range(warmup):
        rt.step(dt, n_sub)
    rt.sync()
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(steps):
        rt.step(dt, n_sub)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    rtb.rt_profile_read(rt.ctx, reset=True)
    rtb.rt_profile_enable(rt.ctx, True)
    rt.step(dt, n_sub)
    prof = rtb.rt_profile_read(rt.ctx, reset=True)
    rtb.rt_profile_enable(rt.ctx, False)
    rt.sync()
    C, F, _ = rt.mesh_info()
    res = dict(ms=ms, C=C, F=F, prof=prof)
    peaks, kind = measured_peaks()
    f = rt.fields()
    rf, kern, rf_mem, rf_sub = roofline(res, "mixed", peaks, kind, fp64pk, attempts=float(f["nsub"].sum()),
                                        n_sub=n_sub, steps=steps)
    v_mixed = C * n_sub * steps / (ms / 1e3)
    v64_first = C * n_sub / (first_ms["fp64"] / 1e3)
    v_mixed_first = C * n_sub / (first_ms["mixed"] / 1e3)
    return {"workload": f"THESAN-like voronoi 128^3 ({C} cells, {F} faces), GRF n_H, 4096 peak sources, "
                        f"c_red 0.2c, {n_sub} subcycles/step, mixed",
            "mixed_vs_fp64_after_one_step": {"metric": "per field: max|mixed - fp64| / max|fp64| (max_rel) and "
                                                       "max over cells of |mixed - fp64| / |fp64| where "
                                                       "|fp64| > 1e-30 max|fp64| (cell_rel), > 1e-6 max|fp64| "
                                                       "(cell_rel_1e-6)",
                                             **field_errors(fields["mixed"], fields["fp64"])},
            "value": v_mixed, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
            "fp64_first_step": {"value": v64_first, "ms": first_ms["fp64"]},
            "mixed_first_step": {"value": v_mixed_first, "ms": first_ms["mixed"]},
            "speedup_mixed_over_fp64_first_step": round(v_mixed_first / v64_first, 2),
            "roofline": rf, "roofline_memory_kernel": rf_mem, "roofline_subcycle": rf_sub,
            "kernels": kern, "mesh_build_s": round(build_s, 1), "x_HII_mean": float(f["x5"][1].mean())}


def measure_hii(steps, warmup, dev, n=64, n_sub=64):
    """Mixed precision on the expanding-HII-region workload: staggered 2 x n^3
    grid (truncated octahedra), 3 bins, 64 subcycles per step."""
    import synth
    import torch
    from paper_2404_17630_gb300 import RT, make_config
    from paper_2404_17630_gb300 import rt as rtb
    mesh, cfg, state = synth.hii_region(n)
    stream = torch.cuda.current_stream(dev)
    rt = RT(make_config(precision="mixed", gather_sum=1, **cfg), mesh, stream=stream)
    rt.set_gas(state["nH"], state["x5"], state["T"])
    rt.set_radiation(state["N"], state["fr"] * cfg["c_red"])
    rt.set_sources(state["cells"], state["Q"])
    dt = rt.max_dt() * n_sub
    for _ in range(warmup):
        rt.step(dt, n_sub)
    rt.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(steps):
        rt.step(dt, n_sub)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    rt.sync()
    rtb.rt_profile_read(rt.ctx, reset=True)
    rtb.rt_profile_enable(rt.ctx, True)
    rt.step(dt, n_sub)
    prof = rtb.rt_profile_read(rt.ctx, reset=True)
    rtb.rt_profile_enable(rt.ctx, False)
    rt.sync()
    C, F, _ = rt.mesh_info()
    f = rt.fields()
    nsub = f["nsub"]
    return {"kernels_ms_per_launch": {k: round(v[0] / max(v[1], 1), 5) for k, v in prof.items()},
            "chem_attempts_last_subcycle": {"mean": float(nsub.mean()), "max": int(nsub.max()),
                                            "cells_above_1": int((nsub > 1).sum())},
            "workload": f"expanding HII region, staggered 2x{n}^3 grid ({C} cells, {F} faces, 7 faces/cell), "
                        f"r^-2 density, 3 bins, c_red 1e-3 c, {n_sub} subcycles/step, mixed",
            "value": C * n_sub * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "warmup": warmup, "t_Myr": (warmup + steps) * dt / 3.15576e13,
            "ionised_volume_fraction": float((f["x5"][1] * mesh.volume).sum() / mesh.volume.sum())}


def measure_timebins(dev, n_steps=8):
    """Individual time steps on the 2e5-cell workload (mixed): the cells on a
    four-level power-of-two hierarchy (10% in the shortest level, then 20%,
    30%, 40%), ranked by a spatially correlated field as the time steps of
    a simulation follow its density structure: a Gaussian random field
    (P(k) ~ k^-2) on a 16^3 grid, ties of its nearest-node sampling broken by
    a 64^3 one; level k is active in steps divisible by 2^k.  Reports active
    cell-updates/s and the time against all-active steps."""
    import torch
    import synth
    from paper_2404_17630_gb300 import RT, make_config
    mesh, cfg, state = workload()
    C = mesh.n_cells
    coarse, _ = synth.grf_density(mesh.gen, L_BOX, 16, 1.5, 1.0, 77)
    fine, _ = synth.grf_density(mesh.gen, L_BOX, 64, 1.5, 1.0, 78)
    order = np.argsort(-(np.log(coarse) + 0.05 * np.log(fine)), kind="stable")
    level = np.empty(C, np.int64)
    cuts = np.cumsum([int(0.1 * C), int(0.2 * C), int(0.3 * C)])
    level[order] = np.searchsorted(cuts, np.arange(C), side="right")
    stream = torch.cuda.current_stream(dev)
    rt = RT(make_config(precision="mixed", gather_sum=1, **cfg), mesh, stream=stream)
    rt.set_gas(state["nH"], state["x5"], state["T"])
    rt.set_radiation(state["N"], state["fr"] * cfg["c_red"])
    rt.set_sources(state["cells"], state["Q"])
    dt = rt.max_dt() * N_SUB
    for _ in range(2):
        rt.step(dt, N_SUB)
    rt.sync()
    masks = [(level <= max(k for k in range(4) if s % (2 ** k) == 0)) for s in range(n_steps)]
    # one untimed cycle: each level's lists and step graph are built once and
    # kept (rt_set_active caches the sets of a hierarchy)
    for m in masks:
        rt.set_active(m)
        rt.step(dt, N_SUB)
    rt.set_active(None)
    rt.step(dt, N_SUB)
    rt.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # all-active steps first (two untimed to settle), then the hierarchy cycle
    for _ in range(2):
        rt.step(dt, N_SUB)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(n_steps):
        rt.step(dt, N_SUB)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms_all = ev0.elapsed_time(ev1)
    ms_masked = 0.0
    for m in masks:
        rt.set_active(m)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        rt.step(dt, N_SUB)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms_masked += ev0.elapsed_time(ev1)
    rt.set_active(None)
    rt.sync()
    active = float(sum(m.sum() for m in masks))
    return {"workload": f"voronoi {LATTICE}^3, 4-level time-step hierarchy (10/20/30/40 %, spatially correlated), "
                        f"{n_steps} steps of {N_SUB} subcycles, mixed",
            "active_fraction": active / (n_steps * C),
            "value": active * N_SUB / (ms_masked / 1e3), "unit": "active cell-updates/s",
            "ms_masked": ms_masked, "ms_all_active": ms_all, "time_ratio": ms_masked / ms_all}


def measure_config5(dev, fp64pk, n=256, n_sub=200, adj_sub=20, k=20, adjoint=True):
    """The large box: Voronoi mesh of a 256^3 jittered lattice (16.8M cells,
    7.16 Mpc, exp(GRF) density as the THESAN-like box, 32768 peak sources,
    c_red = 0.2 c).  Mixed forward of one step of n_sub subcycles (after one
    warm-up step); then the FP64 reverse mode over adj_sub subcycles with a
    checkpoint every k (over all 200 subcycles it takes ~4 minutes, so the
    default run takes 20).  Reports cell-updates/s and the device memory in
    use (cudaMemGetInfo) at the end of each part."""
    import torch
    import synth
    from paper_2404_17630_gb300 import RT, make_config
    from paper_2404_17630_gb300 import rt as rtb
    t0 = time.perf_counter()
    mesh, cfg, state = synth.thesan_like(n, 10, 32768, 7160.0, 256)
    build_s = time.perf_counter() - t0
    C = mesh.n_cells
    stream = torch.cuda.current_stream(dev)
    out = {"workload": f"voronoi {n}^3 ({C} cells, {mesh.n_faces} faces), GRF n_H, 32768 peak sources, c_red 0.2c",
           "mesh_build_s": round(build_s, 1)}
    free0, total = torch.cuda.mem_get_info(dev)
    rt = RT(make_config(precision="mixed", gather_sum=1, **cfg), mesh, stream=stream)
    rt.set_gas(state["nH"], state["x5"], state["T"])
    rt.set_radiation(state["N"], state["fr"] * cfg["c_red"])
    rt.set_sources(state["cells"], state["Q"])
    dt = rt.max_dt() * n_sub
    rt.step(dt, n_sub)
    rt.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rt.step(dt, n_sub)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    rt.sync()
    free1, _ = torch.cuda.mem_get_info(dev)
    rtb.rt_profile_read(rt.ctx, reset=True)
    rtb.rt_profile_enable(rt.ctx, True)
    rt.step(dt, n_sub)
    prof = rtb.rt_profile_read(rt.ctx, reset=True)
    rtb.rt_profile_enable(rt.ctx, False)
    rt.sync()
    Cm, Fm, _ = rt.mesh_info()
    peaks, kind = measured_peaks()
    rf, kern, rf_mem, rf_sub = roofline(dict(ms=ms, C=Cm, F=Fm, prof=prof), "mixed", peaks, kind, fp64pk,
                                        attempts=float(rt.fields()["nsub"].sum()), n_sub=n_sub, steps=1)
    out["forward_mixed"] = {"value": C * n_sub / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "n_sub": n_sub,
                            "device_GB_in_use": round((free0 - free1) / 1e9, 1), "roofline": rf,
                            "roofline_memory_kernel": rf_mem, "roofline_subcycle": rf_sub, "kernels": kern}
    del rt
    if not adjoint:
        return out
    torch.cuda.synchronize(dev)
    rt = RT(make_config(precision="fp64", **dict(cfg, chem_mode=2)), mesh, stream=stream)
    rt.set_gas(state["nH"], state["x5"], state["T"])
    rt.set_radiation(state["N"], state["fr"] * cfg["c_red"])
    rt.set_sources(state["cells"], state["Q"])
    dta = rt.max_dt() * adj_sub
    lx = np.zeros((5, C))
    lx[1] = state["nH"] * mesh.volume / (state["nH"] * mesh.volume).sum()
    t1 = time.perf_counter()
    try:
        res = rt.adjoint(dta, adj_sub, k, lam_x5=torch.as_tensor(lx, device=dev), n_src=len(state["cells"]))
    except rtb.RTError as e:   # e.g. device memory: report it, keep the rest of the line
        out["adjoint_fp64"] = {"error": str(e), "n_sub": adj_sub, "checkpoint_every": k,
                               "tape": rt.adjoint_tape_info()}
        del rt
        return out
    torch.cuda.synchronize(dev)
    adj_s = time.perf_counter() - t1
    free2, _ = torch.cuda.mem_get_info(dev)
    out["adjoint_fp64"] = {"value": C * adj_sub / adj_s, "unit": UNIT, "seconds": round(adj_s, 2),
                           "n_sub": adj_sub, "checkpoint_every": k,
                           "device_GB_in_use": round((free0 - free2) / 1e9, 1),
                           "tape": rt.adjoint_tape_info(),
                           "dL_dQ_finite": bool(np.isfinite(res["dQ"]).all())}
    del rt
    return out


def measure_adjoint(dev, n=64, n_sub=50, k=10):
    """FP64 forward and reverse mode on the 262k-cell differentiable workload."""
    import torch
    from paper_2404_17630_gb300 import RT, make_config
    mesh, cfg, state = differentiable(n)
    C = mesh.n_cells
    stream = torch.cuda.current_stream(dev)
    rt = RT(make_config(precision="fp64", **cfg), mesh, stream=stream)

    def reset():
        rt.set_gas(state["nH"], state["x5"], state["T"])
        rt.set_radiation(state["N"], state["fr"] * cfg["c_red"])
        rt.set_sources(state["cells"], state["Q"])

    reset()
    dt = rt.max_dt() * n_sub
    R = state["region"]
    m = state["nH"] * mesh.volume
    lx = np.zeros((5, C))
    lx[1][R] = m[R] / m[R].sum()
    lx_d = torch.as_tensor(lx, device=dev)
    # forward
    rt.step(dt, n_sub); rt.sync(); reset()
    t0 = time.perf_counter()
    rt.step(dt, n_sub)
    rt.sync()
    fwd = time.perf_counter() - t0
    reset()
    out = rt.adjoint(dt, n_sub, k, lam_x5=lx_d, n_src=len(state["cells"]))  # warm-up (allocations)
    reset()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    out = rt.adjoint(dt, n_sub, k, lam_x5=lx_d, n_src=len(state["cells"]))
    torch.cuda.synchronize(dev)
    adj = time.perf_counter() - t0
    free, total = torch.cuda.mem_get_info(dev)
    return {"workload": f"voronoi {n}^3 ({C} cells), {n_sub} FP64 subcycles, H+He with thermal energy, 8 sources, "
                        f"checkpoint every {k}", "forward_value": C * n_sub / fwd, "adjoint_value": C * n_sub / adj,
            "unit": UNIT, "forward_s": round(fwd, 4), "adjoint_s": round(adj, 4),
            "adjoint_over_forward": round(adj / fwd, 2), "dL_dQ": out["dQ"].sum(axis=1).tolist(),
            "tape": rt.adjoint_tape_info(),
            "device_mem_used_GB": round((total - free) / 1e9, 2)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 2.1M-cell THESAN-like run")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the reverse-mode run")
    ap.add_argument("--no-hii", action="store_true", help="skip the HII-region and time-step-hierarchy runs")
    ap.add_argument("--no-config5", action="store_true",
                    help="skip the 16.8M-cell box (mixed forward and a 20-subcycle FP64 reverse mode; ~190 GB of "
                         "device memory)")
    ap.add_argument("--config5-no-adjoint", action="store_true", help="the 16.8M-cell box without the reverse mode")
    ap.add_argument("--config5-adjoint-sub", type=int, default=20,
                    help="subcycles of the 16.8M-cell box's reverse mode (checkpoint every 20); 200 is the "
                         "full step (~4 minutes, ~211 GB of device memory)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus))
    local = int(os.environ.get("LOCAL_RANK", 0))

    if args.impl == "reference":
        return reference_arm(args, rank)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist_.init_process_group("nccl")
        dist = dist_
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    mesh, cfg, state = workload()
    peaks, peak_kind = measured_peaks()
    fp64pk = fp64_peak(torch.cuda.current_stream(dev))
    clocks = ClockSampler(local)
    res = run_gpu("mixed", mesh, cfg, state, args.steps, args.warmup, rank, world, dev, dist, clocks)
    cl = clocks.summary()
    fp64 = None
    if not args.no_fp64:
        r64 = run_gpu("fp64", mesh, cfg, state, max(2, args.steps // 5), 1, rank, world, dev, dist)
        fp64 = {"value": replica_value(world, r64["C"], N_SUB, max(2, args.steps // 5), r64["ms"]),
                "ms_per_step": r64["ms"] / max(2, args.steps // 5), "dtype": "f64"}
        rf64, k64, rf64m, rf64s = roofline(r64, "fp64", peaks, peak_kind, fp64pk, attempts=r64.get("attempts"),
                                           n_sub=N_SUB, steps=max(2, args.steps // 5))
        fp64["roofline"] = rf64
        fp64["roofline_memory_kernel"] = rf64m
        fp64["roofline_subcycle"] = rf64s
        fp64["kernels"] = k64
    fp64sum = None
    if not args.no_fp64:
        n64s = max(2, args.steps // 2)
        r = run_gpu("mixed", mesh, cfg, state, n64s, 1, rank, world, dev, dist, gather_sum=0)
        fp64sum = {"value": replica_value(world, r["C"], N_SUB, n64s, r["ms"]), "ms_per_step": r["ms"] / n64s,
                   "note": "mixed precision with each FP32 face flux widened and summed in FP64 (gather_sum=0)"}
    e2e = None if args.no_e2e else e2e_measure("mixed", mesh, cfg, state, max(2, args.steps // 2), args.warmup, dev)
    large = None if args.no_large else measure_large(3, 1, dev, fp64pk)
    adjoint = None if args.no_adjoint else measure_adjoint(dev)
    hii = None if args.no_hii else measure_hii(3, 1, dev)
    timebins = None if args.no_hii else measure_timebins(dev)
    config5 = None if args.no_config5 else measure_config5(dev, fp64pk, adj_sub=args.config5_adjoint_sub,
                                                           adjoint=not args.config5_no_adjoint)
    if rank != 0:
        return
    C, F = res["C"], res["F"]
    value = replica_value(world, C, N_SUB, args.steps, res["ms"])
    rf, kern, rf_mem, rf_sub = roofline(res, "mixed", peaks, peak_kind, fp64pk, attempts=res.get("attempts"),
                                        n_sub=N_SUB, steps=args.steps)
    cpu = None if args.no_cpu else cpu_baseline(mesh, cfg, state)
    ws = (C * 3 * (32 + 16 + 48) + F * (64 + 48) + C * 200)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"voronoi {LATTICE}^3 jittered lattice ({C} cells, {F} faces, "
                               f"{F / C:.3f} faces/cell), lognormal n_H, 16 sources, 3 bins, {N_SUB} subcycles/step",
                   "cells": C, "faces": F, "n_sub": N_SUB,
                   "precision": "mixed (FP32 sweep; FP64 state, update and chemistry; face-flux sums as compensated FP32 pairs)",
                   "l2": f"working set ~{ws / 1e6:.0f} MB > L2 129 MB; L2 also flushed once before the timed region",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": rf, "roofline_memory_kernel": rf_mem, "roofline_subcycle": rf_sub, "kernels": kern,
        "fp64_peak": {"tflops": round(fp64pk[0], 4), "source": fp64pk[1]},
        "fp64": fp64,
        "speedup_mixed_over_fp64": (value / fp64["value"]) if fp64 else None,
        "mixed_fp64_sums": fp64sum,
        "e2e": e2e, "cpu_baseline": cpu,
        "thesan_like_2M": large, "adjoint": adjoint, "hii_region": hii, "individual_timesteps": timebins,
        "box_16M": config5,
        "gpu_launches": res["launches"], "clocks": cl,
    }
    print(json.dumps(out))


def reference_arm(args, rank):
    """The FP64 oracle as it stands, timed on the host cores (the OpenMP
    build of its source on all of them, bitwise the single-threaded results),
    on the same workload: each step is a bounded sample (one subcycle of the
    full mesh)."""
    if rank != 0:
        return
    mesh, cfg, state = workload()
    from oracle import Oracle, default_config, oracle_threads_available
    threads = 0 if oracle_threads_available() else 1
    o = Oracle(default_config(**cfg), mesh, threads=threads)
    o.set_radiation(state["N"], state["fr"])
    o.set_gas(state["nH"], state["x5"], state["T"])
    o.set_sources(state["cells"], state["Q"])
    dt = o.max_dt()
    for _ in range(args.warmup):
        o.step(dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(dt, 1)
    sec = time.perf_counter() - t0
    v = mesh.n_cells * args.steps / sec
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"voronoi {LATTICE}^3 jittered lattice ({mesh.n_cells} cells), one subcycle per step",
                      "cells": mesh.n_cells, "n_sub": 1},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": o.threads, "host_cores": os.cpu_count(),
                            "kind": "oracle",
                            "sample": f"{args.steps} timed subcycles of the full mesh after {args.warmup} warm-up "
                                      f"subcycles, {o.threads} threads"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
