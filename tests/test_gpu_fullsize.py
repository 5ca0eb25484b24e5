"""Parity at the full sizes of the THESAN-like boxes (128^3 and 256^3
jittered-lattice Voronoi meshes, 2.1M and 16.8M cells), in the launch
configuration the bench times, where the oracle cannot run the whole mesh:

* sampled outputs the oracle computes one by one: the chemistry of a cell
  depends on that cell alone, so for 256 seeded cells the oracle runs the
  same inputs on a periodic 2^3 box of copies of the cell (a uniform field,
  so only the thermochemistry acts) and the cell's result is compared;
* properties that hold at any size: with recombination and collisional
  ionisation off, sum_i V_i (sum_b N_b + n_e) grows by exactly sum_k Q_k t
  (every photon is in flight or made one electron; the face fluxes enter
  their two cells with opposite signs), and a uniform radiation field stays
  uniform.

Every input is seeded and synthetic; nothing the oracle sees comes from the
CUDA path.
"""
import numpy as np
import pytest

import synth
from tests._cases import make_oracle

pytestmark = pytest.mark.gpu


def _rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def _state(mesh, cfg, seed):
    """Random radiation with |F| <= c N, partly ionised gas, T in [5e3, 3e4]."""
    C, B = mesh.n_cells, cfg["n_bins"]
    rng = np.random.default_rng(seed)
    N = rng.uniform(0.0, 1e-6, size=(B, C))
    d = rng.standard_normal((B, 3, C))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    fr = d * (N * rng.uniform(0, 1, size=(B, C)))[:, None, :]
    xHII = rng.uniform(0, 1, C)
    yII, yIII = rng.uniform(0, 0.5, C), rng.uniform(0, 0.5, C)
    x5 = np.stack([1 - xHII, xHII, 1 - yII - yIII, yII, yIII])
    T = rng.uniform(5e3, 3e4, C)
    return N, fr, x5, T


def _gpu(mesh, cfg, precision, nH, N, fr, x5, T, cells, Q):
    from paper_2404_17630_gb300 import RT, make_config
    rt = RT(make_config(precision=precision, gather_sum=1, **cfg), mesh)
    rt.set_gas(nH, x5, T)
    rt.set_radiation(N, fr * cfg["c_red"])
    rt.set_sources(cells, Q)
    return rt


def _sampled_chemistry(mesh, cfg, precision, seed):
    import torch
    C = mesh.n_cells
    N, fr, x5, T = _state(mesh, cfg, seed)
    nH = synth.lognormal_density(C, 2e-4, 1.5, seed + 1)
    rt = _gpu(mesh, cfg, precision, nH, N, fr, x5, T, np.zeros(0, np.int64), np.zeros((0, 3)))
    dt = rt.max_dt()
    rt.thermochemistry(dt)
    assert rt.sync() == 0
    got = rt.fields()
    del rt
    torch.cuda.empty_cache()
    sample = np.random.default_rng(seed + 2).choice(C, 256, replace=False)
    errs = {"N": 0.0, "F": 0.0, "x5": 0.0, "T": 0.0}
    for i in sample:
        h = 2.0 * np.cbrt(mesh.volume[i])
        box = synth.cartesian_mesh(2, h)
        rep = lambda a: np.repeat(a[..., i:i + 1], 8, axis=-1)
        c = dict(cfg, box=h)
        o = make_oracle(box, c, dict(nH=np.full(8, nH[i]), x5=rep(x5), T=np.full(8, T[i]), N=rep(N), fr=rep(fr),
                                     cells=np.zeros(0, np.int64), Q=np.zeros((0, 3))))
        assert o.thermochemistry(dt) == 0
        oN, ofr = o.radiation()
        ox5, oT = o.gas()
        for k, a, b in (("N", got["N"][:, i], oN[:, 0]), ("F", got["F"][:, :, i] / cfg["c_red"], ofr[:, :, 0]),
                        ("x5", got["x5"][:, i], ox5[:, 0]), ("T", got["T"][i], oT[0])):
            errs[k] = max(errs[k], _rel(np.atleast_1d(a), np.atleast_1d(b)))
    return errs


def _budget(mesh, cfg, precision, seed, n_sub=2):
    """sum V (sum N + n_e) before and after n_sub subcycles, and sum Q t
    (recombination and collisional ionisation off)."""
    C = mesh.n_cells
    c = dict(cfg, chem_mode=1, chem_flags=0)
    # neutral gas and a faint field, so that the injected photons are a
    # large part of the budget
    N, fr, _, T = _state(mesh, c, seed)
    N, fr = N * 1e-6, fr * 1e-6
    x5 = np.zeros((5, C)); x5[0] = 1.0; x5[2] = 1.0
    nH = synth.lognormal_density(C, 2e-4, 1.5, seed + 1)
    srng = np.random.default_rng(seed + 3)
    cells = srng.choice(C, 64, replace=False).astype(np.int64)
    Q = np.outer(10 ** srng.uniform(49, 51, 64), synth.SPECTRAL_SPLIT_E4)
    rt = _gpu(mesh, c, precision, nH, N, fr, x5, T, cells, Q)
    V = mesh.volume * c["unit_length_cm"] ** 3
    yhe = c["y_he"]

    def total(Nb, x):
        return ((Nb.sum(0) + nH * (x[1] + yhe * (x[3] + 2 * x[4]))) * V).sum()

    t0 = total(N, x5)
    dt = rt.max_dt() * n_sub
    rt.step(dt, n_sub)
    assert rt.sync() == 0
    f = rt.fields()
    t1 = total(f["N"], f["x5"])
    return t0, t1, Q.sum() * dt


def _uniform(mesh, cfg, precision):
    C, B = mesh.n_cells, cfg["n_bins"]
    c = dict(cfg, chem_mode=0)
    N = np.full((B, C), 2.5e-6)
    fr = np.zeros((B, 3, C))
    fr[:, 0], fr[:, 1], fr[:, 2] = 1e-6, -0.5e-6, 0.7e-6
    x5 = np.zeros((5, C)); x5[0] = 1.0; x5[2] = 1.0
    rt = _gpu(mesh, c, precision, np.full(C, 2e-4), N, fr, x5, np.full(C, 1e4), np.zeros(0, np.int64),
              np.zeros((0, 3)))
    rt.step(rt.max_dt(), 1)
    assert rt.sync() == 0
    f = rt.fields()
    return _rel(f["N"], N), _rel(f["F"] / c["c_red"], fr)


def _check(mesh, cfg, precisions, seed):
    out = {}
    for p in precisions:
        chem = _sampled_chemistry(mesh, cfg, p, seed)
        t0, t1, inj = _budget(mesh, cfg, p, seed)
        uN, uF = _uniform(mesh, cfg, p)
        out[p] = dict(chem=chem, budget=abs((t1 - t0) / inj - 1), uniform=(uN, uF))
        tol_chem = 1e-12 if p == "fp64" else 1e-5
        assert max(chem.values()) < tol_chem, (p, chem)
        assert inj > 1e-3 * t0
        assert abs((t1 - t0) / inj - 1) < 1e-8, (p, t0, t1, inj)
        tol_u = 1e-12 if p == "fp64" else 1e-6
        assert uN < tol_u and uF < tol_u, (p, uN, uF)
    print("full-size checks", out)


def test_fullsize_thesan_2M():
    """128^3 = 2,097,152 cells: FP64 and mixed."""
    mesh, cfg, _ = synth.thesan_like(128, 4, 4096)
    _check(mesh, cfg, ("fp64", "mixed"), 31)


@pytest.mark.slow
def test_fullsize_thesan_16M():
    """256^3 = 16,777,216 cells (the large-throughput box): mixed."""
    mesh = synth.voronoi_mesh(256, 7160.0, 0.3, seed=10)
    _, cfg, _ = synth.thesan_like(8, 4, 1)
    cfg["box"] = 7160.0
    _check(mesh, cfg, ("mixed",), 41)
