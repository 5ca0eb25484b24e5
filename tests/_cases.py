"""Seeded test cases shared by the oracle pins and the GPU parity tests.

Builds meshes, configurations and initial states from ``synth`` (which holds
no RT arithmetic).  Configurations are plain dicts, turned into the oracle's
struct or the library's struct by the caller.
"""
from __future__ import annotations

import numpy as np

import synth

SIGMA3 = synth.GREY_SIGMA
EPS3 = synth.GREY_EPS


def base_config(**kw) -> dict:
    cfg = dict(n_bins=3, c_red=0.01 * synth.C_LIGHT, unit_length_cm=synth.KPC_CM, box=10.0, cfl=0.3,
               chem_mode=2, chem_flags=15, limiter=1, lim_eps=1e-5, order=2, f_s=0.05, f_max=0.1, x_floor=1e-4,
               max_substeps=10000, y_he=synth.helium_ratio(0.24), sigma=SIGMA3, eps=EPS3)
    cfg.update(kw)
    return cfg


def neutral_gas(C, nH, T=1e4):
    x5 = np.zeros((5, C))
    x5[0] = 1.0
    x5[2] = 1.0
    return np.broadcast_to(np.asarray(nH, dtype=np.float64), (C,)).copy(), x5, np.full(C, float(T))


def corner_cells(n, i0):
    """The 8 cells of an n^3 grid around the lattice corner at index i0."""
    return np.array([(i % n) + n * ((j % n) + n * (k % n))
                     for k in (i0 - 1, i0) for j in (i0 - 1, i0) for i in (i0 - 1, i0)], dtype=np.int64)


def config1(n=32):
    """Periodic 32^3 Cartesian grid, box 10 kpc, n_H = 1e-3, Y = 0.24,
    T = 1e4 K, neutral; one central source of 5e48 photons/s split equally
    over the 8 cells sharing the central corner; c_red = 0.01 c, CFL 0.3."""
    mesh = synth.cartesian_mesh(n, 10.0)
    cfg = base_config()
    C = mesh.n_cells
    nH, x5, T = neutral_gas(C, 1e-3)
    cells = corner_cells(n, n // 2)
    Q = np.outer(np.full(8, 5e48 / 8), synth.SPECTRAL_SPLIT_E4)
    return mesh, cfg, dict(nH=nH, x5=x5, T=T, N=np.zeros((3, C)), fr=np.zeros((3, 3, C)), cells=cells, Q=Q)


def voronoi_case(n=16, seed=1, n_src=4, L=10.0, n_bins=3, radiation_seed=11, **kw):
    """Jittered-lattice Voronoi mesh (jitter 0.3 h), lognormal density
    (median 1e-3, sigma_ln 1), a random radiation field with |F| <= c N,
    partly ionised gas and ``n_src`` sources with log10 Q ~ U(48, 51)."""
    mesh = synth.voronoi_mesh(n, L, 0.3, seed=seed)
    C = mesh.n_cells
    rng = np.random.default_rng(radiation_seed)
    cfg = base_config(box=L, n_bins=n_bins, **kw)
    nH = synth.lognormal_density(C, 1e-3, 1.0, seed + 1)
    N = rng.uniform(0.0, 1e-3, size=(n_bins, C)) * rng.uniform(0, 1, size=(n_bins, 1))
    direc = rng.standard_normal((n_bins, 3, C))
    direc /= np.linalg.norm(direc, axis=1, keepdims=True)
    fr = direc * (N * rng.uniform(0, 1, size=(n_bins, C)))[:, None, :]
    xHII = rng.uniform(0, 1, C)
    yII = rng.uniform(0, 0.5, C)
    yIII = rng.uniform(0, 0.5, C)
    x5 = np.stack([1 - xHII, xHII, 1 - yII - yIII, yII, yIII])
    T = rng.uniform(5e3, 3e4, C)
    srng = np.random.default_rng(seed + 2)
    cells = srng.choice(C, size=n_src, replace=False).astype(np.int64)
    Qtot = 10 ** srng.uniform(48, 51, n_src)
    Q = np.outer(Qtot, synth.SPECTRAL_SPLIT_E4[:n_bins] / synth.SPECTRAL_SPLIT_E4[:n_bins].sum())
    return mesh, cfg, dict(nH=nH, x5=x5, T=T, N=N, fr=fr, cells=cells, Q=Q)


def make_oracle(mesh, cfg, state):
    from oracle import Oracle, default_config
    o = Oracle(default_config(**cfg), mesh)
    o.set_radiation(state["N"], state["fr"])
    o.set_gas(state["nH"], state["x5"], state["T"])
    if len(state.get("cells", [])):
        o.set_sources(state["cells"], state["Q"])
    return o
