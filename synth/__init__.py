"""Seeded synthetic inputs for the RT subcycle: meshes, gas, radiation, sources.

This module holds no arithmetic of the RT method itself.  It produces the
static mesh (cells and faces) and the initial state that the oracle and the
CUDA path both consume:

* periodic Cartesian grids (one face per cell pair, exact geometry);
* periodic Voronoi meshes of jittered cubic lattices (``voronoi.cpp``, built
  on first use with g++), standing in for AREPO's moving-mesh tessellation
  (Sec. 2.1) held static over the RT subcycles (Sec. 2.3);
* lognormal and exp(Gaussian random field) density fields, density peaks;
* point sources binned onto cells, and the travelling-wave initial condition
  of the photon-transport test (Sec. 4.2.1).

Units: geometry in a length unit of the caller's choice (``unit_length_cm``
converts it), number densities in cm^-3, photon rates in photons/s.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "Mesh", "cartesian_mesh", "voronoi_mesh", "jittered_lattice",
    "lognormal_density", "grf_density", "density_peaks", "locate_cells",
    "KPC_CM", "MPC_CM", "C_LIGHT", "helium_ratio", "SPECTRAL_SPLIT_E4", "GREY_SIGMA", "GREY_EPS",
]

KPC_CM = 3.0856775814913673e21
MPC_CM = 1e3 * KPC_CM
C_LIGHT = 2.99792458e10          # cm/s
MYR_S = 3.15576e13               # s
# Photon-rate split over the HI / HeI / HeII bins used by the coupled HII-region
# test of Sec. 4.2.2 (1e50, 5e48, 3e48 photons/s), applied to every source.
SPECTRAL_SPLIT_E4 = np.array([1e50, 5e48, 3e48]) / (1e50 + 5e48 + 3e48)


EV = 1.602176634e-12             # erg
# Grey cross-sections [bin][HI, HeI, HeII] (cm^2) and heat per photoionisation
# (erg) of the HI-, HeI- and HeII-ionising bins.  The paper averages them over
# a blackbody spectrum (Sec. 4.2.2) without printing values; these are
# proposed constants of the right magnitude (thresholds 13.6 / 24.6 / 54.4 eV).
GREY_SIGMA = [[3.0e-18, 0.0, 0.0], [5.7e-19, 4.5e-18, 0.0], [7.9e-20, 1.1e-18, 1.1e-18]]
GREY_EPS = [[5.3 * EV, 0.0, 0.0], [21.5 * EV, 10.5 * EV, 0.0], [52.1 * EV, 41.1 * EV, 11.3 * EV]]


def helium_ratio(Y: float) -> float:
    """n_He / n_H for helium mass fraction Y (He nucleus mass = 4 m_H)."""
    return Y / (4.0 * (1.0 - Y))


@dataclasses.dataclass
class Mesh:
    """Static mesh in structure-of-arrays form.

    Cells: ``volume``, centroid ``cx, cy, cz``.  Faces: ``left, right`` (int32
    cell ids), ``area``, unit normal ``nx, ny, nz`` pointing from left to
    right, centroid ``fx, fy, fz``.  ``box`` is the periodic box length
    (0 = not periodic).  ``gen`` holds the generating points where there are any.
    """
    volume: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    cz: np.ndarray
    left: np.ndarray
    right: np.ndarray
    area: np.ndarray
    nx: np.ndarray
    ny: np.ndarray
    nz: np.ndarray
    fx: np.ndarray
    fy: np.ndarray
    fz: np.ndarray
    box: float
    gen: np.ndarray | None = None
    lattice_n: int = 0

    @property
    def n_cells(self) -> int:
        return int(self.volume.shape[0])

    @property
    def n_faces(self) -> int:
        return int(self.left.shape[0])

    @property
    def faces_per_cell(self) -> float:
        return self.n_faces / max(self.n_cells, 1)

    def centroids(self) -> np.ndarray:
        return np.stack([self.cx, self.cy, self.cz], axis=1)


# ----------------------------------------------------------------------------
# Cartesian grid
# ----------------------------------------------------------------------------

def cartesian_mesh(n: int, L: float) -> Mesh:
    """Periodic n^3 grid of side L.  Cell (i,j,k) has id i + n(j + n k); its
    faces towards +x, +y, +z come in that order, so face 3c+a joins cell c
    (left) to its +a neighbour (right)."""
    h = L / n
    idx = np.arange(n ** 3, dtype=np.int64)
    i, j, k = idx % n, (idx // n) % n, idx // (n * n)
    cx, cy, cz = (i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h
    nbr = [((i + 1) % n) + n * (j + n * k), i + n * (((j + 1) % n) + n * k), i + n * (j + n * ((k + 1) % n))]
    left = np.repeat(idx, 3).astype(np.int32)
    right = np.stack(nbr, axis=1).reshape(-1).astype(np.int32)
    F = 3 * n ** 3
    nx = np.tile(np.array([1.0, 0.0, 0.0]), n ** 3)
    ny = np.tile(np.array([0.0, 1.0, 0.0]), n ** 3)
    nz = np.tile(np.array([0.0, 0.0, 1.0]), n ** 3)
    fx = np.repeat(cx, 3) + 0.5 * h * nx
    fy = np.repeat(cy, 3) + 0.5 * h * ny
    fz = np.repeat(cz, 3) + 0.5 * h * nz
    fx, fy, fz = np.mod(fx, L), np.mod(fy, L), np.mod(fz, L)
    return Mesh(volume=np.full(n ** 3, h ** 3), cx=cx, cy=cy, cz=cz, left=left, right=right,
                area=np.full(F, h * h), nx=nx, ny=ny, nz=nz, fx=fx, fy=fy, fz=fz, box=float(L),
                gen=np.stack([cx, cy, cz], axis=1), lattice_n=n)


# ----------------------------------------------------------------------------
# Staggered (body-centred cubic) grid
# ----------------------------------------------------------------------------

def bcc_mesh(n: int, L: float) -> Mesh:
    """Voronoi mesh of the staggered 2 x n^3 grid in a periodic box of side L:
    generators on the corners (i, j, k) h and the body centres (i+1/2, j+1/2,
    k+1/2) h of an n^3 lattice, h = L / n.  Every cell is the same truncated
    octahedron of volume h^3 / 2: eight hexagonal faces (area 3 sqrt(3) h^2 / 16)
    towards the nearest generators of the other sublattice at (+-1, +-1, +-1)
    h / 2, and six square faces (area h^2 / 8) towards the next generators of
    its own sublattice at h along each axis; each face lies on the bisector
    plane, centred on the midpoint.  Corner cell (i, j, k) has id i + n(j + nk),
    body-centre cell n^3 + i + n(j + nk).  Faces: the 8 n^3 hexagons listed
    from the corner cells (left), then the 6 n^3 squares towards +x, +y, +z
    from every cell (left)."""
    h = L / n
    n3 = n ** 3
    idx = np.arange(n3, dtype=np.int64)
    i, j, k = idx % n, (idx // n) % n, idx // (n * n)

    def cid(a, b, c):
        return (a % n) + n * ((b % n) + n * (c % n))

    pos_a = np.stack([i * h, j * h, k * h], axis=1).astype(np.float64)
    pos_b = pos_a + 0.5 * h
    pos = np.concatenate([pos_a, pos_b])
    left, right, nrm, area = [], [], [], []
    hexa = 3.0 * np.sqrt(3.0) / 16.0 * h * h
    for sx in (-1, 1):
        for sy in (-1, 1):
            for sz in (-1, 1):
                # body-centre neighbour at (i, j, k) h + (sx, sy, sz) h / 2
                nb = n3 + cid(i + (sx - 1) // 2, j + (sy - 1) // 2, k + (sz - 1) // 2)
                left.append(idx)
                right.append(nb)
                d = np.array([sx, sy, sz], dtype=np.float64) / np.sqrt(3.0)
                nrm.append(np.broadcast_to(d, (n3, 3)))
                area.append(np.full(n3, hexa))
    sq = h * h / 8.0
    for base in (0, n3):
        for ax in range(3):
            step = [0, 0, 0]
            step[ax] = 1
            left.append(base + idx)
            right.append(base + cid(i + step[0], j + step[1], k + step[2]))
            d = np.zeros(3)
            d[ax] = 1.0
            nrm.append(np.broadcast_to(d, (n3, 3)))
            area.append(np.full(n3, sq))
    left = np.concatenate(left)
    right = np.concatenate(right)
    nrm = np.concatenate(nrm)
    area = np.concatenate(area)
    # face centre: midpoint of the two generators along the minimum image
    dvec = pos[right] - pos[left]
    dvec -= L * np.round(dvec / L)
    fc = np.mod(pos[left] + 0.5 * dvec, L)
    C = 2 * n3
    return Mesh(volume=np.full(C, 0.5 * h ** 3), cx=pos[:, 0].copy(), cy=pos[:, 1].copy(), cz=pos[:, 2].copy(),
                left=left.astype(np.int32), right=right.astype(np.int32), area=area, nx=nrm[:, 0].copy(),
                ny=nrm[:, 1].copy(), nz=nrm[:, 2].copy(), fx=fc[:, 0].copy(), fy=fc[:, 1].copy(),
                fz=fc[:, 2].copy(), box=float(L), gen=pos, lattice_n=0)


# ----------------------------------------------------------------------------
# Voronoi mesh of a jittered lattice
# ----------------------------------------------------------------------------

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LIB_LOCK = threading.Lock()


def _lib_path() -> str:
    return os.path.join(_HERE, "_voronoi.so")


def build_voronoi_lib(force: bool = False) -> str:
    """Compile voronoi.cpp into _voronoi.so (g++, OpenMP).  Returns the path."""
    src = os.path.join(_HERE, "voronoi.cpp")
    out = _lib_path()
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp])
        os.replace(tmp, out)
    return out


def _load():
    global _LIB
    with _LIB_LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build_voronoi_lib())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            lib.vor_build.restype = ctypes.c_void_p
            lib.vor_build.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp, ctypes.c_int,
                                      ctypes.c_char_p, ctypes.c_int]
            lib.vor_num_faces.restype = ctypes.c_int64
            lib.vor_num_faces.argtypes = [ctypes.c_void_p]
            lib.vor_num_asym.restype = ctypes.c_int64
            lib.vor_num_asym.argtypes = [ctypes.c_void_p]
            lib.vor_fetch.restype = None
            lib.vor_fetch.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, ip, ip, dp, dp, dp, dp, dp, dp, dp]
            lib.vor_free.restype = None
            lib.vor_free.argtypes = [ctypes.c_void_p]
            _LIB = lib
    return _LIB


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def jittered_lattice(n: int, L: float, jitter: float, seed: int) -> np.ndarray:
    """n^3 generators: lattice-cell centres (i+1/2)h plus an offset drawn
    uniformly from [-jitter*h, +jitter*h] per axis (numpy PCG64, ``seed``).
    Point p = i + n(j + n k) stays inside lattice cell (i,j,k) for jitter < 1/2."""
    if not 0 <= jitter < 0.5:
        raise ValueError("jitter must lie in [0, 0.5)")
    h = L / n
    rng = np.random.default_rng(seed)
    idx = np.arange(n ** 3, dtype=np.int64)
    base = np.stack([idx % n, (idx // n) % n, idx // (n * n)], axis=1).astype(np.float64) + 0.5
    off = rng.uniform(-jitter, jitter, size=(n ** 3, 3))
    return (base + off) * h


def voronoi_mesh(n: int, L: float, jitter: float = 0.3, seed: int = 1, nthreads: int = 0) -> Mesh:
    """Periodic Voronoi mesh of an n^3 jittered lattice in a box of side L."""
    if jitter <= 0:
        raise ValueError("use cartesian_mesh for an unjittered lattice (degenerate Voronoi vertices)")
    pts = np.ascontiguousarray(jittered_lattice(n, L, jitter, seed))
    px, py, pz = (np.ascontiguousarray(pts[:, a]) for a in range(3))
    lib = _load()
    err = ctypes.create_string_buffer(256)
    h = lib.vor_build(n, L, _dptr(px), _dptr(py), _dptr(pz), int(nthreads), err, 256)
    if not h:
        raise RuntimeError(err.value.decode())
    try:
        C, F = n ** 3, lib.vor_num_faces(h)
        arr = {k: np.empty(C) for k in ("volume", "cx", "cy", "cz")}
        left, right = np.empty(F, np.int32), np.empty(F, np.int32)
        farr = {k: np.empty(F) for k in ("area", "nx", "ny", "nz", "fx", "fy", "fz")}
        lib.vor_fetch(h, _dptr(arr["volume"]), _dptr(arr["cx"]), _dptr(arr["cy"]), _dptr(arr["cz"]),
                      _iptr(left), _iptr(right), _dptr(farr["area"]), _dptr(farr["nx"]), _dptr(farr["ny"]),
                      _dptr(farr["nz"]), _dptr(farr["fx"]), _dptr(farr["fy"]), _dptr(farr["fz"]))
    finally:
        lib.vor_free(h)
    return Mesh(left=left, right=right, box=float(L), gen=pts, lattice_n=n, **arr, **farr)


# ----------------------------------------------------------------------------
# Density fields and sources
# ----------------------------------------------------------------------------

def lognormal_density(n_cells: int, median: float, sigma_ln: float, seed: int) -> np.ndarray:
    """i.i.d. lognormal n_H per cell: median * exp(sigma_ln * z), z ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    return median * np.exp(sigma_ln * rng.standard_normal(n_cells))


def grf_field(ng: int, slope: float, seed: int) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian random field on a periodic ng^3 grid
    with power spectrum P(k) ~ k^slope (k=0 mode removed)."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((ng, ng, ng))
    wk = np.fft.rfftn(white)
    kx = np.fft.fftfreq(ng)[:, None, None]
    ky = np.fft.fftfreq(ng)[None, :, None]
    kz = np.fft.rfftfreq(ng)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)   # sqrt(P) = k^(slope/2)
    g = np.fft.irfftn(wk * amp, s=(ng, ng, ng), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def grf_density(points: np.ndarray, L: float, ng: int, sigma: float, mean: float, seed: int,
                slope: float = -2.0):
    """exp(sigma * g) of a unit-variance GRF g (P(k) ~ k^slope) on an ng^3 grid,
    sampled at ``points`` by nearest grid node and scaled so that the mean over
    the grid is ``mean``.  Returns (n_H at points, grid field)."""
    g = grf_field(ng, slope, seed)
    rho = np.exp(sigma * g)
    rho *= mean / rho.mean()
    ijk = np.floor(points / L * ng).astype(np.int64) % ng
    # grid axis order (x, y, z)
    return rho[ijk[:, 0], ijk[:, 1], ijk[:, 2]], rho


def density_peaks(rho: np.ndarray, count: int) -> np.ndarray:
    """Grid indices (m, 3) of the ``count`` highest strict local maxima over the
    26 periodic neighbours, in decreasing order of density."""
    is_max = np.ones(rho.shape, dtype=bool)
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                if dx == dy == dz == 0:
                    continue
                is_max &= rho > np.roll(rho, (dx, dy, dz), axis=(0, 1, 2))
    cand = np.argwhere(is_max)
    vals = rho[is_max]
    order = np.argsort(-vals, kind="stable")[:count]
    return cand[order]


def locate_cells(mesh: Mesh, pos: np.ndarray) -> np.ndarray:
    """Cell whose generator is nearest (periodic) to each position; for a
    Voronoi mesh that is the cell containing it.  Uses the lattice: a point
    in lattice cell c is nearest to a generator within +-2 lattice cells."""
    n, L = mesh.lattice_n, mesh.box
    if mesh.gen is None or n == 0:
        raise ValueError("mesh has no lattice generators")
    h = L / n
    base = np.floor(pos / h).astype(np.int64)
    best = np.full(len(pos), -1, dtype=np.int64)
    bestd = np.full(len(pos), np.inf)
    for dk in range(-2, 3):
        for dj in range(-2, 3):
            for di in range(-2, 3):
                c = (base + np.array([di, dj, dk])) % n
                q = c[:, 0] + n * (c[:, 1] + n * c[:, 2])
                d = mesh.gen[q] - pos
                d -= L * np.round(d / L)
                d2 = (d * d).sum(axis=1)
                better = d2 < bestd
                best[better], bestd[better] = q[better], d2[better]
    return best


def thesan_like(n: int = 128, seed: int = 4, n_peaks: int = 4096, L: float = 3580.0, ng: int = 128):
    """THESAN-like reionisation box: Voronoi mesh of an n^3 jittered lattice in a
    periodic box of L kpc (3.58 Mpc physical = 23.3 cMpc at z = 5.5 for the
    full box), n_H = exp(GRF) with P(k) ~ k^-2, sigma 1.5, mean 2e-4 cm^-3 (ng^3
    FFT grid, nearest node), sources at the n_peaks highest density maxima with
    Q = 1e49 rho / rho_min clipped to 1e52 photons/s split over 3 bins, c_red =
    0.2 c, neutral gas at 1e4 K, no radiation.  The 1/8 sub-box instance is
    n = 64, L = 1790, ng = 64, n_peaks = 512.  Returns (mesh, cfg, state)."""
    mesh = voronoi_mesh(n, L, 0.3, seed=seed)
    C = mesh.n_cells
    nH, rho = grf_density(mesh.gen, L, ng, 1.5, 2e-4, seed + 1)
    peaks = density_peaks(rho, n_peaks)
    pos = (peaks + 0.5) * (L / ng)
    cells = locate_cells(mesh, pos).astype(np.int64)
    rp = rho[tuple(peaks.T)]
    Qtot = np.minimum(1e49 * rp / rp.min(), 1e52)
    Q = np.outer(Qtot, SPECTRAL_SPLIT_E4)
    x5 = np.zeros((5, C))
    x5[0] = 1.0
    x5[2] = 1.0
    cfg = dict(n_bins=3, c_red=0.2 * C_LIGHT, unit_length_cm=KPC_CM, box=L, cfl=0.3, chem_mode=2,
               chem_flags=15, limiter=1, lim_eps=1e-5, order=2, f_s=0.05, f_max=0.1, x_floor=1e-4,
               max_substeps=10000, y_he=helium_ratio(0.24), sigma=GREY_SIGMA, eps=GREY_EPS)
    state = dict(nH=nH, x5=x5, T=np.full(C, 1e4), N=np.zeros((3, C)), fr=np.zeros((3, 3, C)), cells=cells, Q=Q)
    return mesh, cfg, state


def hii_region(n: int = 44, n_bins: int = 3, L: float = 1.6, c_frac: float = 1e-3):
    """Expanding HII region on the staggered 2 x n^3 grid: periodic box of
    L kpc, neutral gas at 100 K with n_H = n0 inside r0 and n0 (r0 / r)^2
    outside (n0 = 3.2 cm^-3, r0 = 91.5 pc, r from the box centre), photons
    injected uniformly by volume into the cells within 0.05 kpc of the centre
    at 1e50, 5e48, 3e48 photons/s per bin (the first n_bins), c_red = c_frac c,
    Y = 0.24, full thermal network.  The box centre is a generator, so the
    setup is mirror-symmetric about it.  Returns (mesh, cfg, state)."""
    mesh = bcc_mesh(n, L)
    C = mesh.n_cells
    c = mesh.centroids() - 0.5 * L
    c -= L * np.round(c / L)
    r = np.sqrt((c * c).sum(1))
    n0, r0 = 3.2, 0.0915
    nH = n0 * (r0 / np.maximum(r, r0)) ** 2
    cells = np.nonzero(r < 0.05)[0].astype(np.int64)
    w = mesh.volume[cells] / mesh.volume[cells].sum()
    Qb = np.array([1e50, 5e48, 3e48])[:n_bins]
    Q = np.outer(w, Qb)
    x5 = np.zeros((5, C))
    x5[0] = 1.0
    x5[2] = 1.0
    cfg = dict(n_bins=n_bins, c_red=c_frac * C_LIGHT, unit_length_cm=KPC_CM, box=L, cfl=0.3, chem_mode=2,
               chem_flags=15, limiter=1, lim_eps=1e-5, order=2, f_s=0.05, f_max=0.1, x_floor=1e-4,
               max_substeps=10000, y_he=helium_ratio(0.24), sigma=[row[:3] for row in GREY_SIGMA[:n_bins]],
               eps=[row[:3] for row in GREY_EPS[:n_bins]])
    state = dict(nH=nH, x5=x5, T=np.full(C, 100.0), N=np.zeros((n_bins, C)), fr=np.zeros((n_bins, 3, C)),
                 cells=cells, Q=Q)
    return mesh, cfg, state
