"""ctypes front end of rt_oracle.c (test infrastructure only)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBS = {}
_LOCK = threading.Lock()

ST_OK, ST_CFL, ST_CHEM, ST_NONFINITE = 0, 3, 4, 5


class OracleConfig(ctypes.Structure):
    _fields_ = [
        ("n_bins", ctypes.c_int),
        ("c_red", ctypes.c_double),
        ("unit_length_cm", ctypes.c_double),
        ("box", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("chem_mode", ctypes.c_int),
        ("chem_flags", ctypes.c_int),
        ("limiter", ctypes.c_int),
        ("lim_eps", ctypes.c_double),
        ("order", ctypes.c_int),
        ("f_s", ctypes.c_double),
        ("f_max", ctypes.c_double),
        ("x_floor", ctypes.c_double),
        ("max_substeps", ctypes.c_int),
        ("y_he", ctypes.c_double),
        ("sigma", (ctypes.c_double * 3) * 3),
        ("eps", (ctypes.c_double * 3) * 3),
        ("splitting", ctypes.c_int),
        ("time_order", ctypes.c_int),
    ]


def default_config(**kw) -> OracleConfig:
    """Oracle configuration from keyword values (names as in the C struct).
    ``sigma`` and ``eps`` take nested [bin][species] lists."""
    c = OracleConfig()
    c.n_bins = 3
    c.c_red = 0.01 * 2.99792458e10
    c.unit_length_cm = 3.0856775814913673e21
    c.box = 0.0
    c.cfl = 0.3
    c.chem_mode = 2
    c.chem_flags = 15
    c.limiter = 1
    c.lim_eps = 1e-5
    c.order = 2
    c.f_s = 0.05
    c.f_max = 0.1
    c.x_floor = 1e-4
    c.max_substeps = 10000
    c.y_he = 0.0
    c.splitting = 0
    c.time_order = 1
    for k, v in kw.items():
        if k in ("sigma", "eps"):
            arr = getattr(c, k)
            for b in range(3):
                for s in range(3):
                    arr[b][s] = float(v[b][s]) if b < len(v) else 0.0
        else:
            setattr(c, k, v)
    return c


_FLAGS = ["-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def _build_one(out, extra, force):
    src = os.path.join(_HERE, "rt_oracle.c")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_FLAGS, *extra, src, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


def build_oracle_lib(force: bool = False, omp: bool = False) -> str:
    """The single-threaded oracle library; with omp=True the same source
    built with -fopenmp (its per-cell and per-face loops on all host cores,
    bitwise the same results).  Building the single-threaded one also tries
    the OpenMP one, which is optional: without OpenMP support only
    oracle_threads_available() is False."""
    if omp:
        return _build_one(os.path.join(_HERE, "_rt_oracle_omp.so"), ["-fopenmp"], force)
    out = _build_one(os.path.join(_HERE, "_rt_oracle.so"), [], force)
    try:
        build_oracle_lib(force, omp=True)
    except (OSError, subprocess.CalledProcessError):
        pass
    return out


def oracle_threads_available() -> bool:
    try:
        _lib(True)
        return True
    except (OSError, subprocess.CalledProcessError):
        return False


def _lib(omp: bool = False):
    with _LOCK:
        if omp not in _LIBS:
            lib = ctypes.CDLL(build_oracle_lib(omp=omp))
            vp, dp, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
            ip32 = ctypes.POINTER(ctypes.c_int32)
            ip64 = ctypes.POINTER(ctypes.c_int64)
            lib.orc_create.restype = vp
            lib.orc_create.argtypes = [ctypes.POINTER(OracleConfig), i64, i64, dp, dp, dp, dp, ip32, ip32,
                                       dp, dp, dp, dp, dp, dp, dp]
            lib.orc_free.argtypes = [vp]
            lib.orc_set_active.argtypes = [vp, vp]
            lib.orc_set_active.restype = None
            lib.orc_set_radiation.argtypes = [vp, dp, dp]
            lib.orc_set_gas.argtypes = [vp, dp, dp, dp]
            lib.orc_set_sources.argtypes = [vp, i64, ip64, dp]
            lib.orc_set_sources.restype = ctypes.c_int
            lib.orc_get_radiation.argtypes = [vp, dp, dp]
            lib.orc_get_gas.argtypes = [vp, dp, dp]
            lib.orc_get_minv.argtypes = [vp, dp]
            lib.orc_get_substeps.argtypes = [vp, ip64]
            lib.orc_gradients.argtypes = [vp, dp]
            lib.orc_face_fluxes.argtypes = [vp, dp, dp]
            lib.orc_transport.argtypes = [vp, ctypes.c_double]
            lib.orc_thermochemistry.argtypes = [vp, ctypes.c_double]
            lib.orc_thermochemistry.restype = ctypes.c_int
            lib.orc_max_dt.argtypes = [vp]
            lib.orc_max_dt.restype = ctypes.c_double
            lib.orc_step.argtypes = [vp, ctypes.c_double, ctypes.c_int]
            lib.orc_step.restype = ctypes.c_int
            for name in ("orc_alphaB_HII", "orc_alphaB_HeII", "orc_alphaB_HeIII", "orc_beta_HI"):
                getattr(lib, name).argtypes = [ctypes.c_double]
                getattr(lib, name).restype = ctypes.c_double
            lib.orc_adjoint.argtypes = [vp, ctypes.c_double, ctypes.c_int, dp, dp, dp, dp, dp, dp]
            lib.orc_adjoint.restype = ctypes.c_int
            lib.orc_cooling.argtypes = [ctypes.c_double] * 7
            lib.orc_cooling.restype = ctypes.c_double
            lib.orc_rates.argtypes = [ctypes.c_double, dp]
            lib.orc_rates.restype = None
            lib.orc_cooling_coeffs.argtypes = [ctypes.c_double, dp]
            lib.orc_cooling_coeffs.restype = None
            lib.orc_threads.argtypes = [ctypes.c_int]
            lib.orc_threads.restype = ctypes.c_int
            _LIBS[omp] = lib
    return _LIBS[omp]


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def rate_probe(name: str, *args) -> float:
    return getattr(_lib(), "orc_" + name)(*[float(a) for a in args])


def rates(T: float) -> dict:
    """The oracle's rate coefficients at T (cm^3/s)."""
    out = np.empty(6)
    _lib().orc_rates(float(T), _d(out))
    return dict(zip(("alpha_HII", "alpha_HeII", "alpha_HeIII", "beta_HI", "beta_HeI", "beta_HeII"), out))


COOLING_TERMS = ("ce_HI", "ce_HeII", "ci_HI", "ci_HeI", "ci_HeII", "rc_HII", "rc_HeII", "rc_HeIII", "diel_HeII",
                 "ff")


def cooling_coeffs(T: float) -> dict:
    """The oracle's cooling coefficients K_t(T) (erg cm^3/s), Lambda =
    n_e sum_t K_t n_(t): collisional excitation of HI and HeII, collisional
    ionisation of HI, HeI, HeII, recombination to HI, HeI, HeII, dielectronic
    recombination of HeII, and free-free (on n_HII + n_HeII + 4 n_HeIII)."""
    out = np.empty(10)
    _lib().orc_cooling_coeffs(float(T), _d(out))
    return dict(zip(COOLING_TERMS, out))


class Oracle:
    """One oracle instance over a fixed mesh.  Arrays: N [B, C], fr [B, 3, C]
    (reduced flux F/c_red), x5 [5, C] = (x_HI, x_HII, y_HeI, y_HeII, y_HeIII),
    T [C], sources (cell [n], Q [n, B] photons/s)."""

    def __init__(self, cfg: OracleConfig, mesh, threads: int = 1):
        """threads > 1 (or 0: all host cores) runs the per-cell and per-face
        loops of the OpenMP build, bitwise the results of threads = 1."""
        self.cfg = cfg
        self.B = cfg.n_bins
        self.C, self.F = mesh.n_cells, mesh.n_faces
        self._keep = [_f64(getattr(mesh, k)) for k in ("volume", "cx", "cy", "cz")]
        lr = [np.ascontiguousarray(mesh.left, dtype=np.int32), np.ascontiguousarray(mesh.right, dtype=np.int32)]
        fk = [_f64(getattr(mesh, k)) for k in ("area", "nx", "ny", "nz", "fx", "fy", "fz")]
        lib = _lib(threads != 1)
        self.threads = lib.orc_threads(int(threads) if threads > 1 else os.cpu_count() or 1) if threads != 1 else 1
        ip32 = ctypes.POINTER(ctypes.c_int32)
        self._h = lib.orc_create(ctypes.byref(cfg), self.C, self.F, *[_d(a) for a in self._keep],
                                 lr[0].ctypes.data_as(ip32), lr[1].ctypes.data_as(ip32), *[_d(a) for a in fk])
        if not self._h:
            raise ValueError("oracle: invalid mesh or configuration")
        self._lib = lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_free(h)
            self._h = None

    # state -------------------------------------------------------------
    def set_radiation(self, N, fr):
        N, fr = _f64(N).reshape(self.B, self.C), _f64(fr).reshape(self.B, 3, self.C)
        self._lib.orc_set_radiation(self._h, _d(N), _d(fr))

    def set_gas(self, nH, x5, T):
        nH, x5, T = _f64(nH), _f64(x5).reshape(5, self.C), _f64(T)
        self._lib.orc_set_gas(self._h, _d(nH), _d(x5), _d(T))

    def set_sources(self, cells, Q):
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        Q = _f64(Q).reshape(len(cells), self.B)
        st = self._lib.orc_set_sources(self._h, len(cells), cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       _d(Q))
        if st:
            raise ValueError("oracle: source cell out of range")

    def set_active(self, mask):
        """Individual time steps: mask[C] (nonzero = active) for the following
        steps; None = every cell active."""
        if mask is None:
            self._lib.orc_set_active(self._h, None)
            return
        m = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
        self._lib.orc_set_active(self._h, m.ctypes.data_as(ctypes.c_void_p))

    def radiation(self):
        N, fr = np.empty((self.B, self.C)), np.empty((self.B, 3, self.C))
        self._lib.orc_get_radiation(self._h, _d(N), _d(fr))
        return N, fr

    def gas(self):
        x5, T = np.empty((5, self.C)), np.empty(self.C)
        self._lib.orc_get_gas(self._h, _d(x5), _d(T))
        return x5, T

    def minv(self):
        out = np.empty((self.C, 3, 3))
        self._lib.orc_get_minv(self._h, _d(out))
        return out

    def substeps(self):
        out = np.empty(self.C, dtype=np.int64)
        self._lib.orc_get_substeps(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        return out

    # stages --------------------------------------------------------------
    def gradients(self):
        G = np.empty((self.C, self.B, 4, 3))
        self._lib.orc_gradients(self._h, _d(G))
        return G

    def face_fluxes(self, G=None):
        """Face fluxes [F, B, 4] (area times flux per unit area) from the
        gradients G [C, B, 4, 3]; with G None, from the gradients the last
        gradients() or transport() call left (zero before the first)."""
        out = np.empty((self.F, self.B, 4))
        if G is None:
            self._lib.orc_face_fluxes(self._h, None, _d(out))
        else:
            G = _f64(G).reshape(self.C, self.B, 4, 3)
            self._lib.orc_face_fluxes(self._h, _d(G), _d(out))
        return out

    def transport(self, dt):
        self._lib.orc_transport(self._h, float(dt))

    def thermochemistry(self, dt) -> int:
        return self._lib.orc_thermochemistry(self._h, float(dt))

    def max_dt(self) -> float:
        return self._lib.orc_max_dt(self._h)

    def step(self, dt, n_sub) -> int:
        return self._lib.orc_step(self._h, float(dt), int(n_sub))

    def adjoint(self, dt, n_sub, lam_N=None, lam_fr=None, lam_x5=None, lam_T=None):
        """Reverse mode of step(dt, n_sub) from the current state (which it
        advances like step does).  lam_*: cotangents of the final state
        (zero if None).  Returns dict(status, g_src [B, C] = dL/dS per cell and
        bin, g_nH [C], lam0 = cotangents of the initial state)."""
        B, C = self.B, self.C
        lN = np.zeros((B, C)) if lam_N is None else _f64(lam_N).reshape(B, C).copy()
        lfr = np.zeros((B, 3, C)) if lam_fr is None else _f64(lam_fr).reshape(B, 3, C).copy()
        lx = np.zeros((5, C)) if lam_x5 is None else _f64(lam_x5).reshape(5, C).copy()
        lT = np.zeros(C) if lam_T is None else _f64(lam_T).copy()
        g_src, g_nH = np.zeros((B, C)), np.zeros(C)
        st = self._lib.orc_adjoint(self._h, float(dt), int(n_sub), _d(lN), _d(lfr), _d(lx), _d(lT), _d(g_src),
                                   _d(g_nH))
        return dict(status=st, g_src=g_src, g_nH=g_nH, lam0=dict(N=lN, fr=lfr, x5=lx, T=lT))
