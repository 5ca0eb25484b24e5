"""Python binding of libm1rt.so (include/rt.h): argument marshalling only.

Every step of the RT subcycle runs in the library's CUDA kernels; there is no
CPU path.  If the library cannot be loaded, the functions here raise.

Module-level functions carry the C names (``rt_create``, ``rt_init_mesh``,
``rt_step`` ...) and take plain arrays: numpy arrays or torch tensors (host or
CUDA), float64/int32/int64 as the header states.  ``RT`` wraps one context.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

RT_OK, RT_INVALID_ARG, RT_BAD_MESH, RT_CFL, RT_CHEM_SUBSTEPS, RT_NONFINITE, RT_OOM, RT_CUDA, RT_NOT_READY, RT_TIMEOUT = \
    range(10)
RT_FP64, RT_MIXED = 0, 1
RT_FIELD_N, RT_FIELD_F, RT_FIELD_X, RT_FIELD_T, RT_FIELD_NSUB = 1, 2, 4, 8, 16

STATUS_NAMES = {0: "RT_OK", 1: "RT_INVALID_ARG", 2: "RT_BAD_MESH", 3: "RT_CFL", 4: "RT_CHEM_SUBSTEPS",
                5: "RT_NONFINITE", 6: "RT_OOM", 7: "RT_CUDA", 8: "RT_NOT_READY",
                9: "RT_TIMEOUT"}


class RTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class rt_config(ctypes.Structure):
    _fields_ = [
        ("n_bins", ctypes.c_int),
        ("precision", ctypes.c_int),
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
        ("gather_sum", ctypes.c_int),
        ("splitting", ctypes.c_int),
        ("time_order", ctypes.c_int),
    ]


class rt_cells(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(k, ctypes.c_void_p) for k in ("volume", "cx", "cy", "cz")]


class rt_faces(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("left", ctypes.c_void_p), ("right", ctypes.c_void_p)] + \
               [(k, ctypes.c_void_p) for k in ("area", "nx", "ny", "nz", "fx", "fy", "fz")]


def make_config(**kw) -> rt_config:
    """rt_config with the method's defaults; keywords override (``sigma`` and
    ``eps`` take nested [bin][species] lists)."""
    c = rt_config()
    defaults = dict(n_bins=3, precision=RT_FP64, c_red=0.01 * 2.99792458e10, unit_length_cm=3.0856775814913673e21,
                    box=0.0, cfl=0.3, chem_mode=2, chem_flags=15, limiter=1, lim_eps=1e-5, order=2, f_s=0.05,
                    f_max=0.1, x_floor=1e-4, max_substeps=10000, y_he=0.0, gather_sum=0,
                    splitting=0, time_order=1)
    defaults.update(kw)
    for k, v in defaults.items():
        if k in ("sigma", "eps"):
            arr = getattr(c, k)
            for b in range(3):
                for s in range(3):
                    arr[b][s] = float(v[b][s]) if b < len(v) else 0.0
        elif k == "precision" and isinstance(v, str):
            c.precision = {"fp64": RT_FP64, "mixed": RT_MIXED}[v]
        else:
            setattr(c, k, v)
    return c


_LIB = None
_LOCK = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load():
    """Load libm1rt.so (building it first if the sources are newer)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libm1rt.so not found at {path}")
            lib = ctypes.CDLL(path)
            vp, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
            sig = {
                "rt_create": [ctypes.POINTER(rt_config), vp, ctypes.POINTER(vp)],
                "rt_set_stream": [vp, vp],
                "rt_init_mesh": [vp, ctypes.POINTER(rt_cells), ctypes.POINTER(rt_faces)],
                "rt_set_gas": [vp, vp, vp, vp],
                "rt_set_radiation": [vp, vp, vp],
                "rt_set_sources": [vp, i64, vp, vp],
                "rt_set_active": [vp, vp],
                "rt_step": [vp, dbl, i32],
                "rt_sync": [vp],
                "rt_get_fields": [vp, ctypes.c_uint32, ctypes.POINTER(vp)],
                "rt_max_dt": [vp, ctypes.POINTER(dbl)],
                "rt_mesh_info": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32)],
                "rt_stage_gradients": [vp, vp],
                "rt_stage_fluxes": [vp, vp, vp],
                "rt_stage_transport": [vp, dbl],
                "rt_stage_chemistry": [vp, dbl],
                "rt_profile_enable": [vp, i32],
                "rt_profile_read": [vp, i32, ctypes.POINTER(dbl), ctypes.POINTER(i64), i32],
                "rt_launch_count": [vp, ctypes.POINTER(i64)],
                "rt_selftest_wait_timeout": [vp, ctypes.c_uint32],
                "rt_adjoint": [vp, dbl, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp],
                "rt_adjoint_tape_info": [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(ctypes.c_int)],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.rt_gradients_noalloc.argtypes = [ctypes.POINTER(rt_cells), ctypes.POINTER(rt_faces), vp, vp, i32, i32,
                                                 i32, dbl, dbl, vp, vp, vp, vp, vp]
            lib.rt_gradients_noalloc.restype = ctypes.c_int
            lib.rt_fp64_peak.argtypes = [vp, i32, i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
            lib.rt_fp64_peak.restype = ctypes.c_int
            lib.rt_fp64_peak_last_error.argtypes = []
            lib.rt_fp64_peak_last_error.restype = ctypes.c_char_p
            lib.rt_noalloc_last_error.argtypes = []
            lib.rt_noalloc_last_error.restype = ctypes.c_char_p
            lib.rt_last_error.argtypes = [vp]
            lib.rt_last_error.restype = ctypes.c_char_p
            lib.rt_destroy.argtypes = [vp]
            lib.rt_destroy.restype = None
            _LIB = lib
    return _LIB


# ---------------------------------------------------------------------------
# argument marshalling
# ---------------------------------------------------------------------------

def _ptr(a, dtype, keep: list):
    """Raw pointer of a numpy array or torch tensor of ``dtype`` (contiguous)."""
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            tdt = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64,
                   np.uint8: torch.uint8}[dtype]
            t = a.detach()
            if t.dtype != tdt:
                raise TypeError(f"expected a {tdt} tensor, got {t.dtype}")
            t = t.contiguous()
            keep.append(t)
            return t.data_ptr()
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    keep.append(arr)
    return arr.ctypes.data


def _check(lib, ctx, st):
    if st != RT_OK:
        raise RTError(st, (lib.rt_last_error(ctx) or b"").decode())
    return st


def rt_create(cfg: rt_config, stream=None):
    lib = load()
    out = ctypes.c_void_p()
    s = _stream_handle(stream)
    _check(lib, None, lib.rt_create(ctypes.byref(cfg), s, ctypes.byref(out)))
    return out


def rt_set_stream(ctx, stream):
    lib = load()
    return _check(lib, ctx, lib.rt_set_stream(ctx, _stream_handle(stream)))


def rt_last_error(ctx=None) -> str:
    return (load().rt_last_error(ctx) or b"").decode()


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return getattr(stream, "cuda_stream", None) or getattr(stream, "value", None)


def rt_init_mesh(ctx, mesh):
    lib = load()
    keep = []
    cells = rt_cells(mesh.n_cells, *[_ptr(getattr(mesh, k), np.float64, keep) for k in ("volume", "cx", "cy", "cz")])
    faces = rt_faces(mesh.n_faces, _ptr(mesh.left, np.int32, keep), _ptr(mesh.right, np.int32, keep),
                     *[_ptr(getattr(mesh, k), np.float64, keep) for k in ("area", "nx", "ny", "nz", "fx", "fy", "fz")])
    return _check(lib, ctx, lib.rt_init_mesh(ctx, ctypes.byref(cells), ctypes.byref(faces)))


def rt_set_gas(ctx, nH, x5, T):
    lib, keep = load(), []
    return _check(lib, ctx, lib.rt_set_gas(ctx, _ptr(nH, np.float64, keep), _ptr(x5, np.float64, keep),
                                           _ptr(T, np.float64, keep)))


def rt_set_radiation(ctx, N, F=None):
    lib, keep = load(), []
    return _check(lib, ctx, lib.rt_set_radiation(ctx, _ptr(N, np.float64, keep), _ptr(F, np.float64, keep)))


def rt_set_sources(ctx, cells, Q):
    lib, keep = load(), []
    n = 0 if cells is None else len(cells)
    return _check(lib, ctx, lib.rt_set_sources(ctx, n, _ptr(cells, np.int64, keep) if n else None,
                                               _ptr(Q, np.float64, keep) if n else None))


def rt_set_active(ctx, active):
    """Individual time steps: active[C] (nonzero = active; numpy or torch,
    host or device) for the following steps; None = every cell active."""
    lib, keep = load(), []
    return _check(lib, ctx, lib.rt_set_active(ctx, None if active is None else _ptr(active, np.uint8, keep)))


def rt_step(ctx, dt, n_sub):
    lib = load()
    return _check(lib, ctx, lib.rt_step(ctx, float(dt), int(n_sub)))


def rt_sync(ctx):
    lib = load()
    return _check(lib, ctx, lib.rt_sync(ctx))


def rt_get_fields(ctx, mask, outs):
    """outs: list of writable float64 arrays/tensors, one per set bit of mask."""
    lib, keep = load(), []
    ptrs = (ctypes.c_void_p * max(len(outs), 1))(*[_out_ptr(o) for o in outs])
    return _check(lib, ctx, lib.rt_get_fields(ctx, int(mask), ptrs))


def _out_ptr(o):
    try:
        import torch
        if isinstance(o, torch.Tensor):
            if o.dtype != torch.float64 or not o.is_contiguous():
                raise TypeError("outputs must be contiguous float64")
            return o.data_ptr()
    except ImportError:
        pass
    if not (isinstance(o, np.ndarray) and o.dtype == np.float64 and o.flags.c_contiguous):
        raise TypeError("outputs must be contiguous float64")
    return o.ctypes.data


def rt_max_dt(ctx):
    lib = load()
    out = ctypes.c_double()
    _check(lib, ctx, lib.rt_max_dt(ctx, ctypes.byref(out)))
    return out.value


def rt_mesh_info(ctx):
    lib = load()
    c, f, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(lib, ctx, lib.rt_mesh_info(ctx, ctypes.byref(c), ctypes.byref(f), ctypes.byref(d)))
    return c.value, f.value, d.value


def rt_stage_gradients(ctx, G=None):
    lib = load()
    return _check(lib, ctx, lib.rt_stage_gradients(ctx, None if G is None else _out_ptr(G)))


def rt_stage_fluxes(ctx, G=None, flux=None):
    lib, keep = load(), []
    return _check(lib, ctx, lib.rt_stage_fluxes(ctx, _ptr(G, np.float64, keep), None if flux is None else _out_ptr(flux)))


def rt_stage_transport(ctx, dt):
    lib = load()
    return _check(lib, ctx, lib.rt_stage_transport(ctx, float(dt)))


def rt_stage_chemistry(ctx, dt):
    lib = load()
    return _check(lib, ctx, lib.rt_stage_chemistry(ctx, float(dt)))


def rt_gradients_noalloc(cells: rt_cells, faces: rt_faces, cell_off, cell_faces, n_bins, order, limiter, lim_eps,
                         box, N, F_red, G, bad_cell, stream=None):
    """Allocation-free gradients (see include/rt.h); every array argument is
    a device pointer (int) or a CUDA tensor; cells/faces hold device pointers."""
    lib = load()
    keep = []
    p = lambda a, dt: a if isinstance(a, int) else _ptr(a, dt, keep)
    st = lib.rt_gradients_noalloc(ctypes.byref(cells), ctypes.byref(faces), p(cell_off, np.int32),
                                  p(cell_faces, np.int32), int(n_bins), int(order), int(limiter), float(lim_eps),
                                  float(box), p(N, np.float64), p(F_red, np.float64), _out_ptr(G) if not isinstance(G, int) else G,
                                  bad_cell if isinstance(bad_cell, int) else bad_cell.data_ptr(), _stream_handle(stream))
    if st != RT_OK:
        raise RTError(st, (lib.rt_noalloc_last_error() or b"").decode())
    return st


def rt_fp64_peak(stream=None, iters=4096, reps=5):
    """Measured FP64 peak of the current device (see include/rt.h):
    returns (TFLOP/s, best launch in ms)."""
    lib = load()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    st = lib.rt_fp64_peak(_stream_handle(stream), int(iters), int(reps), ctypes.byref(tf), ctypes.byref(ms))
    if st != RT_OK:
        raise RTError(st, (lib.rt_fp64_peak_last_error() or b"").decode())
    return tf.value, ms.value


def rt_fp64_peak_last_error() -> str:
    return (load().rt_fp64_peak_last_error() or b"").decode()


def rt_noalloc_last_error() -> str:
    return (load().rt_noalloc_last_error() or b"").decode()


def rt_adjoint(ctx, dt, n_sub, checkpoint_every, lam_N=None, lam_F=None, lam_x5=None, lam_T=None, dL_dQ=None,
               dL_dnH=None, lam0_N=None, lam0_F=None, lam0_x5=None, lam0_T=None):
    """Reverse mode of rt_step (see include/rt.h).  Inputs may be None;
    outputs are writable float64 arrays/tensors or None."""
    lib, keep = load(), []
    o = lambda a: None if a is None else _out_ptr(a)
    return _check(lib, ctx, lib.rt_adjoint(ctx, float(dt), int(n_sub), int(checkpoint_every),
                                           _ptr(lam_N, np.float64, keep), _ptr(lam_F, np.float64, keep),
                                           _ptr(lam_x5, np.float64, keep), _ptr(lam_T, np.float64, keep),
                                           o(dL_dQ), o(dL_dnH), o(lam0_N), o(lam0_F), o(lam0_x5), o(lam0_T)))


def rt_adjoint_tape_info(ctx):
    """The last rt_adjoint's chemistry tape: {max_records, capacity, redone}."""
    lib = load()
    m, c, r = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
    _check(lib, ctx, lib.rt_adjoint_tape_info(ctx, ctypes.byref(m), ctypes.byref(c), ctypes.byref(r)))
    return dict(max_records=m.value, capacity=c.value, redone=r.value)


RT_KERNEL_NAMES = ("k_chem", "k_grad", "k_flux", "k_gather")


def rt_profile_enable(ctx, on=True):
    lib = load()
    return _check(lib, ctx, lib.rt_profile_enable(ctx, int(bool(on))))


def rt_profile_read(ctx, reset=True):
    """{kernel: (total ms, launches)} since the last reset."""
    lib = load()
    n = len(RT_KERNEL_NAMES)
    ms, cnt = (ctypes.c_double * n)(), (ctypes.c_int64 * n)()
    _check(lib, ctx, lib.rt_profile_read(ctx, n, ms, cnt, int(bool(reset))))
    return {k: (ms[i], cnt[i]) for i, k in enumerate(RT_KERNEL_NAMES)}


def rt_launch_count(ctx):
    lib = load()
    out = ctypes.c_int64()
    _check(lib, ctx, lib.rt_launch_count(ctx, ctypes.byref(out)))
    return out.value


def rt_selftest_wait_timeout(ctx, polls):
    lib = load()
    _check(lib, ctx, lib.rt_selftest_wait_timeout(ctx, int(polls)))


def rt_destroy(ctx):
    if ctx:
        load().rt_destroy(ctx)


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class RT:
    """One library context: ``RT(cfg, mesh)`` then set_* / step / fields."""

    def __init__(self, cfg: rt_config, mesh=None, stream=None):
        self.cfg = cfg
        self.B = cfg.n_bins
        self.ctx = rt_create(cfg, stream)
        self.C = self.F = 0
        if mesh is not None:
            self.init_mesh(mesh)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            rt_destroy(ctx)
            self.ctx = None

    def set_stream(self, stream):
        rt_set_stream(self.ctx, stream)

    def init_mesh(self, mesh):
        rt_init_mesh(self.ctx, mesh)
        self.C, self.F = mesh.n_cells, mesh.n_faces

    def set_gas(self, nH, x5, T):
        rt_set_gas(self.ctx, nH, x5, T)

    def set_radiation(self, N, F=None):
        rt_set_radiation(self.ctx, N, F)

    def set_sources(self, cells, Q):
        rt_set_sources(self.ctx, cells, Q)

    def set_active(self, active):
        rt_set_active(self.ctx, active)

    def step(self, dt, n_sub):
        rt_step(self.ctx, dt, n_sub)

    def sync(self):
        return rt_sync(self.ctx)

    def max_dt(self):
        return rt_max_dt(self.ctx)

    def mesh_info(self):
        return rt_mesh_info(self.ctx)

    def fields(self):
        """All fields as numpy arrays: N [B,C], F [B,3,C], x5 [5,C], T [C], nsub [C]."""
        B, C = self.B, self.C
        N, F, x5, T, ns = (np.empty((B, C)), np.empty((B, 3, C)), np.empty((5, C)), np.empty(C), np.empty(C))
        rt_get_fields(self.ctx, RT_FIELD_N | RT_FIELD_F | RT_FIELD_X | RT_FIELD_T | RT_FIELD_NSUB, [N, F, x5, T, ns])
        return dict(N=N, F=F, x5=x5, T=T, nsub=ns.astype(np.int64))

    def radiation(self):
        N, F = np.empty((self.B, self.C)), np.empty((self.B, 3, self.C))
        rt_get_fields(self.ctx, RT_FIELD_N | RT_FIELD_F, [N, F])
        return N, F

    def gradients(self):
        G = np.empty((self.C, self.B, 4, 3))
        rt_stage_gradients(self.ctx, G)
        return G

    def face_fluxes(self, G=None):
        out = np.empty((self.F, self.B, 4))
        rt_stage_fluxes(self.ctx, G, out)
        return out

    def adjoint(self, dt, n_sub, checkpoint_every, lam_N=None, lam_F=None, lam_x5=None, lam_T=None, n_src=0):
        """Reverse mode of step(dt, n_sub) from the current state (which it
        advances).  Returns numpy dL/dQ [n_src, B], dL/dn_H [C] and the
        cotangents of the initial fields."""
        B, C = self.B, self.C
        out = dict(dQ=np.empty((n_src, B)), dnH=np.empty(C), N=np.empty((B, C)), F=np.empty((B, 3, C)),
                   x5=np.empty((5, C)), T=np.empty(C))
        rt_adjoint(self.ctx, dt, n_sub, checkpoint_every, lam_N, lam_F, lam_x5, lam_T,
                   out["dQ"] if n_src else None, out["dnH"], out["N"], out["F"], out["x5"], out["T"])
        return out

    def adjoint_tape_info(self):
        return rt_adjoint_tape_info(self.ctx)

    def transport(self, dt):
        rt_stage_transport(self.ctx, dt)

    def thermochemistry(self, dt):
        rt_stage_chemistry(self.ctx, dt)
