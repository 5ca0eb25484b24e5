"""The allocation-free gradient entry point, rt_gradients_noalloc.

It serves callers that cannot allocate device memory (a framework that owns
every device buffer, a loop that must not allocate, a plug-in handed only
device pointers): they pass the mesh and state as device arrays and the
library uses a static device array as its only scratch.  Checked here
through the C ABI against the FP64 oracle's gradients and against the
context-based rt_stage_gradients, on two calls in a row (the second call
reuses the static scratch the first one filled), with the limiter on and
off, first order, a singular least-squares matrix, and arrays that are not
device memory.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from tests._cases import make_oracle, voronoi_case

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _csr(left, right, C):
    """Per-cell face lists, ascending face order, entry (face << 1) | side."""
    F = len(left)
    deg = np.bincount(left, minlength=C) + np.bincount(right, minlength=C)
    off = np.zeros(C + 1, np.int64)
    off[1:] = np.cumsum(deg)
    ent = np.empty(2 * F, np.int64)
    fill = off[:-1].copy()
    for f in range(F):
        for cell, side in ((left[f], 0), (right[f], 1)):
            ent[fill[cell]] = (f << 1) | side
            fill[cell] += 1
    return off.astype(np.int32), ent.astype(np.int32)


class _DeviceMesh:
    """The mesh as caller-owned device arrays (kept alive with the object)."""

    def __init__(self, cx, cy, cz, vol, left, right, area, n, fc):
        import torch
        from paper_2404_17630_gb300 import rt as rtb
        dev = torch.device("cuda", 0)
        d = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        self.C, self.F = len(cx), len(left)
        self.t = [d(cx), d(cy), d(cz), d(vol), d(left, torch.int32), d(right, torch.int32), d(area),
                  d(n[0]), d(n[1]), d(n[2]), d(fc[0]), d(fc[1]), d(fc[2])]
        off, ent = _csr(np.asarray(left), np.asarray(right), self.C)
        self.off, self.ent = d(off, torch.int32), d(ent, torch.int32)
        p = [x.data_ptr() for x in self.t]
        self.cells = rtb.rt_cells(self.C, p[3], p[0], p[1], p[2])
        self.faces = rtb.rt_faces(self.F, p[4], p[5], p[6], p[7], p[8], p[9], p[10], p[11], p[12])
        self.dev = dev


def _from_mesh(mesh):
    return _DeviceMesh(mesh.cx, mesh.cy, mesh.cz, mesh.volume, mesh.left, mesh.right, mesh.area,
                       (mesh.nx, mesh.ny, mesh.nz), (mesh.fx, mesh.fy, mesh.fz))


def _noalloc(dm, N, fr, B, order, limiter, lim_eps, box):
    import torch
    from paper_2404_17630_gb300 import rt as rtb
    G = torch.full((dm.C, B, 4, 3), np.nan, dtype=torch.float64, device=dm.dev)
    bad = torch.full((1,), -1, dtype=torch.int32, device=dm.dev)
    Nd = torch.as_tensor(np.ascontiguousarray(N.reshape(B * dm.C)), device=dm.dev)
    Fd = torch.as_tensor(np.ascontiguousarray(fr.reshape(3 * B * dm.C)), device=dm.dev)
    rtb.rt_gradients_noalloc(dm.cells, dm.faces, dm.off, dm.ent, B, order, limiter, lim_eps, box, Nd, Fd, G, bad)
    torch.cuda.synchronize()
    return G.cpu().numpy(), int(bad.item())


def _rel(got, ref):
    s = np.abs(ref).max()
    return np.abs(got - ref).max() / (s if s > 0 else 1.0)


@pytest.mark.parametrize("limiter", [1, 0])
def test_gradients_noalloc_matches_oracle_and_context_path(limiter):
    from tests.test_gpu_parity import make_gpu

    mesh, cfg, st = voronoi_case(n=12, limiter=limiter)
    B = cfg["n_bins"]
    dm = _from_mesh(mesh)
    for call, scale in enumerate((1.0, 3.0)):
        N = st["N"] * scale
        fr = st["fr"] * scale * (1.0 + 0.5 * call)
        fr = fr * np.minimum(1.0, N / np.maximum(np.linalg.norm(fr, axis=1), 1e-300))[:, None, :]
        s2 = dict(st, N=N, fr=fr)
        oracle = make_oracle(mesh, cfg, s2).gradients()       # the FP64 definition
        context = make_gpu(mesh, cfg, s2).gradients()         # the existing entry point
        got, bad = _noalloc(dm, N, fr, B, cfg["order"], limiter, cfg["lim_eps"], cfg["box"])
        assert bad == 0
        assert np.isfinite(got).all()
        for b in range(B):
            for q in range(4):
                assert _rel(got[:, b, q], oracle[:, b, q]) < TOL64, ("oracle", call, b, q)
                assert _rel(got[:, b, q], context[:, b, q]) < TOL64, ("context", call, b, q)


def test_gradients_noalloc_first_order_is_zero():
    mesh, cfg, st = voronoi_case(n=8)
    dm = _from_mesh(mesh)
    got, bad = _noalloc(dm, st["N"], st["fr"], cfg["n_bins"], 1, 1, cfg["lim_eps"], cfg["box"])
    assert bad == 0
    assert (got == 0.0).all()


def test_gradients_noalloc_singular_matrix():
    """Two cells sharing one face on the x axis: M = A e_x e_x^T is singular
    in both cells.  bad_cell reports it and the gradients stay finite (zero)."""
    C = 2
    dm = _DeviceMesh(np.array([0.0, 1.0]), np.zeros(C), np.zeros(C), np.ones(C), np.array([0]), np.array([1]),
                     np.array([1.0]), (np.array([1.0]), np.zeros(1), np.zeros(1)),
                     (np.array([0.5]), np.zeros(1), np.zeros(1)))
    N = np.array([[1.0, 2.0]])
    fr = np.zeros((1, 3, C))
    got, bad = _noalloc(dm, N, fr, 1, 2, 1, 1e-5, 0.0)
    assert bad == 1
    assert np.isfinite(got).all() and (got == 0.0).all()


def test_gradients_noalloc_refuses_host_arrays():
    """A host array in place of a device array is refused with a status and
    message before anything is enqueued."""
    import torch
    from paper_2404_17630_gb300 import rt as rtb
    from paper_2404_17630_gb300.rt import RTError, RT_INVALID_ARG
    mesh, cfg, st = voronoi_case(n=6)
    dm = _from_mesh(mesh)
    B = cfg["n_bins"]
    host_N = np.ascontiguousarray(st["N"].reshape(-1))
    Fd = torch.as_tensor(np.ascontiguousarray(st["fr"].reshape(-1)), device=dm.dev)
    G = torch.zeros((dm.C, B, 4, 3), dtype=torch.float64, device=dm.dev)
    bad = torch.zeros(1, dtype=torch.int32, device=dm.dev)
    with pytest.raises(RTError) as ei:
        rtb.rt_gradients_noalloc(dm.cells, dm.faces, dm.off, dm.ent, B, 2, 1, 1e-5, cfg["box"],
                                 host_N.ctypes.data, Fd, G, bad)
    assert ei.value.status == RT_INVALID_ARG
    assert "device memory" in rtb.rt_noalloc_last_error()


def test_gradients_noalloc_rejects_oversize():
    from paper_2404_17630_gb300 import rt as rtb
    from paper_2404_17630_gb300.rt import RT_INVALID_ARG
    cells = rtb.rt_cells(262145, None, None, None, None)
    faces = rtb.rt_faces(10, None, None, None, None, None, None, None, None, None)
    lib = rtb.load()
    one = ctypes.c_void_p(1)
    st = lib.rt_gradients_noalloc(ctypes.byref(cells), ctypes.byref(faces), one, one, 3, 2, 1, 1e-5, 1.0, one, one,
                                  one, one, None)
    assert st == RT_INVALID_ARG
    assert "262144" in rtb.rt_noalloc_last_error()
