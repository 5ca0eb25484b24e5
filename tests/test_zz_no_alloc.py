"""The allocation-free gradient entry point, rt_gradients_noalloc.

It serves callers that cannot allocate device memory (a framework that owns
every device buffer, a loop that must not allocate, a plug-in handed only
device pointers): they pass the mesh and state as device arrays and the
library uses a static device array as its only scratch.  Checked here
through the C ABI against the context-based rt_stage_gradients, on two calls
in a row (the second call reuses the static scratch the first one filled).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from tests._cases import voronoi_case

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _csr(mesh):
    """Per-cell face lists, ascending face order, entry (face << 1) | side."""
    C, F = mesh.n_cells, mesh.n_faces
    deg = np.bincount(mesh.left, minlength=C) + np.bincount(mesh.right, minlength=C)
    off = np.zeros(C + 1, np.int64)
    off[1:] = np.cumsum(deg)
    ent = np.empty(2 * F, np.int64)
    fill = off[:-1].copy()
    for f in range(F):
        for cell, side in ((mesh.left[f], 0), (mesh.right[f], 1)):
            ent[fill[cell]] = (f << 1) | side
            fill[cell] += 1
    return off.astype(np.int32), ent.astype(np.int32)


def test_gradients_noalloc_matches_context_path():
    import torch
    from paper_2404_17630_gb300 import rt as rtb
    from tests.test_gpu_parity import make_gpu

    mesh, cfg, st = voronoi_case(n=12)
    C, F, B = mesh.n_cells, mesh.n_faces, cfg["n_bins"]
    dev = torch.device("cuda", 0)
    d = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    cx, cy, cz, vol = d(mesh.cx), d(mesh.cy), d(mesh.cz), d(mesh.volume)
    left, right = d(mesh.left, torch.int32), d(mesh.right, torch.int32)
    area, nx, ny, nz = d(mesh.area), d(mesh.nx), d(mesh.ny), d(mesh.nz)
    fx, fy, fz = d(mesh.fx), d(mesh.fy), d(mesh.fz)
    off, ent = _csr(mesh)
    off_d, ent_d = d(off, torch.int32), d(ent, torch.int32)
    cells = rtb.rt_cells(C, vol.data_ptr(), cx.data_ptr(), cy.data_ptr(), cz.data_ptr())
    faces = rtb.rt_faces(F, left.data_ptr(), right.data_ptr(), area.data_ptr(), nx.data_ptr(), ny.data_ptr(),
                         nz.data_ptr(), fx.data_ptr(), fy.data_ptr(), fz.data_ptr())
    bad = torch.zeros(1, dtype=torch.int32, device=dev)

    for call, scale in enumerate((1.0, 3.0)):
        N = st["N"] * scale
        fr = st["fr"] * scale * (1.0 + 0.5 * call)
        fr = fr * np.minimum(1.0, N / np.maximum(np.linalg.norm(fr, axis=1), 1e-300))[:, None, :]
        # existing entry point: context + stage gradients
        s2 = dict(st, N=N, fr=fr)
        ref = make_gpu(mesh, cfg, s2).gradients()
        # allocation-free entry point, same inputs as device arrays
        G = torch.full((C, B, 4, 3), np.nan, dtype=torch.float64, device=dev)
        Nd = d(N.reshape(B * C))
        Fd = d(fr.reshape(3 * B * C))
        rtb.rt_gradients_noalloc(cells, faces, off_d, ent_d, B, cfg["order"], cfg["limiter"], cfg["lim_eps"],
                                 cfg["box"], Nd, Fd, G, bad)
        torch.cuda.synchronize()
        assert int(bad.item()) == 0
        got = G.cpu().numpy()
        assert np.isfinite(got).all()
        for b in range(B):
            for q in range(4):
                s = np.abs(ref[:, b, q]).max()
                err = np.abs(got[:, b, q] - ref[:, b, q]).max() / (s if s > 0 else 1.0)
                assert err < TOL64, (call, b, q, err)


def test_gradients_noalloc_rejects_oversize():
    from paper_2404_17630_gb300 import rt as rtb
    from paper_2404_17630_gb300.rt import RTError, RT_INVALID_ARG
    cells = rtb.rt_cells(262145, None, None, None, None)
    faces = rtb.rt_faces(10, None, None, None, None, None, None, None, None, None)
    lib = rtb.load()
    one = ctypes.c_void_p(1)
    st = lib.rt_gradients_noalloc(ctypes.byref(cells), ctypes.byref(faces), one, one, 3, 2, 1, 1e-5, 1.0, one, one,
                                  one, one, None)
    assert st == RT_INVALID_ARG
    assert "262144" in rtb.rt_noalloc_last_error()
    with pytest.raises(RTError):
        raise RTError(st, rtb.rt_noalloc_last_error())
