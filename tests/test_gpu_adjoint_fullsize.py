"""Gradients of the differentiable workload at its own size: a 64^3
jittered-lattice Voronoi mesh (262,144 cells), lognormal n_H, 8 sources with
Q ~ U(1e49, 1e50) photons/s, the H+He network with thermal energy, 50 FP64
subcycles with a checkpoint every 10.  Loss: the mass-weighted ionised
fraction of the cells whose generators lie in the 16^3-lattice sub-cube
centred on the first source.

* dL/dQ_k of all 8 sources and dL/dn_H of 20 sampled cells (inside and
  outside the region) from rt_adjoint against central finite differences of
  the GPU forward (relative step h = 1e-4, then h/2 and h/4).  Where the
  difference quotients of two successive steps agree within the tolerance,
  the smaller step's is compared; where no two agree, the +-h runs crossed a
  branch of the forward (a limiter choice, an accepted or rejected chemistry
  attempt), where the map is not differentiable, and the component is
  dropped and counted.
* dL/dQ, dL/dn_H and the cotangents of the initial abundances and
  temperature from rt_adjoint against the oracle's reverse mode on the same
  mesh and sources over 5 subcycles (the serial oracle's reverse mode over
  all 50 subcycles would take many minutes).  The cotangent of the initial
  radiation is compared on the same mesh with a faint positive field in
  every cell: where the field is identically zero the limiter of Sec. 2.3.2
  is positively homogeneous in a perturbation but not linear, so that
  cotangent is a choice among one-sided derivatives, not a derivative.

The loss weights m_i = n_H,i V_i depend on n_H: dL/dn_H is the adjoint's
(the weights held fixed) plus V_i (x_HII,i - L) / sum m over the region.
"""
import numpy as np
import pytest

import bench
from tests._cases import make_oracle
from tests.test_gpu_parity import make_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

H = 1e-4
FD_TOL = 1e-5


def rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def _loss_parts(mesh, st):
    R = st["region"]
    m = st["nH"] * mesh.volume
    w = np.zeros(mesh.n_cells)
    w[R] = m[R] / m[R].sum()
    return R, m, w


def test_config4_gradients_vs_fd():
    mesh, cfg, st = bench.differentiable(64)
    C = mesh.n_cells
    n_sub, k = 50, 10
    R, m, w = _loss_parts(mesh, st)
    rt = make_gpu(mesh, cfg, st)
    dt = rt.max_dt() * n_sub
    lx = np.zeros((5, C))
    lx[1] = w
    adj = rt.adjoint(dt, n_sub, k, lam_x5=lx, n_src=len(st["cells"]))
    x_final = rt.fields()["x5"][1]
    L0 = float((w * x_final).sum())
    # dL/dlog Q_k (all bins of source k scaled together) and dL/dn_H
    gQ = (adj["dQ"] * st["Q"]).sum(axis=1)
    gn = adj["dnH"].copy()
    gn[R] += mesh.volume[R] * (x_final[R] - L0) / m[R].sum()

    def loss(Q=None, nH=None):
        nH = st["nH"] if nH is None else nH
        rt.set_gas(nH, st["x5"], st["T"])
        rt.set_radiation(st["N"], st["fr"] * cfg["c_red"])
        rt.set_sources(st["cells"], st["Q"] if Q is None else Q)
        rt.step(dt, n_sub)
        assert rt.sync() == 0
        x = rt.fields()["x5"][1]
        mm = nH * mesh.volume
        return float((mm[R] * x[R]).sum() / mm[R].sum())

    assert loss() == pytest.approx(L0, rel=1e-14)   # the adjoint's forward is the plain forward

    def fd(perturb, h):
        return (loss(**perturb(1 + h)) - loss(**perturb(1 - h))) / (2 * h)

    def fd_checked(perturb, floor):
        """The smaller step of the first two successive steps whose
        quotients agree, or None."""
        prev = fd(perturb, H)
        for h in (H / 2, H / 4):
            cur = fd(perturb, h)
            if abs(prev - cur) <= FD_TOL * abs(cur) + floor:
                return cur, prev
            prev = cur
        return None, prev

    rng = np.random.default_rng(9)
    inside = rng.choice(np.where(R)[0], 14, replace=False)
    outside = rng.choice(np.where(~R)[0], 4, replace=False)
    sample_cells = list(inside) + list(outside) + list(st["cells"][:2])
    comps = []
    for j in range(len(st["cells"])):
        def pq(s, j=j):
            Q = st["Q"].copy()
            Q[j] *= s
            return dict(Q=Q)
        comps.append((f"Q{j}", pq, gQ[j]))
    for i in sample_cells:
        def pn(s, i=i):
            n = st["nH"].copy()
            n[i] *= s
            return dict(nH=n)
        comps.append((f"nH{i}", pn, gn[i] * st["nH"][i]))   # dL/dlog n_H,i
    scale = max(abs(g) for _, _, g in comps)
    checked, dropped, worst = 0, [], 0.0
    for name, pert, g in comps:
        floor = 1e-9 * scale   # round-off of a difference quotient of L ~ 1
        f, other = fd_checked(pert, floor)
        if f is None:
            dropped.append((name, other, g))
            continue
        checked += 1
        err = abs(g - f) / (abs(f) + floor / FD_TOL)
        worst = max(worst, err)
        assert abs(g - f) <= FD_TOL * abs(f) + floor, (name, g, f, other)
    print(f"config-4 gradients: {checked} components checked against FD (worst relative error {worst:.2e}), "
          f"{len(dropped)} dropped at branch switches: {dropped}; dL/dlogQ = {gQ.tolist()}")
    assert checked >= len(comps) - 3
    assert "Q0" not in [d[0] for d in dropped]   # the source inside the region is checked
    assert abs(gQ[0]) > 1e-3


@pytest.mark.parametrize("faint_field", [False, True])
def test_config4_adjoint_vs_oracle(faint_field):
    mesh, cfg, st = bench.differentiable(64)
    C = mesh.n_cells
    n_sub = 5
    if faint_field:
        rng = np.random.default_rng(12)
        st = dict(st, N=rng.uniform(1e-12, 1e-11, (3, C)))
        d = rng.standard_normal((3, 3, C))
        st["fr"] = d / np.linalg.norm(d, axis=1, keepdims=True) * (0.5 * st["N"])[:, None, :]
    R, m, w = _loss_parts(mesh, st)
    lx = np.zeros((5, C))
    lx[1] = w
    lT = w * 1e-4   # the final temperature on the path too
    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt() * n_sub
    ref = o.adjoint(dt, n_sub, lam_x5=lx, lam_T=lT)
    assert ref["status"] == 0
    rt = make_gpu(mesh, cfg, st)
    got = rt.adjoint(dt, n_sub, 2, lam_x5=lx, lam_T=lT, n_src=len(st["cells"]))
    gQ_ref = ref["g_src"][:, st["cells"]].T
    e = {"dQ": rel(got["dQ"], gQ_ref), "dnH": rel(got["dnH"], ref["g_nH"]), "x5": rel(got["x5"], ref["lam0"]["x5"]),
         "T": rel(got["T"], ref["lam0"]["T"])}
    if faint_field:
        e["N"] = rel(got["N"], ref["lam0"]["N"])
        e["F"] = rel(got["F"], ref["lam0"]["fr"] / cfg["c_red"])
    print(f"config-4 adjoint vs oracle over {n_sub} subcycles (faint field {faint_field}):",
          {k: f"{v:.2e}" for k, v in e.items()})
    assert max(e.values()) < 1e-9, e
