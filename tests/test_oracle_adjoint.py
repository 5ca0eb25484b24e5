"""Pins of the oracle's adjoint: central finite differences of the forward
oracle, taken where no substep decision changes between the two runs."""
import numpy as np
import pytest

from tests._cases import make_oracle, voronoi_case


def _setup(n=7, chem_mode=1, n_bins=3, **kw):
    mesh, cfg, st = voronoi_case(n=n, n_bins=n_bins, chem_mode=chem_mode, n_src=2, **kw)
    st["N"] *= 0.1
    st["fr"] *= 0.1
    # target region: cells whose centroid lies in the lower half-box corner
    c = mesh.centroids()
    R = np.all(c < 0.5 * mesh.box, axis=1)
    return mesh, cfg, st, R


def _loss(o, mesh, st, R):
    x5, _ = o.gas()
    m = st["nH"][R] * mesh.volume[R]
    return float((m * x5[1][R]).sum() / m.sum())


def _run(mesh, cfg, st, R, n_sub):
    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt() * n_sub
    assert o.step(dt, n_sub) == 0
    return _loss(o, mesh, st, R), o.substeps().copy()


def _adjoint(mesh, cfg, st, R, n_sub):
    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt() * n_sub
    C = mesh.n_cells
    m = st["nH"] * mesh.volume
    M = m[R].sum()
    lx = np.zeros((5, C))
    lx[1][R] = m[R] / M
    out = o.adjoint(dt, n_sub, lam_x5=lx)
    assert out["status"] == 0
    L = _loss(o, mesh, st, R)
    x5, _ = o.gas()
    # direct dependence of the mass-weighted loss on n_H
    g_nH = out["g_nH"].copy()
    g_nH[R] += mesh.volume[R] * (x5[1][R] - L) / M
    g_Q = out["g_src"][:, st["cells"]].T  # [n_src, B]
    return L, g_Q, g_nH


def _fd(mesh, cfg, st, R, n_sub, key, idx, h_rel=1e-4):
    vals, pats = [], []
    for sgn in (1, -1):
        s2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.items()}
        base = s2[key][idx]
        s2[key][idx] = base * (1 + sgn * h_rel)
        L, pat = _run(mesh, cfg, s2, R, n_sub)
        vals.append(L)
        pats.append(pat)
    same = np.array_equal(pats[0], pats[1])
    return (vals[0] - vals[1]) / (2 * h_rel * st[key][idx]), same


@pytest.mark.parametrize("n_sub,chem_mode", [(3, 1), (3, 2)])
def test_adjoint_luminosities_and_densities_vs_fd(n_sub, chem_mode):
    mesh, cfg, st, R = _setup(chem_mode=chem_mode)
    L, g_Q, g_nH = _adjoint(mesh, cfg, st, R, n_sub)
    L0, _ = _run(mesh, cfg, st, R, n_sub)
    assert L == L0
    checked = 0
    for k in range(len(st["cells"])):
        for b in range(cfg["n_bins"]):
            fd, same = _fd(mesh, cfg, st, R, n_sub, "Q", (k, b))
            if not same:
                continue
            scale = max(abs(fd), 1e-12 * abs(L))
            assert abs(g_Q[k, b] - fd) <= 1e-5 * scale + 1e-9 * np.abs(g_Q).max(), (k, b, g_Q[k, b], fd)
            checked += 1
    assert checked >= 4
    rng = np.random.default_rng(0)
    cells = np.concatenate([rng.choice(np.where(R)[0], 4, replace=False),
                            rng.choice(np.where(~R)[0], 2, replace=False), st["cells"]])
    for i in cells:
        fd, same = _fd(mesh, cfg, st, R, n_sub, "nH", i)
        if not same:
            continue
        scale = max(abs(fd), 1e-3 * np.abs(g_nH).max())
        assert abs(g_nH[i] - fd) <= 1e-5 * scale, (i, g_nH[i], fd)
        checked += 1
    assert checked >= 10


@pytest.mark.parametrize("chem_mode", [1, 2])
def test_adjoint_temperature_vs_fd(chem_mode):
    """Mass-weighted temperature of the region R (full thermal network:
    photoheating, cooling, n_tot through the abundances) and the ionised
    fraction (isothermal: T enters only through the rate fits),
    differentiated w.r.t. the initial temperatures and source rates."""
    mesh, cfg, st, R = _setup(chem_mode=chem_mode)
    n_sub = 3
    C = mesh.n_cells
    m = st["nH"] * mesh.volume
    w = np.zeros(C)
    w[R] = m[R] / m[R].sum()
    key = "T" if chem_mode == 2 else "x5"

    def loss(o):
        x5, T = o.gas()
        return float((w * (T if key == "T" else x5[1])).sum())

    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt() * n_sub
    if key == "T":
        out = o.adjoint(dt, n_sub, lam_T=w)
    else:
        lx = np.zeros((5, C))
        lx[1] = w
        out = o.adjoint(dt, n_sub, lam_x5=lx)
    assert out["status"] == 0
    gT = out["lam0"]["T"]
    gQ = out["g_src"][:, st["cells"]].T

    def fd(arr, idx, rel):
        vals, pats = [], []
        for sg in (1, -1):
            s2 = {kk: (v.copy() if isinstance(v, np.ndarray) else v) for kk, v in st.items()}
            s2[arr][idx] *= 1 + sg * rel
            o2 = make_oracle(mesh, cfg, s2)
            assert o2.step(dt, n_sub) == 0
            vals.append(loss(o2))
            pats.append(o2.substeps().copy())
        return (vals[0] - vals[1]) / (2 * rel * st[arr][idx]), np.array_equal(pats[0], pats[1])

    rng = np.random.default_rng(3)
    checked = 0
    for i in np.concatenate([rng.choice(np.where(R)[0], 6, replace=False), st["cells"]]):
        f, same = fd("T", i, 1e-4)
        if not same:
            continue
        assert abs(gT[i] - f) <= 1e-5 * max(abs(f), 1e-3 * np.abs(gT).max()), (i, gT[i], f)
        checked += 1
    for k in range(len(st["cells"])):
        for b in range(cfg["n_bins"]):
            f, same = fd("Q", (k, b), 1e-4)
            if not same:
                continue
            # absolute floor: the finite difference of a loss of order one
            # cannot resolve components below ~1e-6 of the largest
            assert abs(gQ[k, b] - f) <= 1e-5 * abs(f) + 1e-6 * np.abs(gQ).max(), (k, b, gQ[k, b], f)
            checked += 1
    assert checked >= 6
    assert np.abs(gT[R]).max() > 0


def test_adjoint_transport_only_vs_fd():
    """Transport only (absorption off): the photon number in the region R
    after three subcycles, differentiated w.r.t. source rates and the
    initial radiation; exercises gradients, limiter, M1 and the gather."""
    mesh, cfg, st, R = _setup(chem_mode=0)
    n_sub = 3
    C, B = mesh.n_cells, cfg["n_bins"]
    V = mesh.volume

    def loss(o):
        N, _ = o.radiation()
        return float((N[:, R] * V[R]).sum() + 0.3 * (N[0] * V * np.sin(np.arange(C))).sum())

    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt() * n_sub
    lN = np.zeros((B, C))
    lN[:, R] = V[R]
    lN[0] += 0.3 * V * np.sin(np.arange(C))
    out = o.adjoint(dt, n_sub, lam_N=lN)
    assert out["status"] == 0
    gQ = out["g_src"][:, st["cells"]].T
    for k in range(2):
        for b in range(B):
            vals = []
            for sg in (1, -1):
                s2 = {kk: (v.copy() if isinstance(v, np.ndarray) else v) for kk, v in st.items()}
                h = 1e-4 * s2["Q"][k, b]
                s2["Q"][k, b] += sg * h
                o2 = make_oracle(mesh, cfg, s2)
                assert o2.step(dt, n_sub) == 0
                vals.append(loss(o2))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(gQ[k, b] - fd) <= 1e-5 * abs(fd), (k, b, gQ[k, b], fd)
    # initial radiation, a few components
    lam0 = out["lam0"]
    rng = np.random.default_rng(1)
    for i in rng.choice(C, 6, replace=False):
        for (arr, idx) in (("N", (1, i)), ("fr", (2, 1, i))):
            vals = []
            for sg in (1, -1):
                s2 = {kk: (v.copy() if isinstance(v, np.ndarray) else v) for kk, v in st.items()}
                h = 1e-5 * max(abs(s2["N"]).max(), 1e-30)
                s2[arr][idx] += sg * h
                o2 = make_oracle(mesh, cfg, s2)
                assert o2.step(dt, n_sub) == 0
                vals.append(loss(o2))
            fd = (vals[0] - vals[1]) / (2 * h)
            g = lam0[arr][idx]
            assert abs(g - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(lam0["N"]).max()), (arr, idx, g, fd)


def test_adjoint_finite_for_tiny_radiation():
    """Photon densities near 1e-160 (far from any source): no squared
    magnitude in a denominator may underflow to zero in the reverse pass."""
    mesh, cfg, st, R = _setup(n=6)
    st["N"] *= 1e-160
    st["fr"] *= 1e-160
    o = make_oracle(mesh, cfg, st)
    lx = np.zeros((5, mesh.n_cells))
    lx[1] = 1.0
    out = o.adjoint(o.max_dt() * 3, 3, lam_x5=lx)
    assert out["status"] == 0
    for a in (out["g_src"], out["g_nH"], out["lam0"]["N"], out["lam0"]["fr"], out["lam0"]["x5"]):
        assert np.isfinite(a).all()


def test_adjoint_neutral_start_thermal():
    """Neutral gas (n_e = 0) and no radiation at the start, full thermal
    network: the reverse mode stays finite and matches finite differences
    of the source rates (the cooling slope in n_e needs no division)."""
    mesh, cfg, st, R = _setup(chem_mode=2)
    C = mesh.n_cells
    st["x5"] = np.zeros((5, C))
    st["x5"][0] = 1.0
    st["x5"][2] = 1.0
    st["N"][:] = 0.0
    st["fr"][:] = 0.0
    L, g_Q, g_nH = _adjoint(mesh, cfg, st, R, 3)
    assert np.isfinite(g_Q).all() and np.isfinite(g_nH).all()
    for k in range(len(st["cells"])):
        fd, same = _fd(mesh, cfg, st, R, 3, "Q", (k, 0))
        if same:
            assert abs(g_Q[k, 0] - fd) <= 1e-5 * abs(fd) + 1e-6 * np.abs(g_Q).max(), (k, g_Q[k, 0], fd)
