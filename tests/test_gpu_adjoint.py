"""GPU reverse mode (rt_adjoint) against the oracle's reverse mode and
against central finite differences of the GPU forward."""
import numpy as np
import pytest

from tests._cases import make_oracle, voronoi_case
from tests.test_gpu_parity import make_gpu

pytestmark = pytest.mark.gpu


def _setup(n=8, chem_mode=1, n_src=2, n_bins=3):
    mesh, cfg, st = voronoi_case(n=n, n_bins=n_bins, chem_mode=chem_mode, n_src=n_src)
    st["N"] *= 0.1
    st["fr"] *= 0.1
    c = mesh.centroids()
    R = np.all(c < 0.5 * mesh.box, axis=1)
    return mesh, cfg, st, R


def _loss_cot(mesh, st, R):
    m = st["nH"] * mesh.volume
    lx = np.zeros((5, mesh.n_cells))
    lx[1][R] = m[R] / m[R].sum()
    return lx


def rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def oracle_tape_records(mesh, cfg, st, dt, n_sub, k):
    """Chemistry records per segment of k subcycles as the oracle's forward
    counts them: every attempt of each cell that made more than one."""
    o = make_oracle(mesh, cfg, st)
    per = []
    for _ in range(n_sub):
        o.step(dt / n_sub, 1)
        ns = np.asarray(o.substeps())
        per.append(int(ns[ns > 1].sum()))
    return [sum(per[i:i + k]) for i in range(0, n_sub, k)]


TAPE_INITIAL = 4096   # the tape's first capacity, max(4096, C / 4) records, for these 512-cell meshes


@pytest.mark.parametrize("chem_mode,k", [(1, 4), (1, 2), (0, 3), (2, 4), (2, 1)])
def test_adjoint_matches_oracle(chem_mode, k):
    """Modes 0-2; in mode 2 the loss also weighs the final temperature, so
    the energy equation, photoheating, cooling and the rate slopes in T are
    all on the path."""
    mesh, cfg, st, R = _setup(chem_mode=chem_mode)
    n_sub = 4
    lx = _loss_cot(mesh, st, R)
    lN = np.zeros((3, mesh.n_cells))
    lN[:, R] = mesh.volume[R]
    lT = lx[1] * 1e-4 if chem_mode == 2 else None
    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt() * n_sub
    ref = o.adjoint(dt, n_sub, lam_N=lN, lam_x5=lx, lam_T=lT)
    assert ref["status"] == 0
    rt = make_gpu(mesh, cfg, st)
    got = rt.adjoint(dt, n_sub, k, lam_N=lN, lam_x5=lx, lam_T=lT, n_src=len(st["cells"]))
    assert rel(got["T"], ref["lam0"]["T"]) < 1e-9
    gQ_ref = ref["g_src"][:, st["cells"]].T
    assert rel(got["dQ"], gQ_ref) < 1e-9
    assert rel(got["dnH"], ref["g_nH"]) < 1e-9
    assert rel(got["N"], ref["lam0"]["N"]) < 1e-9
    # dL/dF = dL/d(F/c) / c
    assert rel(got["F"], ref["lam0"]["fr"] / cfg["c_red"]) < 1e-9
    assert rel(got["x5"], ref["lam0"]["x5"]) < 1e-9
    # the forward part left the same final state as a plain step
    N1, _ = o.radiation()
    assert rel(rt.radiation()[0], N1) < 1e-12
    # the tape held the oracle's attempts; a subcycle that overflowed the
    # first capacity was recorded again (the mode-1 and mode-2 cases do)
    segs = oracle_tape_records(mesh, cfg, st, dt, n_sub, k)
    info = rt.adjoint_tape_info()
    assert info["max_records"] == max(segs), (info, segs)
    assert info["max_records"] <= info["capacity"]
    assert (info["redone"] > 0) == (max(segs) > TAPE_INITIAL), (info, segs)


@pytest.mark.parametrize("n_bins", [1, 2])
def test_adjoint_matches_oracle_fewer_bins(n_bins):
    """The reverse chemistry is compiled per bin count (its state arrays in
    registers): one and two bins against the oracle, full thermal network."""
    mesh, cfg, st, R = _setup(chem_mode=2, n_bins=n_bins)
    n_sub, k = 4, 2
    lx = _loss_cot(mesh, st, R)
    lN = np.zeros((n_bins, mesh.n_cells))
    lN[:, R] = mesh.volume[R]
    lT = lx[1] * 1e-4
    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt() * n_sub
    ref = o.adjoint(dt, n_sub, lam_N=lN, lam_x5=lx, lam_T=lT)
    assert ref["status"] == 0
    rt = make_gpu(mesh, cfg, st)
    got = rt.adjoint(dt, n_sub, k, lam_N=lN, lam_x5=lx, lam_T=lT, n_src=len(st["cells"]))
    gQ_ref = ref["g_src"][:, st["cells"]].T
    e = {"dQ": rel(got["dQ"], gQ_ref), "dnH": rel(got["dnH"], ref["g_nH"]), "N": rel(got["N"], ref["lam0"]["N"]),
         "F": rel(got["F"], ref["lam0"]["fr"] / cfg["c_red"]), "x5": rel(got["x5"], ref["lam0"]["x5"]),
         "T": rel(got["T"], ref["lam0"]["T"])}
    assert max(e.values()) < 1e-9, e
    assert rt.adjoint_tape_info()["max_records"] > 0   # the chains ran through the tape


def test_adjoint_finite_for_tiny_radiation():
    mesh, cfg, st, R = _setup(n=6)
    st["N"] *= 1e-160
    st["fr"] *= 1e-160
    rt = make_gpu(mesh, cfg, st)
    lx = np.zeros((5, mesh.n_cells))
    lx[1] = 1.0
    out = rt.adjoint(rt.max_dt() * 3, 3, 2, lam_x5=lx, n_src=2)
    for k in ("dQ", "dnH", "N", "F", "x5"):
        assert np.isfinite(out[k]).all(), k


def test_adjoint_finite_from_neutral_thermal():
    """Neutral start (n_e = 0), no radiation, full thermal network."""
    mesh, cfg, st, R = _setup(n=6, chem_mode=2)
    C = mesh.n_cells
    st["x5"] = np.zeros((5, C))
    st["x5"][0] = 1.0
    st["x5"][2] = 1.0
    st["N"][:] = 0.0
    st["fr"][:] = 0.0
    rt = make_gpu(mesh, cfg, st)
    out = rt.adjoint(rt.max_dt() * 3, 3, 2, lam_x5=_loss_cot(mesh, st, R), n_src=2)
    for k in ("dQ", "dnH", "N", "F", "x5", "T"):
        assert np.isfinite(out[k]).all(), k


def test_adjoint_checkpointing_is_exact():
    mesh, cfg, st, R = _setup()
    lx = _loss_cot(mesh, st, R)
    outs = []
    for k in (1, 3, 6):
        rt = make_gpu(mesh, cfg, st)
        dt = rt.max_dt() * 6
        outs.append(rt.adjoint(dt, 6, k, lam_x5=lx, n_src=2))
    for o in outs[1:]:
        np.testing.assert_array_equal(o["dQ"], outs[0]["dQ"])
        np.testing.assert_array_equal(o["dnH"], outs[0]["dnH"])


def test_autograd_function_vs_fd():
    """torch.autograd through RTStepFunction: dL/dQ and dL/dn_H of the
    mass-weighted ionised fraction in a region, against central FD
    (h = 1e-4 relative) of the GPU forward."""
    import torch
    from paper_2404_17630_gb300 import rt_step_autograd
    mesh, cfg, st, R = _setup()
    dev = torch.device("cuda", 0)
    rt = make_gpu(mesh, cfg, st)
    n_sub = 5
    dt = rt.max_dt() * n_sub
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    Rm = t(R.astype(np.float64))
    V = t(mesh.volume)
    Q = t(st["Q"]).requires_grad_(True)
    nH = t(st["nH"]).requires_grad_(True)
    args = (t(st["N"]), t(st["fr"] * cfg["c_red"]), t(st["x5"]), t(st["T"]))

    def loss(Qv, nHv):
        N, F, x5, T = rt_step_autograd(rt, st["cells"], Qv, nHv, *args, dt, n_sub, 2)
        m = nHv * V * Rm
        return (m * x5[1]).sum() / m.sum()

    L = loss(Q, nH)
    L.backward()
    gQ, gn = Q.grad.cpu().numpy(), nH.grad.cpu().numpy()

    def Lval(Qv, nHv):
        with torch.no_grad():
            return float(loss(Qv, nHv))

    for kk in range(2):
        for b in range(3):
            vals = []
            for sg in (1, -1):
                Q2 = Q.detach().clone()
                Q2[kk, b] *= (1 + sg * 1e-4)
                vals.append(Lval(Q2, nH.detach()))
            fd = (vals[0] - vals[1]) / (2e-4 * float(Q.detach()[kk, b]))
            assert abs(gQ[kk, b] - fd) <= 1e-5 * abs(fd) + 1e-8 * np.abs(gQ).max(), (kk, b, gQ[kk, b], fd)
    rng = np.random.default_rng(2)
    for i in list(rng.choice(np.where(R)[0], 3, replace=False)) + list(st["cells"]):
        vals = []
        for sg in (1, -1):
            n2 = nH.detach().clone()
            n2[i] *= (1 + sg * 1e-4)
            vals.append(Lval(Q.detach(), n2))
        fd = (vals[0] - vals[1]) / (2e-4 * float(nH.detach()[i]))
        assert abs(gn[i] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gn).max()), (i, gn[i], fd)
