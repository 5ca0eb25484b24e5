"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test checks the oracle against a closed form, an invariant, a textbook
limit or a brute-force solution -- never against a retyped copy of its own
formula.  Together they are chosen so that a dropped term, a wrong sign or a
transposed index in any stage fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import synth
from tests._cases import base_config, config1, corner_cells, make_oracle, neutral_gas, voronoi_case

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# rates
# ---------------------------------------------------------------------------

def test_caseB_recombination_textbook():
    """alpha_B(HII, 1e4 K) = 2.59e-13 cm^3/s (Osterbrock & Ferland, the value
    the Stroemgren pin of the method uses); hydrogenic scaling
    alpha(Z, T) = Z alpha(1, T / Z^2) ties HeIII to HII."""
    from oracle import rate_probe
    g = golden("textbook_rates.json")
    a = rate_probe("alphaB_HII", 1e4)
    assert abs(a / g["alphaB_HII_1e4K"]["value"] - 1) < 5e-3
    for T in (3e3, 1e4, 4e4, 2e5):
        assert rate_probe("alphaB_HeIII", 4 * T) == pytest.approx(2 * rate_probe("alphaB_HII", T), rel=1e-12)
    # recombination slows with temperature
    Ts = np.logspace(3, 6, 20)
    aa = [rate_probe("alphaB_HII", T) for T in Ts]
    assert all(np.diff(aa) < 0)
    # collisional ionisation is negligible in warm gas and grows steeply
    assert rate_probe("beta_HI", 1e4) < 1e-15
    assert rate_probe("beta_HI", 1e5) > 1e2 * rate_probe("beta_HI", 2e4)


# ---------------------------------------------------------------------------
# geometry and gradients (Sec. 2.3.2)
# ---------------------------------------------------------------------------

def test_cartesian_gradient_is_central_difference():
    """On a Cartesian grid the least-squares gradient of Eq. (normalEquation)
    reduces to the central difference (phi_{i+1} - phi_{i-1}) / (2h)."""
    n, L = 8, 8.0
    mesh = synth.cartesian_mesh(n, L)
    cfg = base_config(box=L, n_bins=1, limiter=0, chem_mode=0)
    rng = np.random.default_rng(3)
    N = rng.uniform(1, 2, size=(1, n ** 3))
    st = dict(N=N, fr=np.zeros((1, 3, n ** 3)), **dict(zip(("nH", "x5", "T"), neutral_gas(n ** 3, 1e-3))))
    o = make_oracle(mesh, cfg, st)
    G = o.gradients()
    phi = N[0].reshape(n, n, n)  # axes (k, j, i)
    h = L / n
    gx = (np.roll(phi, -1, 2) - np.roll(phi, 1, 2)) / (2 * h)
    gy = (np.roll(phi, -1, 1) - np.roll(phi, 1, 1)) / (2 * h)
    gz = (np.roll(phi, -1, 0) - np.roll(phi, 1, 0)) / (2 * h)
    ref = np.stack([gx.reshape(-1), gy.reshape(-1), gz.reshape(-1)], 1)
    np.testing.assert_allclose(G[:, 0, 0, :], ref, rtol=1e-12, atol=1e-14)


def test_lsq_gradient_exact_for_linear_field():
    """The least-squares gradient is exact for a linear field on any mesh
    (M g = sum A d d^T / |d|^2 a = M a); periodic wrap excluded."""
    mesh = synth.voronoi_mesh(10, 10.0, 0.3, seed=5)
    C = mesh.n_cells
    a = np.array([0.3, -1.1, 0.7])
    c = mesh.centroids()
    phi = 20.0 + c @ a
    cfg = base_config(box=10.0, n_bins=1, limiter=0, chem_mode=0)
    st = dict(N=phi[None, :], fr=np.zeros((1, 3, C)), **dict(zip(("nH", "x5", "T"), neutral_gas(C, 1e-3))))
    o = make_oracle(mesh, cfg, st)
    G = o.gradients()[:, 0, 0, :]
    # interior cells: all neighbours without wrap
    wrap = np.zeros(C, bool)
    d = c[mesh.right] - c[mesh.left]
    crosses = np.any(np.abs(d) > 5.0, axis=1)
    wrap[mesh.left[crosses]] = True
    wrap[mesh.right[crosses]] = True
    assert (~wrap).sum() > 100
    np.testing.assert_allclose(G[~wrap], np.broadcast_to(a, G[~wrap].shape), rtol=0, atol=1e-11)


def test_linear_field_reaches_every_face_exactly():
    """Second-order reconstruction on a Voronoi mesh (Sec. 2.3.2-2.3.3): for
    a linear N with F = 0 and no limiter the least-squares gradient is exact,
    so both sides extrapolate to the same N(x_f) at every face centroid; the
    Lax-Friedrichs dissipation then vanishes and each face carries exactly the
    Eddington-limit flux N(x_f)/3 n of F and no N (faces of cells next to
    the periodic boundary, where the field jumps, excluded)."""
    mesh = synth.voronoi_mesh(9, 10.0, 0.3, seed=11)
    C = mesh.n_cells
    a = np.array([0.07, -0.11, 0.05])
    c = mesh.centroids()
    N = 5.0 + c @ a
    cfg = base_config(box=10.0, n_bins=1, limiter=0, chem_mode=0)
    st = dict(N=N[None, :], fr=np.zeros((1, 3, C)), **dict(zip(("nH", "x5", "T"), neutral_gas(C, 1e-3))))
    o = make_oracle(mesh, cfg, st)
    fl = o.face_fluxes(o.gradients())[:, 0, :] / mesh.area[:, None]
    d = c[mesh.right] - c[mesh.left]
    crosses = np.any(np.abs(d) > 5.0, axis=1)
    wrap = np.zeros(C, bool)
    wrap[mesh.left[crosses]] = True
    wrap[mesh.right[crosses]] = True
    inner = ~wrap[mesh.left] & ~wrap[mesh.right]
    xf = np.stack([mesh.fx, mesh.fy, mesh.fz], 1)
    assert inner.sum() > 500
    Nf = 5.0 + xf[inner] @ a
    n = np.stack([mesh.nx, mesh.ny, mesh.nz], 1)[inner]
    np.testing.assert_allclose(fl[inner, 0], 0.0, atol=1e-12)
    np.testing.assert_allclose(fl[inner, 1:], Nf[:, None] * n / 3, rtol=0, atol=1e-12)


def test_limiter_bounds_face_values():
    """With the limiter, the value extrapolated to every face centre lies
    within [min, max] of the cell and its neighbours (Sec. 2.3.2) -- up to
    lim_eps |g||x| on faces nearly normal to g, which do not limit -- and the
    limited gradient is a non-negative multiple (<= 1) of the raw one."""
    mesh, cfg, st = voronoi_case(n=8, n_bins=1, chem_mode=0)
    cfg["limiter"] = 0
    g_raw = make_oracle(mesh, cfg, st).gradients()
    cfg["limiter"] = 1
    o = make_oracle(mesh, cfg, st)
    g_lim = o.gradients()
    C = mesh.n_cells
    c = mesh.centroids()
    fc = np.stack([mesh.fx, mesh.fy, mesh.fz], 1)
    L = mesh.box
    for q in range(4):
        phi = st["N"][0] if q == 0 else st["fr"][0, q - 1]
        lo, hi = phi.copy(), phi.copy()
        np.minimum.at(lo, mesh.left, phi[mesh.right])
        np.minimum.at(lo, mesh.right, phi[mesh.left])
        np.maximum.at(hi, mesh.left, phi[mesh.right])
        np.maximum.at(hi, mesh.right, phi[mesh.left])
        for side in (mesh.left, mesh.right):
            x = fc - c[side]
            x -= L * np.round(x / L)
            gs = g_lim[side, 0, q]
            val = phi[side] + np.einsum("ij,ij->i", gs, x)
            slack = 1e-12 * np.abs(phi).max() + cfg["lim_eps"] * np.linalg.norm(gs, axis=1) * np.linalg.norm(x, axis=1)
            assert np.all(val <= hi[side] + slack)
            assert np.all(val >= lo[side] - slack)
        gr, gl = g_raw[:, 0, q], g_lim[:, 0, q]
        nz = np.linalg.norm(gr, axis=1) > 0
        ratio = np.einsum("ij,ij->i", gl[nz], gr[nz]) / np.einsum("ij,ij->i", gr[nz], gr[nz])
        assert np.all(ratio >= -1e-12) and np.all(ratio <= 1 + 1e-12)
        np.testing.assert_allclose(gl[nz], gr[nz] * ratio[:, None], atol=1e-12 * np.abs(gr).max())
    assert C > 0


# ---------------------------------------------------------------------------
# face flux (Sec. 2.3.3, Eq. RT_flux, Eq. edd)
# ---------------------------------------------------------------------------

def _two_cell(NL, fL, NR, fR):
    """Periodic 2-cell-wide grid (2^3 cells) in first order: face 0 joins
    cell 0 (left) and cell 1 (right) with normal +x."""
    mesh = synth.cartesian_mesh(2, 2.0)
    C = 8
    N = np.zeros((1, C))
    fr = np.zeros((1, 3, C))
    even = np.arange(C) % 2 == 0
    N[0, even], N[0, ~even] = NL, NR
    fr[0, :, even], fr[0, :, ~even] = fL, fR
    cfg = base_config(box=2.0, n_bins=1, order=1, chem_mode=0)
    st = dict(N=N, fr=fr, **dict(zip(("nH", "x5", "T"), neutral_gas(C, 1e-3))))
    o = make_oracle(mesh, cfg, st)
    flux = o.face_fluxes()
    assert mesh.left[0] == 0 and mesh.right[0] == 1 and mesh.nx[0] == 1.0
    return flux[0, 0] / mesh.area[0]


def test_flux_free_streaming_is_upwind():
    """Free streaming along the normal (|F| = c N, F || n): M1 gives chi = 1
    and the Lax-Friedrichs flux at signal speed c reduces to exact upwinding
    of the left state, for both N and F."""
    NL, NR = 2.0, 0.5
    fl = _two_cell(NL, [NL, 0, 0], NR, [NR, 0, 0])
    np.testing.assert_allclose(fl, [NL, NL, 0, 0], rtol=1e-15)
    # against the normal: upwind from the right; the momentum flux N D n is
    # still +N n (radiation pressure does not change sign with direction)
    fl = _two_cell(NL, [-NL, 0, 0], NR, [-NR, 0, 0])
    np.testing.assert_allclose(fl, [-NR, NR, 0, 0], rtol=1e-15)


def test_flux_isotropic_eddington_limit():
    """F = 0: the M1 tensor is the Eddington limit D = I/3, so the flux of F
    is N/3 n plus the Lax-Friedrichs dissipation, and the flux of N is the
    pure dissipation -(N_R - N_L)/2."""
    NL, NR = 3.0, 1.2
    fl = _two_cell(NL, [0, 0, 0], NR, [0, 0, 0])
    np.testing.assert_allclose(fl, [-(NR - NL) / 2, (NL + NR) / 6, 0, 0], rtol=1e-15)


def test_flux_transverse_beam_has_no_normal_pressure():
    """Free streaming parallel to the face (F = c N e_y, n = e_x): D = e_y e_y,
    so no N or normal-F flux crosses the face; the flux of F_y is pure
    dissipation.  Equal states on both sides give exactly zero."""
    N = 1.5
    fl = _two_cell(N, [0, N, 0], N, [0, N, 0])
    np.testing.assert_allclose(fl, [0, 0, 0, 0], atol=1e-15)


def test_eddington_factor_bounds_monotone():
    """chi(f) runs from 1/3 (isotropic) to 1 (free streaming), monotone:
    measured through the normal pressure of a state with F || n."""
    vals = []
    for f in np.linspace(0, 1, 11):
        fl = _two_cell(1.0, [f, 0, 0], 1.0, [f, 0, 0])
        vals.append(fl[1])  # = chi (N = 1, u || n)
    vals = np.array(vals)
    assert vals[0] == pytest.approx(1 / 3, rel=1e-15)
    assert vals[-1] == pytest.approx(1.0, rel=1e-15)
    assert np.all(np.diff(vals) > 0)


def test_eddington_factor_is_a_boosted_isotropic_field():
    """The Levermore closure (Sec. 2.3.3) is the one of radiation that is
    isotropic in some frame: a field isotropic in a frame moving at speed
    beta c along n has, in the lab frame, reduced flux f = 4 beta / (3 +
    beta^2) and Eddington factor chi = (1 + 3 beta^2) / (3 + beta^2) (Lorentz
    transformation of an isotropic intensity).  Inverting the first for beta
    and comparing the second with the oracle's normal pressure checks the
    closure between its end points, where other closures with the same end
    points (Minerbo, Kershaw) differ by several per cent (Kershaw's by 7.6 %
    at f = 0.5)."""
    for f in np.linspace(0.05, 0.95, 19):
        beta = (2.0 - np.sqrt(4.0 - 3.0 * f * f)) / f
        assert 4 * beta / (3 + beta * beta) == pytest.approx(f, rel=1e-14)
        chi = (1 + 3 * beta * beta) / (3 + beta * beta)
        fl = _two_cell(1.0, [f, 0, 0], 1.0, [f, 0, 0])
        assert fl[1] == pytest.approx(chi, rel=1e-13), f
    # an oblique field, equal on both sides (no Lax-Friedrichs dissipation):
    # the flux of F/c through n is N D n with the M1 tensor D = (1 - chi)/2 I
    # + (3 chi - 1)/2 u u, whose u (u.n) part the beams along and across n
    # cannot tell from a (u.n) n
    for f, ang in ((1.0, np.pi / 4), (0.5, np.pi / 3), (0.8, 2.0)):
        u = np.array([np.cos(ang), np.sin(ang), 0.0])
        beta = (2.0 - np.sqrt(4.0 - 3.0 * f * f)) / f
        chi = (1 + 3 * beta * beta) / (3 + beta * beta)
        N = 1.7
        fl = _two_cell(N, N * f * u, N, N * f * u)
        Dn = (1 - chi) / 2 * np.array([1.0, 0, 0]) + (3 * chi - 1) / 2 * u[0] * u
        np.testing.assert_allclose(fl, [N * f * u[0], *(N * Dn)], rtol=1e-13, atol=1e-15)
    # Kershaw's chi = (1 + 2 f^2) / 3 has the same end points and differs
    # from the boosted field by more than the tolerance in between
    f = 0.5
    beta = (2.0 - np.sqrt(4.0 - 3.0 * f * f)) / f
    assert abs((1 + 2 * f * f) / 3 - (1 + 3 * beta * beta) / (3 + beta * beta)) > 1e-2


# ---------------------------------------------------------------------------
# transport invariants
# ---------------------------------------------------------------------------

def test_uniform_field_stays_uniform():
    """Uniform N and F: zero gradients and sum_f A n = 0 per closed cell
    leave the field unchanged up to round-off."""
    mesh = synth.voronoi_mesh(12, 10.0, 0.3, seed=7)
    C = mesh.n_cells
    N = np.full((3, C), 2.5e-4)
    fr = np.zeros((3, 3, C))
    fr[:, 0], fr[:, 1], fr[:, 2] = 1e-4, -0.5e-4, 0.7e-4
    cfg = base_config(box=10.0, chem_mode=0)
    o = make_oracle(mesh, cfg, dict(N=N, fr=fr, **dict(zip(("nH", "x5", "T"), neutral_gas(C, 1e-3)))))
    dt = o.max_dt()
    for _ in range(3):
        o.transport(dt)
    N1, fr1 = o.radiation()
    np.testing.assert_allclose(N1, N, rtol=1e-12)
    np.testing.assert_allclose(fr1, fr, rtol=1e-11)


def test_photon_number_and_flux_conserved_transport_only():
    """Absorption off: sum_i N_i V_i and sum_i F_i V_i are constant to
    round-off, because every face flux enters its two cells with opposite
    signs (Sec. 4.1.3)."""
    mesh, cfg, st = voronoi_case(n=12, chem_mode=0)
    o = make_oracle(mesh, cfg, st)
    V = mesh.volume
    N0, fr0 = o.radiation()
    dt = o.max_dt()
    for _ in range(5):
        o.transport(dt)
    N1, fr1 = o.radiation()
    tot0, tot1 = (N0 * V).sum(1), (N1 * V).sum(1)
    np.testing.assert_allclose(tot1, tot0, rtol=1e-13)
    m0, m1 = (fr0 * V).sum(2), (fr1 * V).sum(2)
    assert np.abs(m1 - m0).max() <= 1e-13 * np.abs(fr0 * V).sum()
    assert np.abs(N1 - N0).max() > 1e-3 * N0.max()  # something did move


@pytest.mark.parametrize("T0", [1.5e4, 6e4, 3e5, 3e6])
def test_cooling_energy_budget(T0):
    """Cooling alone (Sec. 2.3.1, the explicit thermal-energy update):
    without radiation, recombination or collisional ionisation the
    abundances stay fixed, so over one short accepted substep the thermal
    energy 3/2 k n_tot T falls by exactly dt Lambda(T0), with Lambda = n_e
    sum_t K_t n_(t) assembled from the separately written per-term
    coefficients (collisional excitation on n_HI and n_HeII, collisional
    ionisation on n_HI, n_HeI, n_HeII, recombination on n_HII, n_HeII,
    n_HeIII, dielectronic on n_HeII, free-free on n_HII + n_HeII + 4
    n_HeIII).  A coefficient on the wrong species, a dropped n_e or a sign
    fails here."""
    import oracle
    kB = 1.380649e-16
    mesh = synth.cartesian_mesh(2, 2.0)
    C = mesh.n_cells
    cfg = base_config(box=2.0, n_bins=1, chem_mode=2, chem_flags=4)
    rng = np.random.default_rng(int(T0))
    xHII = rng.uniform(0.2, 0.8, C)
    yII = rng.uniform(0.1, 0.4, C)
    yIII = rng.uniform(0.1, 0.4, C)
    x5 = np.stack([1 - xHII, xHII, 1 - yII - yIII, yII, yIII])
    nH = rng.uniform(0.5e-3, 2e-3, C)
    st = dict(N=np.zeros((1, C)), fr=np.zeros((1, 3, C)), nH=nH, x5=x5, T=np.full(C, T0),
              cells=np.zeros(0, np.int64), Q=np.zeros((0, 1)))
    yhe = cfg["y_he"]
    nHe = yhe * nH
    ne = nH * xHII + nHe * (yII + 2 * yIII)
    dens = dict(ce_HI=nH * (1 - xHII), ce_HeII=nHe * yII, ci_HI=nH * (1 - xHII), ci_HeI=nHe * (1 - yII - yIII),
                ci_HeII=nHe * yII, rc_HII=nH * xHII, rc_HeII=nHe * yII, rc_HeIII=nHe * yIII, diel_HeII=nHe * yII,
                ff=nH * xHII + nHe * yII + 4 * nHe * yIII)
    K = oracle.cooling_coeffs(T0)
    assert set(K) == set(dens)
    lam = ne * sum(K[t] * dens[t] for t in K)
    e0 = 1.5 * kB * (nH + nHe + ne) * T0
    dt = 1e-3 * float(np.min(e0 / lam))
    o = make_oracle(mesh, cfg, st)
    assert o.thermochemistry(dt) == 0
    x1, T1 = o.gas()
    np.testing.assert_array_equal(x1, x5)
    assert np.all(o.substeps() == 1)
    e1 = 1.5 * kB * (nH + nHe + ne) * T1
    np.testing.assert_allclose(e1 - e0, -dt * lam, rtol=1e-9)


def _photoionisation_decay(f_s, Gt=2.0):
    """Hydrogen only, isothermal, photoionisation alone (recombination,
    collisions, cooling and heating off) in a uniform one-bin field so thin
    (n_H = 1e-8 against N = 1e-3) that absorption leaves the rate Gamma =
    c sigma N constant: x_HI(t) = x_HI(0) exp(-Gamma t) exactly.  One
    thermochemistry call over Gamma t = Gt with the substep rule at f_s and
    f_max = 2 f_s.  Returns (relative error of x_HI, substeps)."""
    sigma, N0, x0 = 3e-18, 1e-3, 0.99
    mesh = synth.cartesian_mesh(2, 2.0)
    C = mesh.n_cells
    cfg = base_config(box=2.0, n_bins=1, chem_mode=1, chem_flags=0, y_he=0.0, f_s=f_s, f_max=2 * f_s,
                      max_substeps=100000, sigma=[[sigma, 0, 0], [0, 0, 0], [0, 0, 0]],
                      eps=[[0, 0, 0], [0, 0, 0], [0, 0, 0]])
    x5 = np.zeros((5, C))
    x5[0], x5[1], x5[2] = x0, 1 - x0, 1.0
    st = dict(N=np.full((1, C), N0), fr=np.zeros((1, 3, C)), nH=np.full(C, 1e-8), x5=x5, T=np.full(C, 1e4),
              cells=np.zeros(0, np.int64), Q=np.zeros((0, 1)))
    o = make_oracle(mesh, cfg, st)
    assert o.thermochemistry(Gt / (cfg["c_red"] * sigma * N0)) == 0
    x, _ = o.gas()
    assert np.all(x[0] == x[0, 0])
    exact = x0 * np.exp(-Gt)
    return (x[0, 0] - exact) / exact, int(o.substeps()[0])


def test_adaptive_substeps_converge_first_order():
    """The semi-implicit update under the 10 % substep rule (Sec. 4.1.1)
    against the exact exponential decay of photoionisation: backward Euler
    over-predicts what remains (1 / (1 + a) > exp(-a)), and with the rule's
    target f_s halved the error halves while the substeps double -- first
    order, as a controller that really sets the step from the relative
    change gives.  The Richardson extrapolation of the two finest runs then
    agrees with exp(-Gamma t) to 1e-4, which also pins Gamma = c sigma N."""
    runs = [_photoionisation_decay(f) for f in (0.05, 0.025, 0.0125)]
    errs = [e for e, _ in runs]
    subs = [n for _, n in runs]
    assert all(e > 0 for e in errs)
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2, errs
    for a, b in zip(subs, subs[1:]):
        assert 1.7 < b / a < 2.3, subs
    assert errs[0] < 0.1                               # ~ Gamma t f_s
    assert abs(2 * errs[2] - errs[1]) < 1e-4, errs


def test_photoheating_energy_budget():
    """Thermal energy (Sec. 2.3.1, reading 10 v) against the ionisation
    count: hydrogen only, one bin, photoheating on and recombination,
    collisional ionisation and cooling off.  Every photoionisation then
    deposits exactly eps of heat, so per cell the thermal energy
    3/2 k n_tot T grows by eps n_H (x_HII' - x_HII) -- the energy equation
    and the abundance update are separate parts of the step, so a dropped
    or misplaced heat term, a wrong n_tot or a wrong eps index fails here.
    Over several adaptive substeps the identity telescopes."""
    kB = 1.380649e-16
    eps = 4.2e-12          # erg per photoionisation (grey; any positive value)
    sigma = 3.0e-18        # cm^2
    mesh, cfg, st = voronoi_case(n=8, n_bins=1, chem_mode=2, chem_flags=8, y_he=0.0,
                                 sigma=[[sigma, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]],
                                 eps=[[eps, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    st["cells"] = np.zeros(0, np.int64)
    st["Q"] = np.zeros((0, 1))
    st["N"] *= 1e2
    C = mesh.n_cells
    x5 = np.zeros((5, C))
    x5[1] = np.random.default_rng(3).uniform(0.0, 0.5, C)
    x5[0] = 1.0 - x5[1]
    x5[2] = 1.0
    st["x5"] = x5
    o = make_oracle(mesh, cfg, st)
    nH = st["nH"]
    x0, T0 = o.gas()
    dt = 4 * o.max_dt()
    assert o.thermochemistry(dt) == 0
    x1, T1 = o.gas()
    assert o.substeps().max() > 1                   # several accepted substeps
    e0 = 1.5 * kB * nH * (1.0 + x0[1]) * T0
    e1 = 1.5 * kB * nH * (1.0 + x1[1]) * T1
    heat = eps * nH * (x1[1] - x0[1])
    assert heat.min() > 0 and np.all(x1[1] > x0[1])
    np.testing.assert_allclose(e1 - e0, heat, rtol=1e-9, atol=1e-12 * np.abs(e0).max())


def test_photon_conservation_with_absorption_no_recombination():
    """Absorption on, recombination and collisional ionisation off, no
    sources: every absorbed photon becomes one free electron, so
    sum_i V_i (sum_b N_b + n_e) is constant to round-off over whole steps."""
    mesh, cfg, st = voronoi_case(n=10, chem_mode=1, chem_flags=0)
    st["cells"] = np.zeros(0, np.int64)
    st["N"] *= 1e3  # photon-rich: strong ionisation
    st["fr"] *= 1e3
    o = make_oracle(mesh, cfg, st)
    V = mesh.volume
    nH, yhe = st["nH"], cfg["y_he"]

    def total():
        N, _ = o.radiation()
        x5, _ = o.gas()
        ne = nH * (x5[1] + yhe * (x5[3] + 2 * x5[4]))
        return ((N.sum(0) + ne) * V).sum()

    t0 = total()
    dt = o.max_dt()
    assert o.step(4 * dt, 4) == 0
    t1 = total()
    assert abs(t1 / t0 - 1) < 1e-12
    x5, _ = o.gas()
    assert (x5 >= 0).all()
    np.testing.assert_allclose(x5[0] + x5[1], 1, atol=1e-14)
    np.testing.assert_allclose(x5[2] + x5[3] + x5[4], 1, atol=1e-14)


@pytest.mark.parametrize("splitting,time_order", [(0, 1), (1, 1), (0, 2), (1, 2)])
def test_photon_budget_with_sources(splitting, time_order):
    """Sources on, absorption on, recombination and collisional ionisation
    off: every photon injected (Q dt per source, Eq. E) is either still in
    flight or has made one free electron, so sum_i V_i (sum_b N_b + n_e)
    grows by exactly sum_k Q_k t, for the Lie and Strang splits and for both
    transport integrators.  A half step applied twice, or a stage weight
    off in Heun's combination, breaks the budget."""
    mesh, cfg, st = voronoi_case(n=10, chem_mode=1, chem_flags=0, splitting=splitting, time_order=time_order)
    o = make_oracle(mesh, cfg, st)
    V = mesh.volume * cfg["unit_length_cm"] ** 3
    nH, yhe = st["nH"], cfg["y_he"]

    def total():
        N, _ = o.radiation()
        x5, _ = o.gas()
        ne = nH * (x5[1] + yhe * (x5[3] + 2 * x5[4]))
        return ((N.sum(0) + ne) * V).sum()

    t0 = total()
    dt = o.max_dt()
    assert o.step(4 * dt, 4) == 0
    t1 = total()
    injected = st["Q"].sum() * 4 * dt
    assert injected > 1e-3 * t0
    assert abs((t1 - t0) / injected - 1) < 1e-10


def test_heun_conserves_photons_and_flux():
    """Heun's two-stage transport keeps the antisymmetric gather's exact
    conservation of sum N V and sum F V (its result is a convex combination
    of conservative stages)."""
    mesh, cfg, st = voronoi_case(n=12, chem_mode=0, time_order=2, n_src=0)
    o = make_oracle(mesh, cfg, st)
    V = mesh.volume
    N0, fr0 = o.radiation()
    dt = o.max_dt()
    assert o.step(5 * dt, 5) == 0
    N1, fr1 = o.radiation()
    np.testing.assert_allclose((N1 * V).sum(1), (N0 * V).sum(1), rtol=1e-13)
    assert np.abs((fr1 * V).sum(2) - (fr0 * V).sum(2)).max() <= 1e-13 * np.abs(fr0 * V).sum()
    assert np.abs(N1 - N0).max() > 1e-3 * N0.max()


def _smooth_wave_error_ratio(time_order, n0=4):
    """Temporal convergence on a fixed mesh (limiter off, smooth field):
    states at t = n0 dt_max from n0, 2 n0 and 4 n0 subcycles; the spatial
    error is common to all three, so |U(n0) - U(2n0)| / |U(2n0) - U(4n0)|
    tends to 2^p for a method of order p in time."""
    mesh = synth.voronoi_mesh(10, 1.0, 0.2, seed=5)
    C = mesh.n_cells
    ph = 2 * np.pi * mesh.centroids()[:, 0]
    N = 1.0 + 0.01 * np.sin(ph)
    fr = np.zeros((1, 3, C))
    fr[0, 0] = 0.5 * N
    cfg = base_config(box=1.0, n_bins=1, c_red=1.0, unit_length_cm=1.0, chem_mode=0, limiter=0,
                      time_order=time_order)
    gas = dict(zip(("nH", "x5", "T"), neutral_gas(C, 1e-3)))
    out = []
    for k in (1, 2, 4):
        o = make_oracle(mesh, cfg, dict(N=N[None], fr=fr, **gas))
        t_end = n0 * o.max_dt()
        assert o.step(t_end, n0 * k) == 0
        out.append(o.radiation()[0][0])
    return np.abs(out[0] - out[1]).max() / np.abs(out[1] - out[2]).max()


def test_heun_is_second_order_in_time():
    """Forward Euler halves its temporal error with the step (ratio 2);
    Heun's method quarters it (ratio 4)."""
    r1 = _smooth_wave_error_ratio(1)
    r2 = _smooth_wave_error_ratio(2)
    assert 1.7 < r1 < 2.4, r1
    assert 3.4 < r2 < 4.6, r2


def _mask_and_touched(mesh, frac, seed):
    rng = np.random.default_rng(seed)
    act = rng.uniform(size=mesh.n_cells) < frac
    touched = act.copy()
    fa = act[mesh.left] | act[mesh.right]
    touched[mesh.left[fa]] = True
    touched[mesh.right[fa]] = True
    return act, touched


def test_individual_timesteps_locality_and_conservation():
    """Individual time steps (Sec. 2.1): with 30% of the cells active, the
    interfaces with an active cell carry flux and no other does (Sec. 4.1.3),
    so sum N V is still conserved to round-off, a cell without an active
    interface keeps its radiation bitwise, and passive cells keep their gas
    (no thermochemistry) while active cells evolve.  With every cell active
    the result is bitwise that of the unmasked step."""
    mesh, cfg, st = voronoi_case(n=10, chem_mode=1, n_src=0)
    act, touched = _mask_and_touched(mesh, 0.3, 4)
    V = mesh.volume
    o = make_oracle(mesh, cfg, st)
    o.set_active(act)
    dt = o.max_dt()
    N0, fr0 = o.radiation()
    assert o.step(3 * dt, 3) == 0
    N1, fr1 = o.radiation()
    x5, T = o.gas()
    # absorption moves photons into electrons: check transport conservation
    # with absorption off
    o2 = make_oracle(mesh, dict(cfg, chem_mode=0), st)
    o2.set_active(act)
    assert o2.step(3 * dt, 3) == 0
    N2, fr2 = o2.radiation()
    np.testing.assert_allclose((N2 * V).sum(1), (N0 * V).sum(1), rtol=1e-13)
    # no active interface within three subcycles: radiation untouched
    far = ~touched
    # cells are touched only through active interfaces, and the active set
    # is fixed, so untouched cells never change
    np.testing.assert_array_equal(N2[:, far], N0[:, far])
    np.testing.assert_array_equal(fr2[:, :, far], fr0[:, :, far])
    assert np.abs(N2[:, touched] - N0[:, touched]).max() > 0
    # passive cells: gas unchanged; active cells: gas evolved
    np.testing.assert_array_equal(x5[:, ~act], st["x5"][:, ~act])
    np.testing.assert_array_equal(T[~act], st["T"][~act])
    assert np.abs(x5[:, act] - st["x5"][:, act]).max() > 0
    # all active = unmasked, bitwise
    oa, ob = make_oracle(mesh, cfg, st), make_oracle(mesh, cfg, st)
    oa.set_active(np.ones(mesh.n_cells, bool))
    assert oa.step(2 * dt, 2) == 0 and ob.step(2 * dt, 2) == 0
    np.testing.assert_array_equal(oa.radiation()[0], ob.radiation()[0])
    np.testing.assert_array_equal(oa.gas()[0], ob.gas()[0])


def test_individual_timesteps_photon_budget():
    """Sources, absorption, no recombination, 40% of the cells active: the
    budget sum V (sum N + n_e) grows by exactly sum over the active source
    cells of Q t (a source in a passive cell emits nothing this step)."""
    mesh, cfg, st = voronoi_case(n=10, chem_mode=1, chem_flags=0, n_src=6)
    act, _ = _mask_and_touched(mesh, 0.4, 7)
    assert act[st["cells"]].any() and not act[st["cells"]].all()
    o = make_oracle(mesh, cfg, st)
    o.set_active(act)
    Vc = mesh.volume * cfg["unit_length_cm"] ** 3
    nH, yhe = st["nH"], cfg["y_he"]

    def total():
        N, _ = o.radiation()
        x5, _ = o.gas()
        return ((N.sum(0) + nH * (x5[1] + yhe * (x5[3] + 2 * x5[4]))) * Vc).sum()

    t0 = total()
    dt = o.max_dt()
    assert o.step(4 * dt, 4) == 0
    inj = st["Q"][act[st["cells"]]].sum() * 4 * dt
    assert abs((total() - t0) / inj - 1) < 1e-10


# ---------------------------------------------------------------------------
# wave and beam: transport speed c_red (Sec. 4.2.1)
# ---------------------------------------------------------------------------

def _wave_run(n, order=2, periods=1):
    """Travelling wave of Sec. 4.2.1: L = 1, c = 1, N = 1 + 1e-6 sin(2 pi (x+y+z)),
    F = c N (1,1,1)/sqrt(3), zero opacity, irregular mesh (10% jitter).
    Returns (amplitude, phase) of the perturbation after ``periods`` periods,
    projected on sin / cos of the initial phase and normalised by the same
    projection of the initial field, and the relative change of sum N V."""
    mesh = synth.voronoi_mesh(n, 1.0, 0.1, seed=21)
    C = mesh.n_cells
    c = mesh.centroids()
    ph = 2 * np.pi * c.sum(1)
    N = 1.0 + 1e-6 * np.sin(ph)
    fr = np.outer(np.ones(3) / np.sqrt(3), N)[None]
    cfg = base_config(box=1.0, n_bins=1, c_red=1.0, unit_length_cm=1.0, chem_mode=0, order=order)
    o = make_oracle(mesh, cfg, dict(N=N[None], fr=fr, **dict(zip(("nH", "x5", "T"), neutral_gas(C, 1e-3)))))
    t_end = periods / np.sqrt(3)  # one period: the pattern moves 1/sqrt(3) along (1,1,1)/sqrt(3)
    n_sub = int(np.ceil(t_end / o.max_dt()))
    assert o.step(t_end, n_sub) == 0
    N1, _ = o.radiation()
    V = mesh.volume

    def proj(field):
        d = (field - 1.0) / 1e-6
        return 2 * (V * d * np.sin(ph)).sum(), 2 * (V * d * np.cos(ph)).sum()

    s0, c0 = proj(N)
    s1, c1 = proj(N1[0])
    z = complex(s1, c1) / complex(s0, c0)
    return abs(z), np.angle(z), (V * N1[0]).sum() / (V * N).sum() - 1


@pytest.mark.slow
def test_travelling_wave_speed_and_conservation():
    """After one period (t = 1/sqrt(3)) the wave is back in phase: the phase
    error is small and falls quickly with resolution, sum N V is exact, and
    the amplitude stays bounded.  The first-order scheme is purely
    dissipative (amplitude < 1).  Forward Euler with linear reconstruction and
    no time extrapolation (Sec. 2.3.3) slightly amplifies long smooth waves;
    the slope limiter bounds that growth."""
    a16, p16, m16 = _wave_run(16)
    a32, p32, m32 = _wave_run(32)
    assert abs(m16) < 1e-13 and abs(m32) < 1e-13
    assert abs(p32) < 0.02 and abs(p32) < abs(p16) / 3
    assert 0.5 < a32 < 1.3
    a1, p1, m1 = _wave_run(16, order=1)
    assert abs(m1) < 1e-13
    assert 0.05 < a1 < a16 and a1 < 1.0
    assert abs(p1) < 0.2


def test_beam_front_moves_at_c_red():
    """A free-streaming slab (F = c N e_x, N = 1 for x < L/4) translates at
    c_red: its half-maximum fronts sit at x = L/4 + c t and x = c t."""
    n, L = 64, 1.0
    mesh = synth.cartesian_mesh(n, L)
    C = mesh.n_cells
    x = mesh.cx
    N = np.where(x < 0.25 * L, 1.0, 0.0)
    fr = np.zeros((1, 3, C))
    fr[0, 0] = N
    cfg = base_config(box=L, n_bins=1, c_red=1.0, unit_length_cm=1.0, chem_mode=0)
    o = make_oracle(mesh, cfg, dict(N=N[None], fr=fr, **dict(zip(("nH", "x5", "T"), neutral_gas(C, 1e-3)))))
    t = 0.3
    n_sub = int(np.ceil(t / o.max_dt()))
    assert o.step(t, n_sub) == 0
    N1, _ = o.radiation()
    prof = N1[0].reshape(n, n, n).mean(axis=(0, 1))
    xc = (np.arange(n) + 0.5) / n
    # leading front: last crossing of 0.5 going down
    i = np.where((prof[:-1] >= 0.5) & (prof[1:] < 0.5))[0][-1]
    xf = xc[i] + (prof[i] - 0.5) / (prof[i] - prof[i + 1]) / n
    assert abs(xf - (0.25 + t)) < 1.5 / n
    j = np.where((prof[:-1] < 0.5) & (prof[1:] >= 0.5))[0][0]
    xb = xc[j] + (0.5 - prof[j]) / (prof[j + 1] - prof[j]) / n
    assert abs(xb - t) < 1.5 / n
    assert abs(prof.mean() - 0.25) < 1e-13


# ---------------------------------------------------------------------------
# chemistry: equilibrium, Stroemgren (Sec. 2.3.1)
# ---------------------------------------------------------------------------

def _uniform_box(n, L, nH, T, n_bins, y_he, rate_per_cell, chem_mode=1, c_red=0.01):
    mesh = synth.cartesian_mesh(n, L)
    C = mesh.n_cells
    cfg = base_config(box=L, n_bins=n_bins, y_he=y_he, chem_mode=chem_mode, c_red=c_red * synth.C_LIGHT)
    nH_, x5, T_ = neutral_gas(C, nH, T)
    cells = np.arange(C, dtype=np.int64)
    Q = np.tile(np.asarray(rate_per_cell, dtype=np.float64)[None, :], (C, 1))
    st = dict(N=np.zeros((n_bins, C)), fr=np.zeros((n_bins, 3, C)), nH=nH_, x5=x5, T=T_, cells=cells, Q=Q)
    return mesh, cfg, st


def test_hydrogen_photoionisation_equilibrium_closed_form():
    """Every cell of a uniform box gets photons at rate S; in steady state
    injection = photoionisations = case-B recombinations, so
    x_HII = sqrt(S / (V alpha_B n_H^2)) exactly, and the radiation level
    satisfies c sigma n_HI N = S / V up to the implicit-step factor."""
    from oracle import rate_probe
    n, L, nH, T = 4, 1.0, 1.0, 1e4
    Vcm3 = (L / n * synth.KPC_CM) ** 3
    alpha = rate_probe("alphaB_HII", T)
    S = 0.25 * alpha * nH ** 2 * Vcm3  # gives x_HII = 0.5
    mesh, cfg, st = _uniform_box(n, L, nH, T, 1, 0.0, [S])
    cfg["chem_flags"] = 1  # recombination only: no collisional ionisation
    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt()
    assert o.step(400 * dt, 400) == 0
    x5, _ = o.gas()
    np.testing.assert_allclose(x5[1], np.sqrt(S / (Vcm3 * alpha * nH ** 2)), rtol=1e-9)
    np.testing.assert_allclose(x5[0] + x5[1], 1.0, atol=1e-15)


def test_hydrogen_helium_equilibrium_brute_force():
    """H+He, three bins, uniform photon injection.  At the fixed point the
    three ionisation balances Gamma_HI x_HI = alpha_HII n_e x_HII,
    Gamma_HeI y_I = alpha_HeII n_e y_II, Gamma_HeII y_II = alpha_HeIII n_e y_III
    hold with Gamma_s = c sum_b sigma_bs Nbar_b (the radiation level of the
    step); solved by brute-force root finding and compared."""
    from scipy.optimize import brentq
    from oracle import rate_probe
    from tests._cases import SIGMA3
    n, L, nH, T = 4, 1.0, 1.0, 2e4
    yhe = synth.helium_ratio(0.24)
    Vcm3 = (L / n * synth.KPC_CM) ** 3
    aH = rate_probe("alphaB_HII", T)
    S = np.array([0.3, 0.05, 0.02]) * aH * nH ** 2 * Vcm3
    mesh, cfg, st = _uniform_box(n, L, nH, T, 3, yhe, S)
    cfg["chem_flags"] = 1  # recombination only (rates at fixed T)
    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt()
    assert o.step(600 * dt, 600) == 0
    x5, _ = o.gas()
    Nend, _ = o.radiation()
    assert np.ptp(x5, axis=1).max() < 1e-12  # uniform
    x = x5[:, 0]
    # radiation level of the (single, accepted) chemistry substep at the fixed point
    c = cfg["c_red"]
    sig = np.array(SIGMA3)
    ns = np.array([nH * x[0], yhe * nH * x[2], yhe * nH * x[3]])
    kap = sig @ ns
    Nstart = Nend[:, 0] + S * dt / Vcm3
    Nbar = Nstart / (1 + c * dt * kap)
    G = c * (sig * Nbar[:, None]).sum(0)
    a2, a3 = rate_probe("alphaB_HeII", T), rate_probe("alphaB_HeIII", T)

    def he_state(ne):
        # HeI <-> HeII <-> HeIII balance at given n_e
        r1 = G[1] / (a2 * ne)   # y_II / y_I
        r2 = G[2] / (a3 * ne)   # y_III / y_II
        yI = 1.0 / (1 + r1 + r1 * r2)
        return yI, yI * r1, yI * r1 * r2

    def resid(ne):
        xh = G[0] / (G[0] + aH * ne)
        _, yII, yIII = he_state(ne)
        return nH * xh + yhe * nH * (yII + 2 * yIII) - ne

    ne = brentq(resid, 1e-12, 3 * nH)
    xh = G[0] / (G[0] + aH * ne)
    yI, yII, yIII = he_state(ne)
    np.testing.assert_allclose([x[1], x[2], x[3], x[4]], [xh, yI, yII, yIII], rtol=2e-6)


@pytest.mark.slow
def test_stroemgren_radius():
    """H only, one bin, isothermal 1e4 K, n_H = 0.1, Q = 5e48 /s in a periodic
    0.75 kpc box at 24^3: after many recombination times the ionised volume
    matches R_s = (3 Q / (4 pi n_H^2 alpha_B))^(1/3) = 0.25 kpc, and total
    recombinations balance Q."""
    from oracle import rate_probe
    n, L, nH, Q = 24, 0.75, 0.1, 5e48
    mesh = synth.cartesian_mesh(n, L)
    C = mesh.n_cells
    cfg = base_config(box=L, n_bins=1, y_he=0.0, chem_mode=1, c_red=0.001 * synth.C_LIGHT,
                      sigma=[[6.3e-18, 0, 0]])
    nH_, x5, T = neutral_gas(C, nH, 1e4)
    cells = corner_cells(n, n // 2)
    st = dict(N=np.zeros((1, C)), fr=np.zeros((1, 3, C)), nH=nH_, x5=x5, T=T, cells=cells,
              Q=np.full((8, 1), Q / 8))
    o = make_oracle(mesh, cfg, st)
    alpha = rate_probe("alphaB_HII", 1e4)
    t_rec = 1 / (nH * alpha)
    dt = o.max_dt()
    n_sub = int(np.ceil(5 * t_rec / dt))
    assert o.step(n_sub * dt, n_sub) == 0
    x5, _ = o.gas()
    Vcm3 = mesh.volume * synth.KPC_CM ** 3
    R = (3 * (x5[1] * Vcm3).sum() / (4 * np.pi)) ** (1 / 3) / synth.KPC_CM
    Rs = (3 * Q / (4 * np.pi * nH ** 2 * alpha)) ** (1 / 3) / synth.KPC_CM
    assert Rs == pytest.approx(golden("textbook_rates.json")["stroemgren_test"]["R_s_kpc"], rel=2e-2)
    assert abs(R / Rs - 1) < 0.05
    rec = (alpha * nH ** 2 * x5[1] ** 2 * Vcm3).sum()
    assert abs(rec / Q - 1) < 0.05


# ---------------------------------------------------------------------------
# symmetry and the first workload (32^3 Cartesian, central source)
# ---------------------------------------------------------------------------

def test_config1_mirror_and_permutation_symmetry():
    """The central source of the 32^3 workload sits on a grid corner split
    over 8 cells: the solution is symmetric under reflection of each axis
    about that corner and under permutation of the axes."""
    mesh, cfg, st = config1(16)
    cfg["box"] = 5.0
    mesh = synth.cartesian_mesh(16, 5.0)
    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt()
    assert o.step(6 * dt, 6) == 0
    N, fr = o.radiation()
    x5, T = o.gas()
    n = 16
    for f in (N[0], N[2], x5[1], T):
        a = f.reshape(n, n, n)
        sc = np.abs(a).max()
        # reflection about the corner between index 7 and 8: i -> 15 - i
        for ax in range(3):
            np.testing.assert_allclose(np.flip(a, ax), a, rtol=0, atol=1e-12 * sc)
        np.testing.assert_allclose(np.transpose(a, (1, 0, 2)), a, rtol=0, atol=1e-12 * sc)
        np.testing.assert_allclose(np.transpose(a, (0, 2, 1)), a, rtol=0, atol=1e-12 * sc)
    # flux components are odd under the matching reflection
    fx = fr[0, 0].reshape(n, n, n)
    np.testing.assert_allclose(np.flip(fx, 2), -fx, rtol=0, atol=1e-12 * np.abs(fx).max())


def test_hii_region_symmetry_on_staggered_grid():
    """Expanding HII region on the staggered 2 x n^3 grid (truncated
    octahedra): source sphere and density profile are centred on a
    generator, so photon density, abundances and temperature are even and
    each flux component odd under reflection of its axis, and the fields are
    invariant under exchange of two axes, to round-off."""
    n = 12
    mesh, cfg, st = synth.hii_region(n)
    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt()
    assert o.step(6 * dt, 6) == 0
    N, fr = o.radiation()
    x5, T = o.gas()
    L = cfg["box"]
    q = np.round((mesh.centroids() - 0.5 * L) / (L / n / 2)).astype(np.int64) % (2 * n)
    index = {tuple(v): i for i, v in enumerate(q)}

    def image(fn):
        return np.array([index[tuple(fn(v) % (2 * n))] for v in q])

    mirror_x = image(lambda v: np.array([-v[0], v[1], v[2]]))
    swap_xy = image(lambda v: np.array([v[1], v[0], v[2]]))
    assert N[0].max() > 0 and x5[1].max() > 1e-3
    for f in (N[0], N[1], x5[1], x5[3], T):
        sc = np.abs(f).max()
        np.testing.assert_allclose(f[mirror_x], f, rtol=0, atol=1e-12 * sc)
        np.testing.assert_allclose(f[swap_xy], f, rtol=0, atol=1e-12 * sc)
    fx, fy = fr[0, 0], fr[0, 1]
    sc = np.abs(fx).max()
    np.testing.assert_allclose(fx[mirror_x], -fx, rtol=0, atol=1e-12 * sc)
    np.testing.assert_allclose(fy[mirror_x], fy, rtol=0, atol=1e-12 * sc)
    np.testing.assert_allclose(fx[swap_xy], fy, rtol=0, atol=1e-12 * sc)


@pytest.mark.slow
def test_config1_early_ionisation_front():
    """H-only, isothermal version of the 32^3 workload: after 100 subcycles
    at the CFL limit (3.06 Myr << t_rec = 122 Myr) the ionised volume plus
    the photons still in flight (c_red is finite: about a sixth of the
    emitted photons) matches the early-time front
    r_I = R_s (1 - exp(-t/t_rec))^(1/3) = 1.57 kpc."""
    from oracle import rate_probe
    mesh, cfg, st = config1(32)
    cfg.update(n_bins=1, y_he=0.0, chem_mode=1, sigma=[[6.3e-18, 0, 0]])
    st["N"], st["fr"] = st["N"][:1], st["fr"][:1]
    st["Q"] = np.full((8, 1), 5e48 / 8)
    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt()
    assert o.step(100 * dt, 100) == 0
    x5, _ = o.gas()
    N, _ = o.radiation()
    Vcm3 = mesh.volume * synth.KPC_CM ** 3
    nH = 1e-3
    R = (3 * ((x5[1] + N[0] / nH) * Vcm3).sum() / (4 * np.pi)) ** (1 / 3) / synth.KPC_CM
    alpha = rate_probe("alphaB_HII", 1e4)
    Rs = (3 * 5e48 / (4 * np.pi * nH ** 2 * alpha)) ** (1 / 3) / synth.KPC_CM
    t = 100 * dt
    rI = Rs * (1 - np.exp(-t * nH * alpha)) ** (1 / 3)
    g = golden("textbook_rates.json")["config1_front"]
    assert Rs == pytest.approx(g["R_s_kpc"], rel=1e-2)
    assert rI == pytest.approx(g["r_I_kpc"], rel=2e-2)
    assert abs(R / rI - 1) < 0.02


def test_cfl_guard():
    """A subcycle above eta * min V^(1/3) / c_red (Eq. timestep) is refused."""
    mesh, cfg, st = config1(8)
    mesh = synth.cartesian_mesh(8, 10.0)
    o = make_oracle(mesh, cfg, st)
    dt = o.max_dt()
    assert dt == pytest.approx(0.3 * 1.25 * synth.KPC_CM / cfg["c_red"], rel=1e-14)
    assert o.step(2.01 * dt, 2) == 3
