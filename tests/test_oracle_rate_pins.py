"""Pins of the oracle's rate fits (Sec. 2.3.1 thermochemistry; the paper
defers the rates to the solver it builds on, so the oracle takes Hui & Gnedin
(1997) recombination and Katz, Weinberg & Hernquist (1996) collisional and
cooling fits) to data that do not come from those fits:

* every Boltzmann factor's activation temperature is the energy of the
  process it models (NIST ionisation energies; the 1s-2p energies of H I and
  He II for collisional excitation and dielectronic recombination), read off
  the oracle as the Arrhenius slope -d ln K / d(1/T) extrapolated to low T;
* collisional-ionisation cooling per ionisation is the ionisation energy,
  and dielectronic-recombination cooling per recombination the He II 1s-2p
  energy;
* case-B recombination of hydrogen at 5000, 10^4 and 2x10^4 K and of He I at
  10^4 K (Osterbrock & Ferland 2006);
* the collisional-ionisation rates against an independent fit of the
  electron-impact data (Voronov 1997), with the high-temperature factor
  1 / (1 + (T / 1e5)^(1/2)) that KWH96 apply to the published rates divided
  out, over the temperatures where the two fits agree;
* the free-free coefficient over the classical bremsstrahlung emissivity
  computed from CODATA constants is the frequency-averaged Gaunt factor,
  which lies between 1.1 and 1.5 (Rybicki & Lightman Sec. 5.2);
* radiative-recombination cooling of HII, and by hydrogenic scaling of
  HeIII, against the case-A coefficient (Osterbrock & Ferland 2006) times
  the mean captured energy that the Maxwellian identity d ln alpha / d ln T
  = <E>/kT - 3/2 gives, loosely (the fits sit 14-22 % from those data).

Each check is a function of the oracle's values; the planted-error tests
scale each pinned coefficient (or activation temperature) of the oracle's
output by 5 % (by a factor 2, a dropped factor or a dropped T^(1/2) for the
loose recombination-cooling window), on the CPU, and require the check to
fail.  Not pinned here: the prefactors of collisional excitation, the He II
radiative-recombination cooling, and the temperature shape of the KWH96
high-temperature factor.
"""
import json
import os

import numpy as np
import pytest

import oracle

A = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "atomic_data.json")))
KEV = A["k_B_eV_per_K"]["value"]
ERG = A["eV_erg"]["value"]
ION = A["ionisation_energies_eV"]
LINE = A["resonance_line_energies_eV"]


def theta(eV):
    return eV / KEV


def rate(name):
    return lambda T: oracle.rates(T)[name]


def cool(name):
    return lambda T: oracle.cooling_coeffs(T)[name]


# ---------------------------------------------------------------------------
# the checks: each returns the largest relative deviation from the datum
# ---------------------------------------------------------------------------

def arrhenius_theta(f, theta0):
    """-d ln f / d(1/T) at T = theta0/150 and theta0/300, extrapolated to
    1/T -> infinity: a factor T^p shifts the slope by p T, which the
    two-point extrapolation removes."""
    def slope(T):
        a, b = T * (1 - 1e-4), T * (1 + 1e-4)
        return -(np.log(f(b)) - np.log(f(a))) / (1 / b - 1 / a)
    s1, s2 = slope(theta0 / 150), slope(theta0 / 300)
    return 2 * s2 - s1


def dev_activation(f, eV):
    th = theta(eV)
    return abs(arrhenius_theta(f, th) / th - 1)


def dev_energy_per_event(cooling, rate_fn, eV, Ts):
    return max(abs(cooling(T) / rate_fn(T) / (eV * ERG) - 1) for T in Ts)


def dev_alphaB_HII(f):
    g = A["alphaB_HII"]
    return max(abs(f(T) / v - 1) for T, v in zip(g["T_K"], g["value"]))


def dev_alphaB_HeI(f):
    return abs(f(1e4) / A["alphaB_HeI_1e4K"]["value"] - 1)


def voronov(species, T):
    c = A["voronov1997"][species]
    U = c["dE"] / (KEV * T)
    return c["A"] * (1 + c["P"] * np.sqrt(U)) * U ** c["K"] * np.exp(-U) / (c["X"] + U)


def dev_voronov(f, species, lo, hi):
    return max(abs(f(T) * (1 + np.sqrt(T / 1e5)) / voronov(species, T) - 1) for T in np.geomspace(lo, hi, 9))


def c_ff():
    """Classical thermal bremsstrahlung emissivity per sqrt(T) n_e n_i Z^2 and
    unit Gaunt factor, 2^5 pi e^6 / (3 h m c^3) (2 pi k / (3 m))^(1/2)."""
    c = A["cgs_constants"]
    e, h, m, cl, k = c["e_esu"], c["h_erg_s"], c["m_e_g"], c["c_cm_s"], c["k_erg_K"]
    return 2 ** 5 * np.pi * e ** 6 / (3 * h * m * cl ** 3) * np.sqrt(2 * np.pi * k / (3 * m))


def gaunt_range(f):
    g = [f(T) / (c_ff() * np.sqrt(T)) for T in np.geomspace(1e4, 1e7, 13)]
    return min(g), max(g)


def betaA_HII():
    """Case-A radiative-recombination cooling coefficient of hydrogen (erg
    cm^3 s^-1) at the table's temperatures, from the tabulated alpha_A and
    an exact property of Maxwellian averages: for any capture cross-section
    sigma(E), alpha(T) = <v sigma> is proportional to T^(-3/2) times the
    integral of E sigma(E) exp(-E/kT) dE, so d ln alpha / d ln T = -3/2 +
    <E>/kT, where <E> is the mean kinetic energy of the captured electrons,
    which recombination cooling removes.  Hence beta = alpha kT (3/2 + d ln
    alpha / d ln T), the slope taken from a quadratic in ln T through the
    three tabulated points."""
    g = A["alphaA_HII"]
    T, a = np.array(g["T_K"]), np.array(g["value"])
    c = np.polyfit(np.log(T), np.log(a), 2)
    slope = np.polyval(np.polyder(c), np.log(T))
    return T, a * A["cgs_constants"]["k_erg_K"] * T * (1.5 + slope)


def dev_recomb_cooling_HII(f):
    """max |f / beta_A - 1| at 5000, 1e4 and 2e4 K."""
    T, b = betaA_HII()
    return max(abs(f(t) / bt - 1) for t, bt in zip(T, b))


def dev_recomb_cooling_HeIII(f):
    """He III -> He II against the hydrogenic scaling of the same data: for
    a one-electron ion of charge Z, alpha(Z, T) = Z alpha(1, T / Z^2), the
    mean captured energy over kT is the same function of T / Z^2, so beta(Z,
    T) = Z^3 beta(1, T / Z^2); here Z = 2, at 2e4, 4e4 and 8e4 K."""
    T, b = betaA_HII()
    return max(abs(f(4 * t) / (8 * bt) - 1) for t, bt in zip(T, b))


# (name, check(f) -> deviation, the oracle's function, tolerance)
ACTIVATION = [
    ("beta_HI", ION["HI"], rate("beta_HI")), ("beta_HeI", ION["HeI"], rate("beta_HeI")),
    ("beta_HeII", ION["HeII"], rate("beta_HeII")), ("ci_HI", ION["HI"], cool("ci_HI")),
    ("ci_HeI", ION["HeI"], cool("ci_HeI")), ("ci_HeII", ION["HeII"], cool("ci_HeII")),
    ("ce_HI", LINE["HI_Lyman_alpha"], cool("ce_HI")), ("ce_HeII", LINE["HeII_Lyman_alpha"], cool("ce_HeII")),
]
ACT_TOL = 1e-3            # the fits' constants carry 4-6 digits
DIEL_TOL = 1.2e-2         # Aldrovandi & Pequignot's 4.7e5 K is He II 2p to 0.8 %
EPE_TOL = 5e-3            # energies quoted to 3 digits in the fits
VORONOV = [("beta_HI", "HI", 1.5e4, 1e5, 0.07), ("beta_HeI", "HeI", 3e4, 6e4, 0.06),
           ("beta_HeII", "HeII", 7e4, 1.2e5, 0.065)]
# The KWH96 recombination-cooling fits (after Black 1981) predate the
# accurate case-A data and sit 14-22 % (HII) and 16 % (HeIII) from them:
# a loose window, which catches a dropped factor, a wrong exponent or a
# factor 2, not a 5 % error
RC_TOL = 0.25


# ---------------------------------------------------------------------------
# the oracle passes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,eV,f", ACTIVATION, ids=[a[0] for a in ACTIVATION])
def test_activation_temperatures_are_the_process_energies(name, eV, f):
    assert dev_activation(f, eV) < ACT_TOL


def test_dielectronic_activation_is_heii_2p():
    assert dev_activation(cool("diel_HeII"), LINE["HeII_Lyman_alpha"]) < DIEL_TOL


@pytest.mark.parametrize("s", ["HI", "HeI", "HeII"])
def test_collisional_ionisation_cooling_is_the_ionisation_energy(s):
    Ts = np.geomspace(1e4, 1e6, 7)
    assert dev_energy_per_event(cool("ci_" + s), rate("beta_" + s), ION[s], Ts) < EPE_TOL


def test_dielectronic_cooling_per_recombination():
    """At 5e5-1e6 K the He II recombination rate is dielectronic to 0.5 %;
    each such recombination radiates the He II 1s-2p energy."""
    Ts = (5e5, 7e5, 1e6)
    assert dev_energy_per_event(cool("diel_HeII"), rate("alpha_HeII"), LINE["HeII_Lyman_alpha"], Ts) < DIEL_TOL


def test_caseB_recombination_tables():
    assert dev_alphaB_HII(rate("alpha_HII")) < 1e-2     # Hui & Gnedin state 0.7 % for this fit
    assert dev_alphaB_HeI(rate("alpha_HeII")) < 5e-2


@pytest.mark.parametrize("key,species,lo,hi,tol", VORONOV, ids=[v[0] for v in VORONOV])
def test_collisional_ionisation_against_voronov(key, species, lo, hi, tol):
    assert dev_voronov(rate(key), species, lo, hi) < tol


def test_recombination_cooling_against_case_A_data():
    """Radiative-recombination cooling of HII and HeIII within RC_TOL of the
    case-A coefficient times the mean captured energy (and its hydrogenic
    scaling); the derived mean energy, 0.78 kT at 1e4 K, lies below the
    Maxwellian 3/2 kT as the 1/v rise of the capture cross-section makes
    it."""
    T, b = betaA_HII()
    g = A["alphaA_HII"]["value"]
    mean_e = b[1] / (g[1] * A["cgs_constants"]["k_erg_K"] * T[1])
    assert 0.7 < mean_e < 0.85
    assert dev_recomb_cooling_HII(cool("rc_HII")) < RC_TOL
    assert dev_recomb_cooling_HeIII(cool("rc_HeIII")) < RC_TOL


def test_free_free_gaunt_factor_range():
    assert c_ff() == pytest.approx(1.4256e-27, rel=1e-3)
    lo, hi = gaunt_range(cool("ff"))
    gr = A["gaunt_ff_range"]["value"]
    assert gr[0] <= lo and hi <= gr[1]


# ---------------------------------------------------------------------------
# a 5 % error in any pinned coefficient fails its check
# ---------------------------------------------------------------------------

def _scaled(f, s):
    return lambda T: s * f(T)


def _shifted(f, eV, s):
    """The same fit with its activation temperature scaled by s."""
    th = theta(eV)
    return lambda T: f(T) * np.exp(-(s - 1) * th / T)


def test_planted_errors_fail_the_checks():
    for s in (1.05, 0.95):
        for name, eV, f in ACTIVATION:
            assert dev_activation(_shifted(f, eV, s), eV) > ACT_TOL, (name, s)
        d = cool("diel_HeII")
        assert dev_activation(_shifted(d, LINE["HeII_Lyman_alpha"], s), LINE["HeII_Lyman_alpha"]) > DIEL_TOL
        Ts = np.geomspace(1e4, 1e6, 7)
        for sp in ("HI", "HeI", "HeII"):
            assert dev_energy_per_event(_scaled(cool("ci_" + sp), s), rate("beta_" + sp), ION[sp], Ts) > EPE_TOL
            assert dev_energy_per_event(cool("ci_" + sp), _scaled(rate("beta_" + sp), s), ION[sp], Ts) > EPE_TOL
        assert dev_energy_per_event(_scaled(d, s), rate("alpha_HeII"), LINE["HeII_Lyman_alpha"],
                                    (5e5, 7e5, 1e6)) > DIEL_TOL
        assert dev_alphaB_HII(_scaled(rate("alpha_HII"), s)) > 1e-2
        for key, sp, lo, hi, tol in VORONOV:
            assert dev_voronov(_scaled(rate(key), s), sp, lo, hi) > tol, (key, s)
    # one-sided: He I case B at 5 % sits 4 % below the table, so only a
    # low-side error of the coefficient shows; the Gaunt range catches a
    # 5 % high error at its peak
    assert dev_alphaB_HeI(_scaled(rate("alpha_HeII"), 0.95)) > 5e-2
    lo, hi = gaunt_range(_scaled(cool("ff"), 1.05))
    assert hi > A["gaunt_ff_range"]["value"][1]


def test_planted_gross_errors_fail_the_recombination_cooling_checks():
    """The loose window still fails a factor 2 either way, a dropped
    (T / 1e3)^(-0.2) factor and a dropped T^(1/2)."""
    for key, dev in (("rc_HII", dev_recomb_cooling_HII), ("rc_HeIII", dev_recomb_cooling_HeIII)):
        f = cool(key)
        for s in (2.0, 0.5):
            assert dev(_scaled(f, s)) > RC_TOL, (key, s)
        assert dev(lambda T: f(T) * (T / 1e3) ** 0.2) > RC_TOL, key
        assert dev(lambda T: f(T) / np.sqrt(T)) > RC_TOL, key
