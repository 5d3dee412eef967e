"""Pins of the oracle's equation of state (Eq. 7), pseudo-potential (Eq. 6)
and interaction forces (Eqs. 8-9, adhesion) against textbook forms,
critical-point conditions, the Maxwell construction and continuum limits."""
import numpy as np
import pytest
from scipy import integrate, optimize

from oracle import oracle as O
from paper_1510_03560_gb300 import workloads as W

A, B, RGAS, OMEGA = 2.0 / 49.0, 2.0 / 21.0, 1.0, 0.344


def textbook_pr(v, T, Tc):
    """Peng & Robinson (1976) in molar volume v = 1/rho:
    p = RT/(v-b) - a alpha(T) / (v (v+b) + b (v-b))."""
    kappa = 0.37464 + 1.54226 * OMEGA - 0.26992 * OMEGA ** 2
    alpha = (1.0 + kappa * (1.0 - np.sqrt(T / Tc))) ** 2
    return RGAS * T / (v - B) - A * alpha / (v * (v + B) + B * (v - B))


def test_critical_point_conditions():
    """At T = Tc the isotherm has an inflection with zero slope: both
    dp/drho and d2p/drho2 vanish at one density (this fixes Tc and the
    reading of the garbled denominator of Eq. 7)."""
    p = lambda r: O.pressure(r, T_over_Tc=1.0)
    h = 1e-4
    dp = lambda r: (p(r + h) - p(r - h)) / (2 * h)
    d2p = lambda r: (p(r + h) - 2 * p(r) + p(r - h)) / h ** 2
    rc = optimize.brentq(d2p, 0.5, 5.0)
    Tc = O.eos_constants()["Tc"]
    assert abs(dp(rc)) < 2e-4 * RGAS * Tc  # 5-digit constants 0.45724 / 0.07780
    # below Tc the slope turns negative there, above Tc it stays positive
    assert O.pressure(rc + 0.3, T_over_Tc=0.9) < O.pressure(rc - 0.3, T_over_Tc=0.9)
    slope_above = [(O.pressure(r + h, T_over_Tc=1.1) - O.pressure(r - h, T_over_Tc=1.1)) / (2 * h)
                   for r in np.linspace(0.2, 8.0, 200)]
    assert min(slope_above) > 0


def test_eos_constants_textbook():
    c = O.eos_constants()
    assert c["Tc"] == pytest.approx(0.0778 * A / (0.45724 * B * RGAS), rel=1e-15)
    assert c["T"] == pytest.approx(0.85 * c["Tc"], rel=1e-15)
    assert c["kappa"] == pytest.approx(0.873236, abs=1e-6)
    assert c["theta"] == pytest.approx((1 + c["kappa"] * (1 - np.sqrt(0.85))) ** 2, rel=1e-14)


@pytest.mark.parametrize("rho", [0.05, 0.341309, 1.0, 3.3, 6.629339, 9.0])
def test_pressure_matches_molar_volume_form(rho):
    c = O.eos_constants()
    assert O.pressure(rho) == pytest.approx(textbook_pr(1.0 / rho, c["T"], c["Tc"]), rel=1e-13)


def maxwell(T, Tc):
    """Equal-area construction in v: p(v_l) = p(v_g) = p0 and
    int_{v_l}^{v_g} p dv = p0 (v_g - v_l)."""
    p = lambda v: textbook_pr(v, T, Tc)
    dp = lambda v: (p(v * (1 + 1e-7)) - p(v * (1 - 1e-7))) / (2e-7 * v)
    vs = np.linspace(0.11, 10.0, 20000)
    s = np.sign([dp(v) for v in vs])
    idx = np.where(np.diff(s) != 0)[0]
    v_min, v_max = vs[idx[0]], vs[idx[1]]  # spinodal volumes (liquid, vapour)

    def resid(p0):
        vl = optimize.brentq(lambda v: p(v) - p0, 0.1 + 1e-9, v_min)
        vg = optimize.brentq(lambda v: p(v) - p0, v_max, 1e3)
        return integrate.quad(p, vl, vg, epsabs=1e-14, epsrel=1e-13)[0] - p0 * (vg - vl), vl, vg

    lo, hi = max(p(v_min), 1e-3), p(v_max)
    p0 = optimize.brentq(lambda q: resid(q)[0], lo + 1e-12, hi - 1e-12, xtol=1e-15)
    _, vl, vg = resid(p0)
    return 1.0 / vg, 1.0 / vl, p0, 1.0 / v_max, 1.0 / v_min


def test_maxwell_coexistence_densities():
    """The liquid / vapour input densities are the Maxwell equal-area
    densities of Eq. 7 at T = 0.85 Tc (independent construction)."""
    c = O.eos_constants()
    rg, rl, p0, sp_g, sp_l = maxwell(c["T"], c["Tc"])
    assert rg == pytest.approx(W.RHO_VAP, abs=2e-6)
    assert rl == pytest.approx(W.RHO_LIQ, abs=2e-6)
    assert O.pressure(W.RHO_VAP) == pytest.approx(p0, rel=2e-5)
    assert O.pressure(W.RHO_LIQ) == pytest.approx(p0, rel=2e-5)
    assert 1.0 < sp_g < 1.2 and 5.0 < sp_l < 5.2


def test_psi_values_and_sign():
    """Eq. 6 with g = -1 and c_s^2 = 1/3 reads psi^2 = 2 rho - 6 p; with the
    textbook pressure it is real and increasing across both phases."""
    c = O.eos_constants()
    vals = []
    for rho in (W.RHO_VAP, 1.0, 2.0, 4.0, W.RHO_LIQ):
        p = textbook_pr(1.0 / rho, c["T"], c["Tc"])
        assert O.psi(rho) ** 2 == pytest.approx(2 * rho - 6 * p, rel=1e-12)
        vals.append(O.psi(rho))
    assert all(b > a > 0 for a, b in zip(vals, vals[1:]))
    assert O.psi(1.0, g_self=0.0) == 0.0


def _profile_case(n=64, width=6.0, ncomp=1, **kw):
    z = np.arange(n) + 0.5
    prof = W.RHO_VAP + (W.RHO_LIQ - W.RHO_VAP) * 0.5 * (
        np.tanh((z - n / 4) / width) - np.tanh((z - 3 * n / 4) / width))
    ct = np.zeros((n, 8, 8), np.uint8)
    rho = np.empty((ncomp, n, 8, 8))
    rho[0] = prof[:, None, None]
    amb = [W.RHO_VAP]
    if ncomp == 2:
        rho[1] = (1.0 - 0.1 * (prof - W.RHO_VAP) / (W.RHO_LIQ - W.RHO_VAP))[:, None, None]
        amb.append(1.0)
    params = dict(W.PHYSICS)
    params.update(ncomp=ncomp, periodic=(1, 1, 1), progressive=0, grav=(0, 0, 0))
    params.update(kw)
    return O.OracleSim(ct, rho, None, np.array(amb), **params)


def test_cohesion_continuum_limit():
    """On a smooth interface the discrete Eq. 8 force tends to
    -d/dz (p - c_s^2 rho) with p from the textbook EOS (mechanical
    consistency of Eqs. 6-8, sign and prefactors)."""
    s = _profile_case(width=8.0)
    rho = s.macro(0)[0][:, 4, 4]
    Fz = s.forces(0)[:, 4, 4, 2]
    c = O.eos_constants()
    pe = np.array([textbook_pr(1.0 / r, c["T"], c["Tc"]) for r in rho]) - rho / 3.0
    expect = -(np.roll(pe, -1) - np.roll(pe, 1)) / 2.0
    scale = np.abs(expect).max()
    assert scale > 1e-3
    assert np.abs(Fz - expect).max() < 0.03 * scale


def test_beta_invariance_of_g_scaling():
    """Only g psi^2 enters the force: rescaling g in Eqs. 6 and 8 together
    leaves the force unchanged (the reading that makes Eq. 6 and Eq. 8
    consistent)."""
    F1 = _profile_case(width=4.0, g_self=-1.0).forces(0)
    F2 = _profile_case(width=4.0, g_self=-3.7).forces(0)
    np.testing.assert_allclose(F2, F1, rtol=0, atol=1e-14 * np.abs(F1).max())


def test_cross_force_sign_and_balance():
    """Eq. 9 with g_12 > 0 pushes each component away from the other one's
    high-density side, and the two reactions cancel in total."""
    s = _profile_case(width=5.0, ncomp=2, g_self=0.0, g_cross=0.1)
    F0 = s.forces(0)
    F1 = s.forces(1)
    np.testing.assert_allclose(F0.sum(axis=(0, 1, 2)) + F1.sum(axis=(0, 1, 2)), 0.0, atol=1e-13)
    r1 = s.macro(1)[0][:, 4, 4]
    grad1 = (np.roll(r1, -1) - np.roll(r1, 1)) / 2
    fz0 = F0[:, 4, 4, 2]
    mask = np.abs(grad1) > 1e-4
    assert np.all(np.sign(fz0[mask]) == -np.sign(grad1[mask]))


def test_adhesion_sign():
    """Fluid-solid force: with g_ads < 0 liquid next to a wall is pulled
    towards it; at or below the ambient density it feels nothing."""
    n = 16
    ct = np.zeros((n, 8, 8), np.uint8)
    ct[0] = 1
    ct[n - 1] = 1
    rho = np.full((1, n, 8, 8), W.RHO_VAP)
    rho[0, 1:4] = W.RHO_LIQ
    p = dict(W.PHYSICS)
    p.update(ncomp=1, periodic=(1, 1, 0), progressive=0, g_self=0.0, g_ads=(-0.2, 0.0))
    s = O.OracleSim(ct, rho, None, np.array([W.RHO_VAP]), **p)
    F = s.forces(0)
    assert F[1, 4, 4, 2] < 0          # liquid above the floor: pulled down onto it
    assert abs(F[n - 2, 4, 4, 2]) < 1e-15  # vapour under the lid: no adhesion
    assert F[6, 4, 4, 2] == 0.0       # away from walls: nothing
