"""Pins of the oracle's LDA against the uniform-gas closed form and thermodynamic identities."""
import os

import numpy as np
import pytest

from oracle import xc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    for line in open(os.path.join(GOLDEN, "closed_forms.txt")):
        if line.strip() and not line.startswith("#"):
            k, v, _ = line.split()
            if k == name:
                return float(v)
    raise KeyError(name)


def test_exchange_matches_uniform_gas_rs_form():
    C = _golden("slater_exchange_coefficient")
    rs = np.array([0.1, 0.5, 1.0, 2.0, 5.0, 20.0])
    rho = 3.0 / (4.0 * np.pi * rs ** 3)
    ex, _ = xc.exchange(rho)
    np.testing.assert_allclose(ex, -C / rs, rtol=1e-14)


def test_potential_is_density_derivative_of_energy_density():
    # V_xc = d(rho eps_xc)/d rho, central differences on both PZ81 branches
    rho = np.logspace(-6, 3, 40)
    h = 1e-5 * rho
    ep, _ = xc.lda(rho + h)
    em, _ = xc.lda(rho - h)
    fd = ((rho + h) * ep - (rho - h) * em) / (2 * h)
    _, V = xc.lda(rho)
    np.testing.assert_allclose(V, fd, rtol=1e-8, atol=1e-12)


def test_pz81_branches_meet_at_rs_one():
    # the published (rounded) PZ81 parameters make eps_c and V_c continuous to ~3e-5 at r_s = 1
    rho1 = 3.0 / (4.0 * np.pi)
    e_lo, v_lo = xc.correlation(np.array([rho1 * (1 + 1e-12)]))   # r_s just below 1
    e_hi, v_hi = xc.correlation(np.array([rho1 * (1 - 1e-12)]))   # r_s just above 1
    assert abs(e_lo[0] - e_hi[0]) < 5e-5
    assert abs(v_lo[0] - v_hi[0]) < 5e-5


def _branch_slopes_at_rs_one():
    """d eps_c / d r_s at r_s = 1 from each branch of the oracle (one-sided differences)."""
    h = 1e-6
    rs = np.array([1.0 - 2 * h, 1.0 - h, 1.0 + h, 1.0 + 2 * h])
    e, _ = xc.correlation(3.0 / (4.0 * np.pi * rs ** 3))
    return (e[1] - e[0]) / h, (e[3] - e[2]) / h      # high-density branch, low-density branch


def check_pz81_continuity_constants():
    # Perdew and Zunger chose C and D so that eps_c and its first derivative are continuous at
    # r_s = 1 (Phys. Rev. B 23, 5048, 1981); solving those two conditions with the oracle's
    # gamma, beta1, beta2, A, B must give its C and D to their published four decimals.
    g, b1, b2, A, B = xc.PZ_GAMMA, xc.PZ_BETA1, xc.PZ_BETA2, xc.PZ_A, xc.PZ_B
    den = 1.0 + b1 + b2
    eps1 = g / den
    deps1 = -g * (b1 / 2.0 + b2) / den ** 2
    D = eps1 - B
    C = deps1 - A - D
    assert abs(C - xc.PZ_C) <= 5e-5, (C, xc.PZ_C)
    assert abs(D - xc.PZ_D) <= 5e-5, (D, xc.PZ_D)
    # and the oracle's two branches have slopes that meet at r_s = 1 to the constants' rounding
    s_hi, s_lo = _branch_slopes_at_rs_one()
    assert abs(s_hi - s_lo) < 3e-5, (s_hi, s_lo)


def test_pz81_high_density_constants_follow_from_continuity():
    check_pz81_continuity_constants()


@pytest.mark.parametrize("name,value", [("PZ_GAMMA", -0.1432), ("PZ_GAMMA", -0.1424), ("PZ_BETA1", 1.0592),
                                        ("PZ_BETA2", 0.3434), ("PZ_BETA2", 0.3324), ("PZ_A", 0.0313),
                                        ("PZ_C", 0.0002), ("PZ_D", -0.0161), ("PZ_D", -0.0106)])
def test_pz81_continuity_pin_catches_planted_typos(monkeypatch, name, value):
    monkeypatch.setattr(xc, name, value)
    with pytest.raises(AssertionError):
        check_pz81_continuity_constants()


def test_correlation_high_density_slope():
    # high-density limit of the uniform gas: d eps_c / d ln r_s -> (1 - ln 2)/pi^2 (Gell-Mann and
    # Brueckner 1957); PZ81 fits this coefficient to four digits
    rs = np.array([1e-8, 1e-7])
    e, _ = xc.correlation(3.0 / (4.0 * np.pi * rs ** 3))
    slope = (e[1] - e[0]) / np.log(10.0)
    assert abs(slope - (1.0 - np.log(2.0)) / np.pi ** 2) < 5e-5


def test_below_threshold_is_zero():
    e, V = xc.lda(np.array([0.0, 1e-15, xc.RHO_MIN]))
    assert e[0] == 0 and V[0] == 0 and e[1] == 0 and V[1] == 0
    assert e[2] < 0 and V[2] < 0
