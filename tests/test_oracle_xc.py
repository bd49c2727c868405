"""Pins of the oracle's LDA against the uniform-gas closed form and thermodynamic identities."""
import os

import numpy as np

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
    assert abs(e_lo[0] - e_hi[0]) < 1e-4
    assert abs(v_lo[0] - v_hi[0]) < 1e-4


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
