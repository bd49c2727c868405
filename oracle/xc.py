"""Local density approximation, spin-unpolarized (oracle).

The paper takes V_xc and eps_xc from Libxc's LDA (Sec. 2.1, Sec. 4.1); Libxc is not
available, so the functional is written out from its published definition:

* Slater (Dirac) exchange: eps_x = -(3/4) (3 rho / pi)^(1/3), V_x = (4/3) eps_x.
* Perdew-Zunger 1981 correlation (Phys. Rev. B 23, 5048), unpolarized parameters,
  with the Wigner-Seitz radius r_s = (3 / (4 pi rho))^(1/3):
    r_s >= 1:  eps_c = gamma / (1 + beta1 sqrt(r_s) + beta2 r_s)
    r_s <  1:  eps_c = A ln r_s + B + C r_s ln r_s + D r_s
  V_c = eps_c - (r_s / 3) d eps_c / d r_s   (from V = d(rho eps)/d rho).

Densities below RHO_MIN give eps = V = 0.

Pins: the exchange constant of the uniform gas, V = d(rho eps)/d rho, the Gell-Mann-Brueckner
slope (A), and the two continuity conditions at r_s = 1 by which PZ81 fixed C and D from
gamma, beta1, beta2, A and B (value and first derivative).  Parity unpinned: the last digit of
beta1 and of beta2 (a change of about 1e-3 in either keeps C and D within their rounding; no
published table of eps_c is at hand to fix them further).
"""
from __future__ import annotations

import numpy as np

RHO_MIN = 1e-14
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def exchange(rho):
    """Slater exchange energy per particle and potential."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = -0.75 * np.cbrt(3.0 * rho / np.pi)
    return eps, (4.0 / 3.0) * eps


def correlation(rho):
    """PZ81 correlation energy per particle and potential."""
    rho = np.asarray(rho, dtype=np.float64)
    rs = np.cbrt(3.0 / (4.0 * np.pi * rho))
    eps = np.empty_like(rs)
    deps = np.empty_like(rs)
    hi = rs >= 1.0
    r = rs[hi]
    den = 1.0 + PZ_BETA1 * np.sqrt(r) + PZ_BETA2 * r
    eps[hi] = PZ_GAMMA / den
    deps[hi] = -PZ_GAMMA * (PZ_BETA1 / (2.0 * np.sqrt(r)) + PZ_BETA2) / den ** 2
    lo = ~hi
    r = rs[lo]
    lr = np.log(r)
    eps[lo] = PZ_A * lr + PZ_B + PZ_C * r * lr + PZ_D * r
    deps[lo] = PZ_A / r + PZ_C * (lr + 1.0) + PZ_D
    return eps, eps - rs / 3.0 * deps


def lda(rho):
    """(eps_xc, V_xc) at densities rho; zero below RHO_MIN."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    V = np.zeros_like(rho)
    m = rho >= RHO_MIN
    ex, vx = exchange(rho[m])
    ec, vc = correlation(rho[m])
    eps[m] = ex + ec
    V[m] = vx + vc
    return eps, V
