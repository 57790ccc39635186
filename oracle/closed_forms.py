"""Closed forms the paper prints or implies (test infrastructure)."""
from __future__ import annotations

import math


def coverage_noninteracting(t: float, theta0: float, ka: float, kd: float) -> float:
    """Mean coverage of independent adsorption/desorption sites (Eq. adsdesrate
    with J = 0): each site is a two-state chain with rates ka (0->1) and kd
    (1->0), so theta(t) = a + (theta0 - a) exp(-(ka+kd) t), a = ka/(ka+kd)."""
    a = ka / (ka + kd)
    return a + (theta0 - a) * math.exp(-(ka + kd) * t)


BETA_C_J = 0.5 * math.asinh(1.0)  # sinh(2 beta_c J) = 1, i.e. sinh(beta_c K / 2) = 1 with K = 4J


def onsager_magnetisation(betaJ: float) -> float:
    """Spontaneous magnetisation of the square-lattice Ising model in +-1
    spins: (1 - sinh(2 beta J)^-4)^(1/8) below the critical temperature, 0
    above (Eq. exactcov2d gives the coverage (1 + m)/2 with beta K/2 = 2 beta J)."""
    if betaJ <= BETA_C_J:
        return 0.0
    return (1.0 - math.sinh(2.0 * betaJ) ** -4) ** 0.125


def onsager_coverage(betaJ: float) -> float:
    """Eq. exactcov2d: mean lattice-gas coverage of the majority phase."""
    return 0.5 * (1.0 + onsager_magnetisation(betaJ))
