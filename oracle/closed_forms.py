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


def ising1d_coverage(betaK: float, betah: float) -> float:
    """Infinite-ring equilibrium coverage of the 1D lattice gas with
    H = -K sum s_x s_{x+1} + h sum s_x (Section 7, Eq. exactcov1d; ka = kd).
    In +-1 spins s = (1 + m)/2 this is the 1D Ising chain with coupling
    beta K / 4 and field beta (K - h) / 2, whose transfer-matrix
    magnetisation is sinh(B) / sqrt(sinh(B)^2 + exp(-4 J)); hence
    theta = (1 + sinh(b) / sqrt(sinh(b)^2 + exp(-beta K))) / 2, b = beta (K - h) / 2."""
    b = 0.5 * (betaK - betah)
    sb = math.sinh(b)
    return 0.5 * (1.0 + sb / math.sqrt(sb * sb + math.exp(-betaK)))


def ising1d_ring(L: int, betaK: float, betah: float, rmax: int = 0):
    """Exact equilibrium of a finite ring of L sites by the 2x2 transfer
    matrix T[s, s'] = z^(s/2) exp(beta K s s') z^(s'/2), z = exp(-beta h):
    returns (coverage, [<s_0 s_r> for r = 1..rmax])."""
    import numpy as np
    z = math.exp(-betah)
    v = np.array([1.0, math.sqrt(z)])
    T = np.outer(v, v) * np.array([[1.0, 1.0], [1.0, math.exp(betaK)]])
    D = np.diag([0.0, 1.0])
    # scale T by its top eigenvalue to keep the powers finite
    lam = np.linalg.eigvalsh(T).max()
    T = T / lam
    Z = np.trace(np.linalg.matrix_power(T, L))
    cov = np.trace(D @ np.linalg.matrix_power(T, L)) / Z
    corr = [np.trace(D @ np.linalg.matrix_power(T, r) @ D @ np.linalg.matrix_power(T, L - r)) / Z
            for r in range(1, rmax + 1)]
    return float(cov), [float(c) for c in corr]


def ising1d_covariance(betaK: float, betah: float, r: int) -> float:
    """Infinite-ring connected correlation <s_0 s_r> - theta^2 of the same
    chain (Eq. exactcorr1d): theta (1 - theta) (lambda_- / lambda_+)^r, with
    lambda_(+-) = e^{K'} cosh(h') +- sqrt(e^{2K'} sinh(h')^2 + e^{-2K'}) the
    eigenvalues of the +-1 transfer matrix, K' = beta K / 4, h' = beta (K - h) / 2.
    theta (1 - theta) = (1 - m^2) / 4 = 1 / (4 (1 + e^{4K'} sinh(h')^2))."""
    kp = 0.25 * betaK
    hp = 0.5 * (betaK - betah)
    root = math.sqrt(math.exp(2 * kp) * math.sinh(hp) ** 2 + math.exp(-2 * kp))
    lp = math.exp(kp) * math.cosh(hp) + root
    lm = math.exp(kp) * math.cosh(hp) - root
    pre = 0.25 / (1.0 + math.exp(4 * kp) * math.sinh(hp) ** 2)
    return pre * (lm / lp) ** r
