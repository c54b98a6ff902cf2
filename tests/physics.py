"""Textbook formulas used by the oracle pins (independent statements, not the oracle's code).

Planck function, rigid-rotor partition-function limits, Keplerian speed and the solid angle
of a pixel are written here from their standard definitions so that the pins compare the
oracle's march with physics it must reproduce.
"""

import math

H = 6.62607015e-27
K = 1.380649e-16
C = 2.99792458e10
AMU = 1.66053906660e-24
GM_SUN = 1.3271244e26
AU = 1.495978707e13


def planck_nu(nu, T):
    """B_nu(T) = 2 h nu^3 / c^2 / (exp(h nu / k T) - 1)  [erg s^-1 cm^-2 Hz^-1 sr^-1]."""
    return 2.0 * H * nu ** 3 / C ** 2 / math.expm1(H * nu / (K * T))


def rayleigh_jeans(nu, T):
    return 2.0 * nu ** 2 * K * T / C ** 2


def rotor_Z_high_T(T, B):
    """High-temperature expansion of the rigid-rotor partition function
    Z = (1/x)(1 + x/3 + x^2/15 + 4x^3/315 + x^4/315 + ...), x = h B / k T."""
    x = H * B / (K * T)
    return (1.0 / x) * (1.0 + x / 3.0 + x * x / 15.0 + 4.0 * x ** 3 / 315.0 + x ** 4 / 315.0)


def rotor_Z_low_T(T, B, jmax=3):
    """Low-temperature limit: the first few terms of sum (2J+1) exp(-x J(J+1))."""
    x = H * B / (K * T)
    return sum((2 * J + 1) * math.exp(-x * J * (J + 1)) for J in range(jmax + 1))


def kepler_speed_kms(mstar_msun, r_au):
    return math.sqrt(GM_SUN * mstar_msun / (r_au * AU)) / 1e5


def pixel_solid_angle(pix_au, dist_pc):
    """A length L au at d pc subtends L/d arcsec; 1 arcsec = pi/648000 rad."""
    a = pix_au / dist_pc * math.pi / 648000.0
    return a * a
