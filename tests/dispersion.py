"""Linear kinetic dispersion relation of an electron plasma (closed form).

For a sum of drifting Maxwellians with density fractions n_s, drifts u_s and
thermal speeds s_s along k (unit plasma frequency, q/m = -1, eps0 = 1):

    1 - sum_s n_s Z'(zeta_s) / (2 k^2 s_s^2) = 0,   zeta_s = (w - k u_s) / (sqrt(2) k s_s)

with the plasma dispersion function Z(z) = i sqrt(pi) w(z) (Faddeeva w) and
Z'(z) = -2 (1 + z Z(z)).  Used only to pin the oracle's physics: it is
textbook plasma theory and shares nothing with either implementation.
"""
import math

import numpy as np
from scipy.optimize import fsolve
from scipy.special import wofz


def _zprime(z):
    Z = 1j * math.sqrt(math.pi) * wofz(z)
    return -2.0 * (1.0 + z * Z)


def root(k, guess, species=((1.0, 0.0, 1.0),)):
    """Complex frequency w solving the dispersion relation near ``guess``."""

    def f(w):
        ww = w[0] + 1j * w[1]
        r = 1.0 + 0j
        for n_s, u_s, s_s in species:
            z = (ww - k * u_s) / (math.sqrt(2.0) * k * s_s)
            r -= n_s * _zprime(z) / (2.0 * k * k * s_s * s_s)
        return [r.real, r.imag]

    sol = fsolve(f, [guess.real, guess.imag], xtol=1e-14)
    res = f(sol)
    assert abs(res[0]) + abs(res[1]) < 1e-9, res
    return complex(sol[0], sol[1])
