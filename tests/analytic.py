"""Closed forms used to pin the oracle (no oracle or CUDA code here).

Ricker derivatives are written out by hand from w(t) = (1 - 2a tau^2) e^{-a tau^2},
a = (pi f0)^2, tau = t - delay. The Green's functions are those of
p_tt - c^2 lap p = s'(t) delta(x), which is what Eq. (1) reduces to for a
pressure source f_p = s(t) delta(x) in a homogeneous medium.
"""
import math

import numpy as np


def ricker_deriv(t, f0, delay, k):
    a = (math.pi * f0) ** 2
    tau = np.asarray(t, dtype=np.float64) - delay
    e = np.exp(-a * tau ** 2)
    if k == 0:
        return (1 - 2 * a * tau ** 2) * e
    if k == 1:
        return (-6 * a * tau + 4 * a ** 2 * tau ** 3) * e
    if k == 2:
        return ((-6 * a + 12 * a ** 2 * tau ** 2) + (12 * a ** 2 * tau ** 2 - 8 * a ** 3 * tau ** 4)) * e
    if k == 3:
        p = -6 * a + 24 * a ** 2 * tau ** 2 - 8 * a ** 3 * tau ** 4
        dp = 48 * a ** 2 * tau - 32 * a ** 3 * tau ** 3
        return (dp - 2 * a * tau * p) * e
    raise ValueError(k)


def green3d_pressure(r, t, c, f0, delay):
    """p(r, t) = s'(t - r/c) / (4 pi c^2 r) for s = Ricker(f0, delay)."""
    return ricker_deriv(t - r / c, f0, delay, 1) / (4 * math.pi * c * c * r)


def green2d_pressure(r, t, c, f0, delay, nquad=20001):
    """2D line-source response p = (1/(2 pi c^2)) int_0^U s'(t - (r/c) cosh u) du,
    U = arccosh(ct/r): the convolution of H(t - r/c)/(2 pi c^2 sqrt(t^2 - r^2/c^2))
    with s', after the substitution t' = (r/c) cosh u removes the singularity."""
    out = np.zeros_like(np.asarray(t, dtype=np.float64))
    for i, ti in enumerate(np.asarray(t)):
        if c * ti <= r:
            continue
        U = math.acosh(c * ti / r)
        u = np.linspace(0.0, U, nquad)
        f = ricker_deriv(ti - (r / c) * np.cosh(u), f0, delay, 1)
        out[i] = np.trapezoid(f, u) / (2 * math.pi * c * c)
    return out


def born3d_kappa_point(r1, r2, t, c, f0, delay, amp, cellvol):
    """Scattered pressure from a point dln kappa = amp of volume cellvol:
    dp = amp * V * s'''(t - (r1+r2)/c) / (16 pi^2 c^4 r1 r2)."""
    return amp * cellvol * ricker_deriv(t - (r1 + r2) / c, f0, delay, 3) / (
        16 * math.pi ** 2 * c ** 4 * r1 * r2)
