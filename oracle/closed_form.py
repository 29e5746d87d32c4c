"""Independent closed forms and brute-force references that pin the C oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring). None of these functions reuses the
C oracle's quadrature; each one reaches the same quantity by a different route:

* ``phi_gauss_closed``: Phi(tau) for the Gaussian power spectrum in closed form, from
  int w^n G(w - w0) e^{i w tau} dw = (-i d/dtau)^n [sqrt(2 pi) s e^{i w0 tau - s^2 tau^2 / 2}]
  applied to Eq. Kernel_freq with the even extension of W.
* ``phi_gauss_slope0``: Phi'(0) = E[w^4] / E[w^2] of the Gaussian.
* ``uniform_dc_prolate``: the integral of K0 over all space in prolate-spheroidal
  coordinates, where dV / (R_xs R_xr) = (L/2) dsigma dtau dphi makes it collapse to
  -(L / c0^2) * int Phi (the ray-theory limit, Sec. II-B / Fig. 1 dashed line).
* ``born_cc_traveltime``: the cross-correlation traveltime shift (Eqs. cc_funct,
  relation_CC) of Born-scattered waveforms (Eqs. pressure_field1, pressure_field2,
  Green_freq) from one point scatterer, found by Newton iteration on C'(tau) = 0
  evaluated as a frequency sum in double precision.
"""
from __future__ import annotations

import math
from typing import Callable, Tuple

import numpy as np


def phi_gauss_closed(tau, f_center: float, f_sigma: float):
    """Closed-form Phi(tau) (1/s) for W(w) = G(w - w0) + G(w + w0), G(x) = exp(-x^2 / (2 s^2)).

    With psi = i w0 - s^2 tau, the numerator is Re[(psi^3 - 3 s^2 psi) e^{i w0 tau}]
    times sqrt(2 pi) s e^{-s^2 tau^2/2}, and the denominator sqrt(2 pi) s (w0^2 + s^2).
    """
    tau = np.asarray(tau, dtype=np.float64)
    w0 = 2 * math.pi * f_center
    s = 2 * math.pi * f_sigma
    a = -s * s * tau                  # Re psi
    b = w0                            # Im psi
    X = a ** 3 - 3 * a * b * b - 3 * s * s * a
    Y = 3 * a * a * b - b ** 3 - 3 * s * s * b
    return np.exp(-0.5 * s * s * tau * tau) * (X * np.cos(w0 * tau) - Y * np.sin(w0 * tau)) / (w0 * w0 + s * s)


def phi_gauss_slope0(f_center: float, f_sigma: float) -> float:
    """Phi'(0) = int w^4 W / int w^2 W = (w0^4 + 6 w0^2 s^2 + 3 s^4) / (w0^2 + s^2)."""
    w0 = 2 * math.pi * f_center
    s = 2 * math.pi * f_sigma
    return (w0 ** 4 + 6 * w0 ** 2 * s ** 2 + 3 * s ** 4) / (w0 ** 2 + s ** 2)


def gauss_legendre(n: int) -> Tuple[np.ndarray, np.ndarray]:
    return np.polynomial.legendre.leggauss(n)


def uniform_dc_prolate(k0_at: Callable[[np.ndarray], float], xs, xr, c0: float, dt_max: float,
                       n_table: int, n_tau: int = 6, n_phi: int = 5, sub: int = 2) -> float:
    """Integral of K0 over space in prolate-spheroidal coordinates about the pair.

    x = o + (L/2) [sigma tau e + sqrt((sigma^2 - 1)(1 - tau^2)) (cos phi u + sin phi w)],
    dV = (L/2)^3 (sigma^2 - tau^2) dsigma dtau dphi. The detour is R = L (sigma - 1), so
    sigma runs over [1, 1 + c0 dt_max / L]; the sigma rule is the trapezoid rule on the
    table knots (subdivided `sub` times), exact for the piecewise-linear Phi.
    """
    xs = np.asarray(xs, dtype=np.float64)
    xr = np.asarray(xr, dtype=np.float64)
    ax = xr - xs
    L = float(np.linalg.norm(ax))
    e = ax / L
    tmp = np.array([1.0, 0.0, 0.0]) if abs(e[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u = np.cross(e, tmp)
    u /= np.linalg.norm(u)
    w = np.cross(e, u)
    o = 0.5 * (xs + xr)
    hl = 0.5 * L
    n_knots = (n_table - 1) * sub + 1
    sig = 1.0 + np.linspace(0.0, c0 * dt_max / L, n_knots)
    wsig = np.full(n_knots, sig[1] - sig[0])
    wsig[0] *= 0.5
    wsig[-1] *= 0.5
    tn, tw = gauss_legendre(n_tau)
    phis = 2 * math.pi * (np.arange(n_phi) + 0.5) / n_phi
    total = 0.0
    for a, wa in zip(sig, wsig):
        acc = 0.0
        for t, wt in zip(tn, tw):
            rad = hl * math.sqrt(max((a * a - 1.0) * (1.0 - t * t), 0.0))
            for ph in phis:
                x = o + hl * a * t * e + rad * (math.cos(ph) * u + math.sin(ph) * w)
                acc += wt * (2 * math.pi / n_phi) * k0_at(x) * hl ** 3 * (a * a - t * t)
        total += wa * acc
    return total


def wavelet_spectrum(omega: np.ndarray, a: float, w0: float) -> np.ndarray:
    """F(w) = int f(t) e^{-i w t} dt of f(t) = exp(-a t^2) cos(w0 t) (real and even)."""
    c = 0.5 * math.sqrt(math.pi / a)
    return c * (np.exp(-(omega - w0) ** 2 / (4 * a)) + np.exp(-(omega + w0) ** 2 / (4 * a)))


def born_cc_traveltime(xs, xr, xp, eps: float, c0: float, a: float, w0: float,
                       omega: np.ndarray, n_newton: int = 30) -> float:
    """Cross-correlation time shift of p0 + dp against p0 for a point scatterer at xp.

    Convention F(w) = int f(t) e^{-i w t} dt, G0(x; y, w) = exp(-i w |x-y| / c0) / (4 pi |x-y|).
    p0(w) = F(w) G0(xr; xs) and dp(w) = -(2 w^2 eps / c0^3) F(w) G0(xp; xs) G0(xr; xp), with
    eps = dc * dV the scatterer strength. C(tau) = int pobs(t + tau) p0(t) dt, so
    C'(tau) = (1/pi) Re int_0^inf i w Pobs P0* e^{i w tau} dw. The root of C' nearest 0 is
    found by Newton's method (trapezoid rule over the given omega nodes).
    """
    xs, xr, xp = (np.asarray(v, dtype=np.float64) for v in (xs, xr, xp))
    F = wavelet_spectrum(omega, a, w0)

    def g0(x, y):
        r = float(np.linalg.norm(x - y))
        return np.exp(-1j * omega * r / c0) / (4 * math.pi * r)

    p0 = F * g0(xr, xs)
    dp = -(2 * omega ** 2 * eps / c0 ** 3) * F * g0(xp, xs) * g0(xr, xp)
    cross = (p0 + dp) * np.conj(p0)
    wq = np.full(len(omega), omega[1] - omega[0])
    wq[0] *= 0.5
    wq[-1] *= 0.5
    tau = 0.0
    for _ in range(n_newton):
        ph = np.exp(1j * omega * tau)
        c1 = np.sum(wq * (1j * omega * cross * ph).real)
        c2 = np.sum(wq * (-(omega ** 2) * cross * ph).real)
        step = c1 / c2
        tau -= step
        if abs(step) < 1e-30:
            break
    return tau
