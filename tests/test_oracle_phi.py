"""Pins for the oracle's Phi table and lookup (Sec. II-C, Eq. Kernel_freq, truncation).

Each check reaches the value by a route other than the oracle's own quadrature:
the closed form for the Gaussian power spectrum, Phi(0) = 0, Phi'(0) = E[w^4]/E[w^2],
the normalisation int_0^inf Phi = 1, and the exact lookup rules at knots and cut-offs.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import closed_form as cf

BANDS = [(1.0e6, 0.3e6), (1.0e6, 0.4e6), (0.6e6, 0.2e6), (1.0e6, 0.2e6), (1.4e6, 0.2e6)]


@pytest.mark.parametrize("fc,fs", BANDS)
def test_table_matches_closed_form(fc, fs):
    n, dt_max = 4096, 3.0 / fc
    tab = oracle.phi_table_gauss(fc, fs, n, dt_max)
    ref = cf.phi_gauss_closed(np.arange(n) * dt_max / (n - 1), fc, fs)
    assert np.max(np.abs(tab - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_closed_form_max_value():
    # Peak of Phi for the 1 MHz / 0.3 MHz band: 6.909e6 1/s, reached inside the first period.
    tau = np.linspace(0, 3e-6, 300001)
    phi = cf.phi_gauss_closed(tau, 1e6, 0.3e6)
    assert abs(phi.max() / 6.909238e6 - 1) < 1e-6
    assert tau[np.argmax(phi)] < 0.5e-6


@pytest.mark.parametrize("fc,fs", BANDS)
def test_table_zero_slope_and_mass(fc, fs):
    n, dt_max = 4096, 3.0 / fc
    tab = oracle.phi_table_gauss(fc, fs, n, dt_max)
    step = dt_max / (n - 1)
    assert tab[0] == 0.0                                   # sin(0) = 0
    slope = (tab[1] - tab[0]) / step
    assert abs(slope / cf.phi_gauss_slope0(fc, fs) - 1) < 2e-5
    # int_0^inf Phi = int w^3 W / w / int w^2 W = 1: the table's mass plus the closed-form
    # tail beyond the cut-off (Gaussian envelope, small for wide bands) is 1.
    s = 2 * math.pi * fs
    tail_t = np.linspace(dt_max, dt_max + 12.0 / s, 200001)
    tail = np.trapezoid(cf.phi_gauss_closed(tail_t, fc, fs), tail_t)
    # trapezoid with its Euler-Maclaurin end correction -h^2/12 (Phi'(b) - Phi'(0))
    end_slope = (tab[-1] - tab[-2]) / step
    mass = np.trapezoid(tab, dx=step) - step ** 2 / 12 * (end_slope - cf.phi_gauss_slope0(fc, fs))
    assert abs(mass + tail - 1) < 1e-8
    if fs / fc >= 0.3:
        assert abs(tail) < 1e-5


def test_sampled_spectrum_matches_gaussian():
    # kind=1 (sampled W on a node grid) reproduces kind=0 for the same Gaussian W.
    fc, fs = 1.0e6, 0.3e6
    w0, s = 2 * math.pi * fc, 2 * math.pi * fs
    om = np.linspace(0, w0 + 12 * s, 20001)
    W = np.exp(-0.5 * ((om - w0) / s) ** 2) + np.exp(-0.5 * ((om + w0) / s) ** 2)
    a = oracle.phi_table_sampled(om, W, 1024, 3e-6)
    b = oracle.phi_table_gauss(fc, fs, 1024, 3e-6)
    assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))


def test_lookup_rules():
    n, dt_max = 4096, 3e-6
    tab = oracle.phi_table_gauss(1e6, 0.3e6, n, dt_max)
    step = dt_max / (n - 1)
    for k in (1, 7, 1000, 4094):
        assert oracle.phi_lookup(tab, dt_max, k * step) == pytest.approx(tab[k], rel=1e-12, abs=1e-6)
        mid = oracle.phi_lookup(tab, dt_max, (k + 0.5) * step)
        assert mid == pytest.approx(0.5 * (tab[k] + tab[k + 1]), rel=1e-9, abs=1e-6)
    assert oracle.phi_lookup(tab, dt_max, 0.0) == 0.0
    assert oracle.phi_lookup(tab, dt_max, -1e-9) == 0.0
    assert oracle.phi_lookup(tab, dt_max, dt_max) == 0.0
    assert oracle.phi_lookup(tab, dt_max, 2 * dt_max) == 0.0
    # Linear interpolation error against the exact function stays below 1e-5 of max|Phi|.
    t = np.random.default_rng(0).uniform(0, dt_max, 2000)
    got = np.array([oracle.phi_lookup(tab, dt_max, x) for x in t])
    ref = cf.phi_gauss_closed(t, 1e6, 0.3e6)
    assert np.max(np.abs(got - ref)) < 1e-5 * np.max(np.abs(ref))


def test_narrower_kernels_at_higher_frequency():
    # Sec. II-B: higher frequencies give narrower kernels; the first zero crossing of Phi
    # (edge of the first Fresnel zone in detour time) moves in as 1/fc.
    def first_zero(fc):
        tab = oracle.phi_table_gauss(fc, 0.2e6, 4096, 3.0 / fc)
        k = int(np.argmax(tab[1:] < 0)) + 1
        return k * (3.0 / fc) / 4095
    z06, z10, z14 = first_zero(0.6e6), first_zero(1.0e6), first_zero(1.4e6)
    assert z06 > z10 > z14
