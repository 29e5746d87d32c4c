"""Pins for the oracle's sine-series form of Phi (Sec. II-C: the operator is stored as the
amplitudes and frequencies of the sine terms of Eq. Kernel_freq) and for the geometry that
uses it.

* the series against the closed form of Phi for the Gaussian power spectrum, for the
  spectra of the reference workloads (the rectangle rule on equally spaced nodes is exact
  up to aliasing and term truncation, below 2e-8 of max |Phi| with the default rule);
* the error falls with the number of terms (accuracy against term count);
* truncation: 0 at dt <= 0 and at dt >= dt_max;
* J entries of a geometry in series mode against K0 written out in numpy from the closed
  form (band selection and node spacing passed per band), and J / J^T of the series
  geometry against the table geometry within the table's interpolation error.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from oracle import closed_form as cf

SPECTRA = [(1.0e6, 0.3e6, 3.0e-6), (1.0e6, 0.4e6, 3.0e-6), (0.6e6, 0.2e6, 5.0e-6),
           (1.0e6, 0.2e6, 3.0e-6), (1.4e6, 0.2e6, 3.0 / 1.4e6)]


@pytest.mark.parametrize("fc,fs,dtm", SPECTRA)
def test_series_matches_closed_form(fc, fs, dtm):
    a, dw = oracle.trig_coefs(fc, fs, dtm)
    assert 15 <= len(a) <= 30             # a short series
    t = np.linspace(0.0, dtm, 2001)[1:-1]
    ph = np.array([oracle.phi_trig(a, dw, dtm, x) for x in t])
    ex = cf.phi_gauss_closed(t, fc, fs)
    assert np.abs(ph - ex).max() <= 3e-8 * np.abs(ex).max()
    # node spacing: period T = max(2 dt_max, dt_max + 6.5 / s)
    s = 2 * np.pi * fs
    assert dw == pytest.approx(2 * np.pi / max(2 * dtm, dtm + 6.5 / s), rel=1e-15)


def test_error_falls_with_term_count():
    fc, fs, dtm = 1.0e6, 0.4e6, 3.0e-6
    t = np.linspace(0.0, dtm, 1501)[1:-1]
    ex = cf.phi_gauss_closed(t, fc, fs)
    errs = []
    for n in (10, 13, 16, 19, 22):
        a, dw = oracle.trig_coefs(fc, fs, dtm, n_terms=n)
        assert len(a) == n
        ph = np.array([oracle.phi_trig(a, dw, dtm, x) for x in t])
        errs.append(np.abs(ph - ex).max() / np.abs(ex).max())
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[0] > 1e-3 and errs[-1] < 1e-8


def test_series_truncation_and_sign():
    a, dw = oracle.trig_coefs(1.0e6, 0.3e6, 3.0e-6)
    assert oracle.phi_trig(a, dw, 3.0e-6, 0.0) == 0.0
    assert oracle.phi_trig(a, dw, 3.0e-6, -1e-7) == 0.0
    assert oracle.phi_trig(a, dw, 3.0e-6, 3.0e-6) == 0.0
    assert oracle.phi_trig(a, dw, 3.0e-6, 5.0e-6) == 0.0
    assert oracle.phi_trig(a, dw, 3.0e-6, 0.05e-6) > 0.0    # Phi > 0 near 0 (first zone K0 < 0)


def _k0_numpy(xs, xr, x, c0, fc, fs, dtm):
    rs, rr, L = np.linalg.norm(x - xs), np.linalg.norm(x - xr), np.linalg.norm(xr - xs)
    dt = (rs + rr - L) / c0
    if dt <= 0 or dt >= dtm:
        return 0.0
    return -L / (2 * np.pi * c0 ** 3 * rs * rr) * float(cf.phi_gauss_closed(np.array([dt]), fc, fs)[0])


def test_series_geometry_entries_multiband():
    # three bands with different term counts and spacings on a small slice geometry
    w = wl.tiny()
    bands = [(0.6e6, 0.2e6, 5.0e-6), (1.0e6, 0.2e6, 3.0e-6), (1.4e6, 0.2e6, 3.0 / 1.4e6)]
    series = [oracle.trig_coefs(*b) for b in bands]
    rows = w.row_pairs()
    M = len(rows)
    band = (np.arange(M) % 3).astype(np.int32)
    og = oracle.Geometry(w.tx, rows, band, [a for a, _ in series], [b[2] for b in bands], w.grid, w.c0,
                         trig_dw=[dw for _, dw in series])
    rng = np.random.default_rng(5)
    centres = w.grid.centres()
    checked = 0
    for _ in range(400):
        p, v = int(rng.integers(M)), int(rng.integers(w.grid.n_vox))
        xs, xr = w.tx[rows[p, 0]], w.tx[rows[p, 1]]
        fc, fs, dtm = bands[band[p]]
        x = centres[v]
        ref = _k0_numpy(xs, xr, x, w.c0, fc, fs, dtm) * w.grid.h ** 3
        got = og.entry(p, v)
        if ref != 0.0:
            checked += 1
        # the series is exact to 1e-8 of max |Phi|: scale the bound by A h^3 max |Phi|
        L, rs, rr = np.linalg.norm(xr - xs), np.linalg.norm(x - xs), np.linalg.norm(x - xr)
        tt = np.linspace(0.0, dtm, 4001)
        scale = L / (2 * np.pi * w.c0 ** 3 * rs * rr) * np.abs(cf.phi_gauss_closed(tt, fc, fs)).max() * w.grid.h ** 3
        assert abs(got - ref) <= 1e-8 * scale, (p, v, got, ref)
    assert checked > 20


def test_series_and_table_operators_agree():
    w = wl.ring32()
    og_t = oracle.Geometry.from_workload(w)
    og_s = oracle.Geometry.from_workload(w, phi="trig")
    m = wl.model_for(w)
    dt, ds = og_t.J(m), og_s.J(m)
    # the table's linear interpolation error is a few 1e-6 of max |Phi|
    assert np.linalg.norm(ds - dt) / np.linalg.norm(dt) < 2e-5
    d = np.random.default_rng(2).standard_normal(og_t.M)
    vox = np.arange(0, og_t.V, 97)
    gt, gs = og_t.JT(d, vox), og_s.JT(d, vox)
    assert np.linalg.norm(gs - gt) / np.linalg.norm(gt) < 2e-5
    # same support: the series is truncated at the same dt_max
    assert og_s.count_support() == og_t.count_support()
