"""Parity of the sine-series Phi path (Sec. II-C: Phi stored as the amplitudes and frequencies
of its sine terms, evaluated inside every product) with the FP64 oracle's series, through the C ABI.

Tolerances as for the table path: J and J^T <= 1e-5 relative L2, CG model <= 1e-4. The FP32
Clenshaw recurrence is good to a few 1e-6 of max |Phi| (it amplifies the rounding of cos x by
up to ~n^2 near x = 0), so these bars leave a margin of ~5.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_common import rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_03302_gb300 as m
    m._lib.load()
    return m


def _geoms(fg, w, bands=None, band_of_row=None, n_terms=0):
    """Series geometries of the same workload on both sides (bands: (fc, fs, dt_max) list)."""
    if bands is None:
        bands = [(b.f_center_hz, b.f_sigma_hz, b.dt_max) for b in w.bands]
    tabs = [fg.TrigTable(fc, fs, dtm, n_terms) for fc, fs, dtm in bands]
    geo = fg.Geometry(w.tx, w.row_pairs(), w.grid, w.c0, tabs, band_of_row=band_of_row)
    series = [oracle.trig_coefs(fc, fs, dtm, n_terms) for fc, fs, dtm in bands]
    og = oracle.Geometry(w.tx, w.row_pairs(), band_of_row, [a for a, _ in series], [b[2] for b in bands],
                         w.grid, w.c0, trig_dw=[dw for _, dw in series])
    return geo, og, tabs


def test_series_coefficients_match_oracle(fg):
    for fc, fs, dtm in [(1e6, 0.3e6, 3e-6), (1e6, 0.4e6, 3e-6), (0.6e6, 0.2e6, 5e-6), (1.4e6, 0.2e6, 3 / 1.4e6)]:
        t = fg.TrigTable(fc, fs, dtm)
        a, dw = oracle.trig_coefs(fc, fs, dtm)
        assert t.n == len(a)
        assert t.dw == pytest.approx(dw, rel=1e-14)
        assert np.max(np.abs(t.coef - a)) <= 1e-10 * np.max(np.abs(a))
        t8 = fg.TrigTable(fc, fs, dtm, n_terms=8)
        assert t8.n == 8 and np.allclose(t8.coef, oracle.trig_coefs(fc, fs, dtm, 8)[0], rtol=1e-10, atol=0)


def test_series_J_JT_CG_ring32(fg):
    w = wl.ring32()
    geo, og, _ = _geoms(fg, w)
    assert geo.info().phi_terms == len(oracle.trig_coefs(1e6, 0.3e6, 3e-6)[0])
    m = wl.model_for(w)
    assert rel_l2(to_np(geo.J(to_dev(m))), og.J(m)) <= 1e-5
    dd = np.random.default_rng(7).normal(size=og.M) * 1e-8
    assert rel_l2(to_np(geo.JT(to_dev(dd))), og.JT(dd)) <= 1e-5
    # the support count does not depend on Phi
    assert abs(geo.support_evals - og.count_support()) <= 1e-4 * og.count_support()
    d = og.J(m) + wl.noise(og.M, w.noise_seed)
    m_ref, hist_ref, rc = og.cgls(d, og.lambda_abs(w.lambda_rel), w.cg_iters)
    assert rc == 0
    assert geo.frob2() == pytest.approx(og.frob2(), rel=1e-5)
    m_gpu, hist = geo.cg_solve(to_dev(d), w.lambda_rel, w.cg_iters, with_history=True)
    assert rel_l2(to_np(m_gpu), m_ref) <= 1e-4
    assert np.allclose(hist, hist_ref, rtol=1e-3)


def test_series_three_bands_ragged(fg):
    # three bands with different term counts on a grid that is ragged in every axis
    w = wl.tiny()
    M = len(w.row_pairs())
    bor = (np.arange(M) % 3).astype(np.int32)
    bands = [(0.6e6, 0.2e6, 5.0e-6), (1.0e6, 0.2e6, 3.0e-6), (1.4e6, 0.2e6, 3.0 / 1.4e6)]
    geo, og, tabs = _geoms(fg, w, bands, bor)
    m = np.random.default_rng(3).normal(size=og.V)
    assert rel_l2(to_np(geo.J(to_dev(m))), og.J(m)) <= 1e-5
    dd = np.random.default_rng(4).normal(size=og.M)
    assert rel_l2(to_np(geo.JT(to_dev(dd))), og.JT(dd)) <= 1e-5


def test_series_sharp_cut(fg):
    # a cut-off well inside the kernel (dt_max = 1.2 us at 1 MHz): Phi at the cut is not small,
    # so the in/out decision near it is taken in FP64 (sharp-band path of the series kernel)
    w = wl.ring32()
    bands = [(1.0e6, 0.3e6, 1.2e-6)]
    geo, og, _ = _geoms(fg, w, bands)
    a, dw = oracle.trig_coefs(*bands[0])
    t = np.linspace(0, 1.2e-6, 2001)
    ph = np.array([oracle.phi_trig(a, dw, 1.2e-6, x) for x in t])
    assert abs(oracle.phi_trig(a, dw, 1.2e-6, 1.2e-6 * (1 - 1e-9))) > 1e-3 * np.abs(ph).max()
    m = wl.model_for(w)
    assert rel_l2(to_np(geo.J(to_dev(m))), og.J(m)) <= 1e-5
    dd = np.random.default_rng(9).normal(size=og.M)
    assert rel_l2(to_np(geo.JT(to_dev(dd))), og.JT(dd)) <= 1e-5


def test_series_fewer_terms_follow_the_oracle(fg):
    # truncated series (8 terms) are a different Phi; both sides must still agree on it
    w = wl.ring32()
    geo, og, _ = _geoms(fg, w, n_terms=8)
    m = wl.model_for(w)
    assert rel_l2(to_np(geo.J(to_dev(m))), og.J(m)) <= 1e-5


def test_series_rejections(fg):
    w = wl.tiny()
    t = fg.TrigTable(1e6, 0.3e6, 3e-6)
    with pytest.raises(fg.FFTError):
        fg.Geometry(w.tx, w.row_pairs(), w.grid, w.c0, [t], dt_mode=fg.FFT_DT_NAIVE)
    with pytest.raises(fg.FFTError):   # mixed representations
        fg.Geometry(w.tx, w.row_pairs(), w.grid, w.c0, [t, fg.Table(1e6, 0.3e6, 4096, 3e-6)],
                    band_of_row=np.zeros(len(w.row_pairs()), np.int32))
    with pytest.raises(fg.FFTError):
        fg.TrigTable(1e6, 0.3e6, 3e-6, n_terms=300)
    geo = fg.Geometry(w.tx, w.row_pairs(), w.grid, w.c0, [t])
    with pytest.raises(fg.FFTError):
        geo.psf_batch([5], [np.arange(len(w.row_pairs()), dtype=np.int32)], mode=0)
