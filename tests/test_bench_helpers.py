"""Host helpers of bench.py that need no GPU."""
import numpy as np

import bench


def test_fwhm_of_a_gaussian_and_missing_edges():
    h = 1e-3
    x = np.arange(-20, 21) * h
    sig = 3e-3
    p = np.exp(-0.5 * (x / sig) ** 2)
    # linear interpolation between 1 mm samples of a 3 mm Gaussian: within 1 %
    assert abs(bench.fwhm(p, h, 20) - 2 * np.sqrt(2 * np.log(2)) * sig) < 0.01 * 7.06e-3
    assert bench.fwhm(np.ones(9), h, 4) is None          # never falls to half
    assert bench.fwhm(-p, h, 20) is None                 # no positive peak


def test_ring256_3band_workload():
    # ring256's array and grid with slices3d's three bands, rows ordered (band, pair)
    import workloads as wl
    a, b, s = wl.by_name("ring256_3band"), wl.ring256(), wl.slices3d()
    assert np.array_equal(a.tx, b.tx) and np.array_equal(a.pairs, b.pairs)
    assert (a.grid.nx, a.grid.ny, a.grid.nz, a.grid.h) == (b.grid.nx, b.grid.ny, b.grid.nz, b.grid.h)
    assert [(x.f_center_hz, x.f_sigma_hz) for x in a.bands] == [(x.f_center_hz, x.f_sigma_hz) for x in s.bands]
    assert a.n_rows == 3 * len(b.pairs)
    assert np.array_equal(a.band_of_row, np.repeat(np.arange(3), len(b.pairs)))
    assert np.array_equal(a.row_pairs()[len(b.pairs):2 * len(b.pairs)], b.pairs)
