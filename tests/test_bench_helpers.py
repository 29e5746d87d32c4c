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
