"""Numbers the paper prints for its lab inversion (Sec. IV), reproduced by the input helpers:
the 2-D operator has 64768 rows (A-scans) and 15373 unknowns (pixels of a 1 mm grid inside
the 70 mm-radius region of interest). The unknown count pins the grid convention: pixel
centres on whole millimetres; centres on half millimetres would give 15380."""
import numpy as np

import workloads as wl


def test_roi_pixel_count_of_the_lab_inversion():
    px = wl.roi_pixels(70e-3, 1e-3)
    assert len(px) == 15373
    assert len(wl.roi_pixels(70e-3, 1e-3, half_offset=True)) == 15380
    # every pixel lies inside the ROI, and the grid is symmetric about both axes
    assert np.all(np.hypot(px[:, 0], px[:, 1]) <= 70e-3 * (1 + 1e-12))
    assert np.isclose(px[:, 0].sum(), 0.0, atol=1e-9) and np.isclose(px[:, 1].sum(), 0.0, atol=1e-9)


def test_lab_acquisition_rows():
    assert wl.lab_ascan_count() == 64768
    assert (wl.lab_ascan_count(), len(wl.roi_pixels(70e-3, 1e-3))) == (64768, 15373)
