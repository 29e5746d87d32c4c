"""Host logic of the tensor-core PSF path (fft_psf_row_groups, no device work): rows grouped by
the set of subsets that hold them, so that each subset's PSF (Sec. II-D, Eq. resolution_2) is
the sum of the groups inside it. Checked against the membership sets written out in numpy."""
import numpy as np
import pytest

import workloads as wl


@pytest.fixture(scope="module")
def fg():
    import paper_1908_03302_gb300 as fg
    fg._lib.load()
    return fg


def membership(n_rows, subsets):
    m = np.zeros(n_rows, dtype=np.int64)
    for s, rows in enumerate(subsets):
        m[np.asarray(rows)] |= 1 << s
    return m


def check_grouping(n_rows, subsets, grp, gmask):
    m = membership(n_rows, subsets)
    assert np.all((grp == 255) == (m == 0))
    inside = grp != 255
    assert np.all(gmask[grp[inside]] == m[inside])          # each row's group is its set
    assert len(set(gmask.tolist())) == len(gmask)            # one group per distinct set
    first = [int(np.flatnonzero(grp == g)[0]) for g in range(len(gmask))]
    assert first == sorted(first)                            # numbered by first row
    # each subset is the union of the groups whose set holds it
    for s, rows in enumerate(subsets):
        gs = [g for g in range(len(gmask)) if (int(gmask[g]) >> s) & 1]
        assert np.array_equal(np.sort(np.flatnonzero(np.isin(grp, gs))), np.sort(np.asarray(rows)))


def test_nested_ring_subsets_give_one_group_per_subset(fg):
    subsets = wl.ring_subsets(n_tx=32, n_slices=2, n_bands=2)      # every 4th / 2nd / every element
    n_rows = 2 * 2 * 32 * 31 // 2
    grp, gmask = fg.psf_row_groups(n_rows, subsets)
    assert sorted(gmask.tolist()) == [0b100, 0b110, 0b111]
    check_grouping(n_rows, subsets, grp, gmask)


def test_overlapping_subsets(fg):
    n_rows = 200
    a, b = np.arange(0, 120, dtype=np.int32), np.arange(80, 190, dtype=np.int32)
    grp, gmask = fg.psf_row_groups(n_rows, [a, b, np.zeros(0, np.int32)])
    assert gmask.tolist() == [0b01, 0b11, 0b10]
    check_grouping(n_rows, [a, b, np.zeros(0, np.int32)], grp, gmask)


def test_more_than_32_groups_and_refusals(fg):
    rng = np.random.default_rng(40)
    n_rows = 500
    subsets = [np.flatnonzero(rng.random(n_rows) < 0.5).astype(np.int32) for _ in range(6)]
    assert len(np.unique(membership(n_rows, subsets)[membership(n_rows, subsets) > 0])) > 32
    assert fg.psf_row_groups(n_rows, subsets) == (None, None)
    with pytest.raises(fg.FFTError) as ei:                    # a row listed twice
        fg.psf_row_groups(n_rows, [np.array([3, 7, 7], dtype=np.int32)])
    assert ei.value.status == fg._lib.FFT_ERR_ARG
    with pytest.raises(fg.FFTError):                          # a row out of range
        fg.psf_row_groups(n_rows, [np.array([3, n_rows], dtype=np.int32)])
