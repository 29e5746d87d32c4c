"""Edge cases of the CUDA path against the FP64 oracle, through the C ABI: the largest number
of bands (8 tables of 2048 samples; 8 of 4096 do not fit in shared memory and are refused), the smallest table (2 samples: Phi is the straight line from 0
to its value at the cut-off, where the truncation sets it to 0), a single row, grids of one voxel and of one voxel
per axis but long along another, a PSF subset with no rows, and a spike that no row reaches."""
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


def _pair(fg, tx, rows, grid, bands, bor=None, n=4096):
    geo = fg.Geometry(tx, rows, grid, 1500.0, [fg.Table(fc, fs, n, d) for fc, fs, d in bands], band_of_row=bor)
    og = oracle.Geometry(tx, rows, bor, [oracle.phi_table_gauss(fc, fs, n, d) for fc, fs, d in bands],
                         [b[2] for b in bands], grid, 1500.0)
    return geo, og


def test_eight_bands(fg):
    w = wl.tiny()
    rows = w.row_pairs()
    bands = [(0.5e6 + 0.15e6 * k, 0.2e6, 3.0 / (0.5e6 + 0.15e6 * k)) for k in range(8)]
    bor = (np.arange(len(rows)) % 8).astype(np.int32)
    # 8 tables of 4096 samples (256 KB) do not fit in shared memory: a clear refusal
    with pytest.raises(fg.FFTError):
        _pair(fg, w.tx, rows, w.grid, bands, bor)
    geo, og = _pair(fg, w.tx, rows, w.grid, bands, bor, n=2048)
    m = np.random.default_rng(1).normal(size=og.V)
    d = np.random.default_rng(2).normal(size=og.M)
    assert rel_l2(to_np(geo.J(to_dev(m))), og.J(m)) <= 1e-5
    assert rel_l2(to_np(geo.JT(to_dev(d))), og.JT(d)) <= 1e-5
    with pytest.raises(fg.FFTError):   # nine tables are refused
        fg.Geometry(w.tx, rows, w.grid, 1500.0, [fg.Table(1e6, 0.3e6, 4096, 3e-6)] * 9,
                    band_of_row=np.zeros(len(rows), np.int32))


def test_two_sample_table(fg):
    w = wl.tiny()
    geo, og = _pair(fg, w.tx, w.row_pairs(), w.grid, [(1e6, 0.3e6, 3e-6)], n=2)
    m = np.random.default_rng(3).normal(size=og.V)
    ref = og.J(m)
    assert np.linalg.norm(ref) > 0
    assert rel_l2(to_np(geo.J(to_dev(m))), ref) <= 1e-5


def test_single_row_and_thin_grids(fg):
    tx = np.array([[-0.03, 0.002, 0.001], [0.03, -0.004, 0.0]])
    rows = np.array([[0, 1]], dtype=np.int32)
    for n in ((1, 1, 1), (1, 1, 41), (53, 1, 1), (1, 29, 3)):
        grid = wl.Grid(n[0], n[1], n[2], 1e-3, tuple(-0.5 * (np.array(n) - 1) * 1e-3))
        geo, og = _pair(fg, tx, rows, grid, [(1e6, 0.3e6, 3e-6)])
        m = np.random.default_rng(4).normal(size=og.V)
        ref = og.J(m)
        got = to_np(geo.J(to_dev(m)))
        assert abs(got[0] - ref[0]) <= 1e-5 * max(abs(ref[0]), 1e-30) + 1e-30
        d = np.array([1.0])
        assert rel_l2(to_np(geo.JT(to_dev(d))), og.JT(d)) <= 1e-5 or np.all(og.JT(d) == 0.0)


def test_psf_empty_subset_and_unreached_spike(fg):
    # one short pair near a corner of a larger grid: the far corner is outside its support
    tx = np.array([[-0.016, -0.016, 0.0], [-0.010, -0.016, 0.0], [-0.016, -0.010, 0.0]])
    rows = np.array([[0, 1], [0, 2], [1, 2]], dtype=np.int32)
    grid = wl.Grid.centred(20, 20, 4, 2e-3)
    geo, og = _pair(fg, tx, rows, grid, [(1e6, 0.3e6, 3e-6)])
    far = og.V - 1
    assert np.all(og.J(np.eye(1, og.V, far)[0]) == 0.0)
    near = int(np.argmin(np.linalg.norm(grid.centres() - np.array([-0.013, -0.015, 0.001]), axis=1)))
    spikes = np.array([near, far], dtype=np.int64)
    subsets = [np.zeros(0, dtype=np.int32), np.arange(og.M, dtype=np.int32)]
    ref = og.psf(spikes, subsets)
    assert np.linalg.norm(ref[1, 0]) > 0
    for mode in (0, 1):
        out = to_np(geo.psf_batch(spikes, subsets, mode=mode))
        assert np.all(out[0] == 0.0)                     # no rows: zero PSFs
        assert rel_l2(out[1, 0], ref[1, 0]) <= (1e-5 if mode == 0 else 1e-2)
        assert np.all(out[1, 1] == 0.0)                  # nothing reaches the far spike
