"""Parity on seeded random 3-D acquisitions, through the C ABI: transducers scattered in a
box (pairs not in one plane, some short), random ragged grids (1 to 37 voxels per axis,
random spacing and offset, so rows leave the grid and tiles are partial), 1 to 3 bands with
random spectra and cut-offs (some with Phi far from zero at the cut: the FP64 cut decision),
and one acquisition with a transducer exactly on a voxel centre (the guarded kernel).
J, J^T and the coverage against the FP64 oracle within 1e-5 (relative L2); the support
count within 1e-4; both Phi representations."""
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


def _acquisition(seed, on_voxel=False):
    rng = np.random.default_rng(seed)
    n_tx = int(rng.integers(6, 17))
    tx = np.stack([rng.uniform(-0.04, 0.04, n_tx), rng.uniform(-0.04, 0.04, n_tx),
                   rng.uniform(-0.015, 0.015, n_tx)], axis=1)
    n = [int(v) for v in rng.integers(1, 38, 3)]
    h = float(rng.uniform(0.7e-3, 2.5e-3))
    origin = tuple(float(v) for v in (-0.5 * (np.array(n) - 1) * h + rng.uniform(-5e-3, 5e-3, 3)))
    grid = wl.Grid(n[0], n[1], n[2], h, origin)
    if on_voxel:   # put transducer 0 exactly on the centre of voxel (i, j, k)
        i, j, k = (int(rng.integers(0, v)) for v in n)
        tx[0] = [origin[0] + i * h, origin[1] + j * h, origin[2] + k * h]
    pairs = wl.unordered_pairs(range(n_tx))
    nb = int(rng.integers(1, 4))
    bands = []
    for _ in range(nb):
        fc = float(rng.uniform(0.6e6, 1.5e6))
        bands.append((fc, float(rng.uniform(0.15e6, 0.45e6)), float(rng.uniform(2.0, 3.5)) / fc))
    bor = rng.integers(0, nb, len(pairs)).astype(np.int32)
    return tx, pairs, grid, bands, bor


def _check(fg, tx, pairs, grid, bands, bor, phi):
    if phi == "table":
        tabs = [fg.Table(fc, fs, 4096, dtm) for fc, fs, dtm in bands]
        og = oracle.Geometry(tx, pairs, bor, [oracle.phi_table_gauss(fc, fs, 4096, dtm) for fc, fs, dtm in bands],
                             [b[2] for b in bands], grid, 1500.0)
    else:
        tabs = [fg.TrigTable(fc, fs, dtm) for fc, fs, dtm in bands]
        series = [oracle.trig_coefs(fc, fs, dtm) for fc, fs, dtm in bands]
        og = oracle.Geometry(tx, pairs, bor, [a for a, _ in series], [b[2] for b in bands], grid, 1500.0,
                             trig_dw=[dw for _, dw in series])
    geo = fg.Geometry(tx, pairs, grid, 1500.0, tabs, band_of_row=bor)
    rng = np.random.default_rng(len(pairs))
    m = rng.normal(size=og.V)
    d = rng.normal(size=og.M)
    ref_J = og.J(m)
    if np.linalg.norm(ref_J) == 0.0:   # nothing of any row reaches the grid
        assert np.all(to_np(geo.J(to_dev(m))) == 0.0)
        return
    assert rel_l2(to_np(geo.J(to_dev(m))), ref_J) <= 1e-5
    assert rel_l2(to_np(geo.JT(to_dev(d))), og.JT(d)) <= 1e-5
    assert rel_l2(to_np(geo.coverage(device=torch.device("cuda"))), og.coverage()) <= 1e-5
    n_ref = og.count_support()
    assert abs(geo.support_evals - n_ref) <= 1e-4 * n_ref + 2


@pytest.mark.parametrize("seed", range(6))
def test_random_acquisitions_table(fg, seed):
    _check(fg, *_acquisition(100 + seed), "table")


@pytest.mark.parametrize("seed", range(2))
def test_random_acquisitions_series(fg, seed):
    _check(fg, *_acquisition(200 + seed), "trig")


def test_transducer_on_a_voxel_centre(fg):
    _check(fg, *_acquisition(300, on_voxel=True), "table")
