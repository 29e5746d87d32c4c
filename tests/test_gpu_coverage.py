"""Parity of the sensitivity coverage (Sec. III-A, sum_p |J[p, v] w_p|) with the FP64 oracle,
through the C ABI: relative L2 <= 1e-5 like J^T (the same gather, with |J|)."""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_common import gpu_geometry, oracle_geometry, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_03302_gb300 as m
    m._lib.load()
    return m


def test_coverage_ring32(fg):
    w, og = oracle_geometry("ring32")
    geo, _ = gpu_geometry(w)
    assert rel_l2(to_np(geo.coverage()), og.coverage()) <= 1e-5
    rng = np.random.default_rng(3)
    mask = (rng.random(og.M) < 0.3).astype(np.float64)      # a row subset
    assert rel_l2(to_np(geo.coverage(to_dev(mask))), og.coverage(mask)) <= 1e-5
    wt = rng.normal(size=og.M)                               # signed weights: |J w|
    assert rel_l2(to_np(geo.coverage(to_dev(wt))), og.coverage(wt)) <= 1e-5
    # deterministic
    assert torch.equal(geo.coverage(to_dev(wt)), geo.coverage(to_dev(wt)))


def test_coverage_three_bands_ragged_and_series(fg):
    w = wl.tiny()
    M = len(w.row_pairs())
    bor = (np.arange(M) % 3).astype(np.int32)
    bands = [(0.6e6, 0.2e6, 5.0e-6), (1.0e6, 0.2e6, 3.0e-6), (1.4e6, 0.2e6, 3.0 / 1.4e6)]
    tabs = [fg.Table(fc, fs, 4096, dtm) for fc, fs, dtm in bands]
    geo = fg.Geometry(w.tx, w.row_pairs(), w.grid, w.c0, tabs, band_of_row=bor)
    og = oracle.Geometry(w.tx, w.row_pairs(), bor, [oracle.phi_table_gauss(fc, fs, 4096, dtm) for fc, fs, dtm in bands],
                         [b[2] for b in bands], w.grid, w.c0)
    assert rel_l2(to_np(geo.coverage(device=torch.device("cuda"))), og.coverage()) <= 1e-5
    ttabs = [fg.TrigTable(fc, fs, dtm) for fc, fs, dtm in bands]
    geo_t = fg.Geometry(w.tx, w.row_pairs(), w.grid, w.c0, ttabs, band_of_row=bor)
    series = [oracle.trig_coefs(fc, fs, dtm) for fc, fs, dtm in bands]
    og_t = oracle.Geometry(w.tx, w.row_pairs(), bor, [a for a, _ in series], [b[2] for b in bands], w.grid, w.c0,
                           trig_dw=[dw for _, dw in series])
    assert rel_l2(to_np(geo_t.coverage(device=torch.device("cuda"))), og_t.coverage()) <= 1e-5
