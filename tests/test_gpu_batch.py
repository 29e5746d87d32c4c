"""The four-column J / J^T kernels (fft_J_apply_batch, fft_JT_apply_batch) against the
single-vector calls, column by column, and against the FP64 oracle: 1e-6 relative L2 to the
single calls (same entries and summation order, different instruction schedules) and the
usual 1e-5 to the oracle, for 6 columns (a group of four and a remainder of two), on the
ring, on a three-band ragged grid with sharp bands, on a sine-series geometry and with a
transducer on a voxel centre."""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_common import gpu_geometry, oracle_geometry, rel_l2, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_03302_gb300 as m
    m._lib.load()
    return m


def _compare(geo, og, n=6, seed=0, check_oracle=True):
    rng = np.random.default_rng(seed)
    X = torch.as_tensor(rng.normal(size=(n, geo.V)), dtype=torch.float32, device="cuda")
    D = torch.as_tensor(rng.normal(size=(n, geo.M)), dtype=torch.float32, device="cuda")
    JX, JTD = geo.J_batch(X), geo.JT_batch(D)
    for c in range(n):
        assert rel_l2(to_np(JX[c]), to_np(geo.J(X[c].contiguous()))) <= 1e-6
        assert rel_l2(to_np(JTD[c]), to_np(geo.JT(D[c].contiguous()))) <= 1e-6
    if check_oracle:
        for c in (0, 3, 5):
            assert rel_l2(to_np(JX[c]), og.J(to_np(X[c]))) <= 1e-5
            assert rel_l2(to_np(JTD[c]), og.JT(to_np(D[c]))) <= 1e-5


def test_batch_ring32(fg):
    w, og = oracle_geometry("ring32")
    geo, _ = gpu_geometry(w)
    _compare(geo, og)
    # repeated calls are deterministic
    X = torch.randn((4, geo.V), device="cuda")
    assert torch.equal(geo.J_batch(X), geo.J_batch(X))


def test_batch_three_sharp_bands_ragged(fg):
    w = wl.tiny()
    M = len(w.row_pairs())
    bor = (np.arange(M) % 3).astype(np.int32)
    bands = [(0.6e6, 0.2e6, 5.0e-6), (1.0e6, 0.2e6, 3.0e-6), (1.4e6, 0.2e6, 3.0 / 1.4e6)]
    geo = fg.Geometry(w.tx, w.row_pairs(), w.grid, w.c0, [fg.Table(fc, fs, 4096, d) for fc, fs, d in bands],
                      band_of_row=bor)
    og = oracle.Geometry(w.tx, w.row_pairs(), bor, [oracle.phi_table_gauss(fc, fs, 4096, d) for fc, fs, d in bands],
                         [b[2] for b in bands], w.grid, w.c0)
    _compare(geo, og, seed=1)


def test_batch_series_and_guard(fg):
    w = wl.tiny()
    geo = fg.Geometry(w.tx, w.row_pairs(), w.grid, w.c0, [fg.TrigTable(1e6, 0.3e6, 3e-6)])
    a, dw = oracle.trig_coefs(1e6, 0.3e6, 3e-6)
    og = oracle.Geometry(w.tx, w.row_pairs(), None, [a], [3e-6], w.grid, w.c0, trig_dw=[dw])
    _compare(geo, og, seed=2)
    # a transducer exactly on a voxel centre (guarded kernels)
    g = w.grid
    tx = w.tx.copy()
    tx[0] = [g.origin[0] + 3 * g.h, g.origin[1] + 5 * g.h, g.origin[2] + 2 * g.h]
    geo = fg.Geometry(tx, w.row_pairs(), g, w.c0, [fg.Table(1e6, 0.3e6, 4096, 3e-6)])
    og = oracle.Geometry(tx, w.row_pairs(), None, [oracle.phi_table_gauss(1e6, 0.3e6, 4096, 3e-6)], [3e-6], g, w.c0)
    _compare(geo, og, seed=3)


def test_batch_naive_geometry_falls_back(fg):
    w, og = oracle_geometry("tiny")
    geo, _ = gpu_geometry(w, dt_mode=fg.FFT_DT_NAIVE)
    _compare(geo, og, n=5, check_oracle=False)
