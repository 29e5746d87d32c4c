"""Parity at the full size of the single-ring workload the benchmark times (256 elements on a
100 mm ring, 32640 pairs, 200 x 200 x 40 voxels at 1 mm, nested-cylinder model): J on
sampled rows and J^T on sampled voxels against the FP64 oracle (which computes those
outputs one by one), and properties of the 30-iteration CG that hold at any size: the
normal-equations residual it reports falls, the solution reduces the damped misfit
(CGLS minimises it over growing Krylov spaces), the graph replay is bit-reproducible and
the reconstruction correlates with the true model."""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_common import gpu_geometry, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ring256():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = wl.ring256()
    og = oracle.Geometry.from_workload(w)
    geo, tabs = gpu_geometry(w)
    return w, og, geo


def test_ring256_J_sampled_rows(ring256):
    w, og, geo = ring256
    m = wl.model_for(w)
    rows = np.sort(np.random.default_rng(41).choice(og.M, 256, replace=False)).astype(np.int64)
    d = to_np(geo.J(to_dev(m)))
    assert rel_l2(d[rows], og.J(m, rows)) <= 1e-5


def test_ring256_JT_sampled_voxels(ring256):
    w, og, geo = ring256
    rng = np.random.default_rng(42)
    dd = rng.normal(size=og.M) * 1e-8
    g = to_np(geo.JT(to_dev(dd)))
    for vox in (wl.random_voxels(w.grid, 256, 43, rho_max=0.095, z_max=0.019),
                np.sort(rng.choice(og.V, 512, replace=False)).astype(np.int64)):
        assert rel_l2(g[vox], og.JT(dd, vox)) <= 1e-5


def test_ring256_cg_properties(ring256):
    w, og, geo = ring256
    m_true = to_dev(wl.model_for(w))
    d = geo.J(m_true) + to_dev(wl.noise(og.M, w.noise_seed))
    m, hist = geo.cg_solve(d, w.lambda_rel, w.cg_iters, with_history=True)
    assert np.all(np.isfinite(hist)) and hist[-1] < 0.1 * hist[0]
    lam = w.lambda_rel * geo.frob2() / geo.V

    def damped(x):
        r = (geo.J(x) - d).double()
        return float(r.dot(r)) + lam * float(x.double().dot(x.double()))

    assert damped(m) < 0.5 * damped(torch.zeros_like(m))
    m2 = geo.cg_solve(d, w.lambda_rel, w.cg_iters)
    assert torch.equal(m, m2)
    c = float(torch.nn.functional.cosine_similarity(m.double(), m_true.double(), dim=0))
    assert c > 0.3
