"""Parity at the full size of the single-ring workload (256 elements on a 100 mm ring, 32640
pairs, 200 x 200 x 40 voxels at 1 mm, nested-cylinder model): J on sampled rows and J^T on
sampled voxels against the FP64 oracle (which computes those outputs one by one); the
30-iteration damped CGLS solve against the oracle's own solve of the same data, stored in
tests/golden/ring256_cgls30.npz by tests/golden/make_ring256_cgls.py (the oracle needs over
an hour for it); and properties of the solve that hold at any size: the normal-equations
residual it reports falls, the solution reduces the damped misfit (CGLS minimises it over
growing Krylov spaces), the graph replay is bit-reproducible and the reconstruction
correlates with the true model."""
import os

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


def test_ring256_cg_matches_stored_oracle_solve(ring256):
    # Sec. II-D, Eq. leastSquare_misfit: CGLS from m0 = 0 with relative damping 1e-3 on the
    # oracle's own data. On this acquisition the damped normal equations are ill-conditioned
    # enough that CG amplifies rounding: the FP32 iterates follow the FP64 ones to ~1e-5 for
    # the first seven iterations, after which perturbations of 1e-7 (the FP32 operator's
    # rounding, or of the data) grow to ~1e-2 in the model; two GPU solves that differ only in
    # the summation order of J^T differ by as much. Parity (relative L2 <= 1e-4 on the model,
    # the residual history within 1e-3) is therefore asserted after 6 iterations; the
    # 30-iteration solve is compared on its residual history up to there, and its model,
    # predicted data and damped misfit are reported with bounds that only catch gross errors.
    w, og, geo = ring256
    ref = np.load(os.path.join(os.path.dirname(__file__), "golden", "ring256_cgls30.npz"))
    assert geo.frob2() == pytest.approx(float(ref["frob2"]), rel=1e-5)
    d = to_dev(ref["d"])
    m6, hist6 = geo.cg_solve(d, w.lambda_rel, 6, with_history=True)
    err6 = rel_l2(to_np(m6), ref["m6"].astype(np.float64))
    m30, hist30 = geo.cg_solve(d, w.lambda_rel, w.cg_iters, with_history=True)
    lam = float(ref["lam"])
    jm = to_np(geo.J(m30))
    m30d = to_np(m30)
    f = 0.5 * np.sum((jm - ref["d"]) ** 2) + 0.5 * lam * np.sum(m30d ** 2)
    df = f / float(ref["f"]) - 1.0
    err_jm = rel_l2(jm, ref["Jm"])
    err30 = rel_l2(m30d, ref["m"].astype(np.float64))
    print(f"ring256 CG vs the stored FP64 oracle solves: model after 6 iterations {err6:.2e}; after 30: model "
          f"{err30:.2e}, predicted data {err_jm:.2e}, damped misfit {df:+.2e} (relative)")
    assert err6 <= 1e-4
    assert np.allclose(hist6, ref["hist6"], rtol=1e-3)
    assert np.allclose(hist30[:7], ref["hist"][:7], rtol=1e-3)
    assert err30 <= 0.1 and err_jm <= 0.05 and abs(df) <= 0.5
