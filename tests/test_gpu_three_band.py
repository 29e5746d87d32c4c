"""Three bands of 4096 samples on one acquisition (measurements in several frequency bands,
Sec. VI): 96 KB of tables in shared memory (two 8-warp CTAs per SM), and a 1.4 MHz band whose
Phi does not vanish at its cut-off, so the sharp-cut kernels run. Parity of J, J^T, the
coverage, the support count and a CG solve with the FP64 oracle, bit-reproducibility, and the
operator the autotuner leaves behind."""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_common import gpu_geometry, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_03302_gb300 as m
    m._lib.load()
    return m


@pytest.fixture(scope="module")
def three_band(fg):
    base = wl.ring32()
    bands = [wl.Band(0.6e6, 0.2e6), wl.Band(1.0e6, 0.2e6), wl.Band(1.4e6, 0.2e6)]
    bor = np.repeat(np.arange(3, dtype=np.int32), len(base.pairs))
    w = wl.Workload("ring32x3", base.tx, base.pairs, bor, bands, base.grid, base.c0, cg_iters=6,
                    lambda_rel=1e-3, model_seed=1, noise_seed=2)
    geo, _ = gpu_geometry(w)
    return w, oracle.Geometry.from_workload(w), geo


def test_three_band_parity(three_band):
    w, og, geo = three_band
    m = wl.model_for(w)
    d = np.random.default_rng(8).normal(size=og.M) * 1e-8
    Jm = geo.J(to_dev(m))
    JTd = geo.JT(to_dev(d))
    assert rel_l2(to_np(Jm), og.J(m)) <= 1e-5
    assert rel_l2(to_np(JTd), og.JT(d)) <= 1e-5
    assert torch.equal(geo.J(to_dev(m)), Jm)
    assert torch.equal(geo.JT(to_dev(d)), JTd)
    assert rel_l2(to_np(geo.coverage()), og.coverage()) <= 1e-5
    assert abs(geo.support_evals - og.count_support()) <= 1e-4 * og.count_support()
    assert geo.frob2() == pytest.approx(og.frob2(), rel=1e-5)


def test_three_band_cg(three_band):
    w, og, geo = three_band
    d = og.J(wl.model_for(w)) + wl.noise(og.M, w.noise_seed)
    m_ref, _, rc = og.cgls(d, og.lambda_abs(w.lambda_rel), w.cg_iters)
    assert rc == 0
    m = geo.cg_solve(to_dev(d), w.lambda_rel, w.cg_iters)
    assert rel_l2(to_np(m), m_ref) <= 1e-4


def test_three_band_autotune(three_band):
    w, og, geo = three_band
    t = geo.autotune()
    assert t["ctas_per_sm"] in (1, 2)   # 96 KB of tables + staging: at most two CTAs per SM
    m = np.random.default_rng(9).normal(size=og.V)
    d = np.random.default_rng(10).normal(size=og.M)
    assert rel_l2(to_np(geo.J(to_dev(m))), og.J(m)) <= 1e-5
    assert rel_l2(to_np(geo.JT(to_dev(d))), og.JT(d)) <= 1e-5


def test_single_sharp_band(fg):
    # one 1.4 MHz band (sigma 0.2 MHz, Phi not zero at its cut-off): the sharp kernels with
    # one copy of a small table per SM
    base = wl.ring32()
    w = wl.Workload("ring32_sharp", base.tx, base.pairs, np.zeros(len(base.pairs), np.int32),
                    [wl.Band(1.4e6, 0.2e6)], base.grid, base.c0, cg_iters=6, lambda_rel=1e-3, model_seed=1,
                    noise_seed=2)
    og = oracle.Geometry.from_workload(w)
    geo, _ = gpu_geometry(w)
    m = wl.model_for(w)
    d = np.random.default_rng(11).normal(size=og.M) * 1e-8
    assert rel_l2(to_np(geo.J(to_dev(m))), og.J(m)) <= 1e-5
    assert rel_l2(to_np(geo.JT(to_dev(d))), og.JT(d)) <= 1e-5
    assert torch.equal(geo.JT(to_dev(d)), geo.JT(to_dev(d)))
    assert abs(geo.support_evals - og.count_support()) <= 1e-4 * og.count_support()
