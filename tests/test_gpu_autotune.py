"""The work-decomposition autotuner (fft_geom_autotune): it times up to nine of twelve
candidates, keeps one of them, and the operator it leaves behind still matches the FP64 oracle (J bit for bit as
before: its per-row sums do not depend on the items; J^T within rounding), including a CG
solve whose captured loop the tuner invalidates."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("name", ["ring32", "tiny"])
def test_autotune_keeps_the_operator(fg, name):
    w, og = oracle_geometry(name)
    geo, _ = gpu_geometry(w)
    m = to_dev(wl.model_for(w) if name == "ring32" else np.random.default_rng(1).normal(size=og.V))
    d = to_dev(np.random.default_rng(2).normal(size=og.M) * 1e-8)
    J0, JT0 = geo.J(m), geo.JT(d)
    if name == "ring32":   # a captured CG loop before tuning
        m_cg0 = geo.cg_solve(J0, w.lambda_rel, 5)
    t = geo.autotune()
    assert 2 <= t["candidates"] <= 9
    assert t["items_per_cta"] in (4, 8, 16, 32, 64, 128) and t["ctas_per_sm"] >= 1
    assert t["ms_J"] > 0 and t["ms_JT"] > 0
    assert torch.equal(geo.J(m), J0)
    assert rel_l2(to_np(geo.JT(d)), to_np(JT0)) <= 1e-6
    assert rel_l2(to_np(geo.J(m)), og.J(to_np(m))) <= 1e-5
    assert rel_l2(to_np(geo.JT(d)), og.JT(to_np(d))) <= 1e-5
    if name == "ring32":
        m_cg1 = geo.cg_solve(J0, w.lambda_rel, 5)
        assert rel_l2(to_np(m_cg1), to_np(m_cg0)) <= 1e-5
