"""Parity of the 2-D approximation (Sec. II-B, Eq. forward_2D: the kernel integrated over the
grid's z layers, acting on a plane map) with the FP64 oracle, through the C ABI:
relative L2 <= 1e-5 for J2 and J2^T (the FP32 sums of J and J^T plus a z sum)."""
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
def test_J2d_JT2d_match_oracle(fg, name):
    w, og = oracle_geometry(name)
    geo, _ = gpu_geometry(w)
    g = w.grid
    n2 = g.nx * g.ny
    assert geo.V2 == n2
    rng = np.random.default_rng(11)
    m2 = rng.normal(size=n2)
    assert rel_l2(to_np(geo.J2d(to_dev(m2))), og.J2d(m2)) <= 1e-5
    d = rng.normal(size=og.M)
    assert rel_l2(to_np(geo.JT2d(to_dev(d))), og.JT2d(d)) <= 1e-5
    # J2 is J of the extruded map, bit for bit (same kernels, same order)
    m3 = to_dev(np.tile(m2, g.nz))
    assert torch.equal(geo.J2d(to_dev(m2)), geo.J(m3))
    # J2^T is J^T summed over the layers
    gt = geo.JT(to_dev(d)).view(g.nz, n2).double().sum(0)
    assert rel_l2(to_np(geo.JT2d(to_dev(d))), to_np(gt)) <= 1e-6
