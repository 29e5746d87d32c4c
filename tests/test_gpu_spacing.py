"""Resolution against elevation spacing (Sec. III-C) on synthetic ring stacks: Hessian PSFs
H e_k = J^T J e_k with all rows, 128-element rings stacked at 3 mm (11 elevations) and 8 mm
(7 elevations). The vertical and horizontal profiles through the spike match the FP64
oracle (relative L2 <= 1e-5), and they show the paper's observation: with overlapping
sensitivities (3 mm) the response is stronger and its trade-offs (negative lobes) are much
smaller than with 8 mm spacing."""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_common import rel_l2, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_03302_gb300 as m
    m._lib.load()
    return m


def _profiles(fg, spacing, npos, x_mm):
    w = wl.elevation_stack(spacing, npos, n_tx=128)
    g = w.grid
    geo = fg.Geometry(w.tx, w.row_pairs(), g, w.c0, [fg.Table(1.0e6, 0.4e6, 4096, 3e-6)])
    ic, kc = (g.nx - 1) // 2, (g.nz - 1) // 2
    i = ic + int(round(x_mm * 1e-3 / g.h))
    v = (kc * g.ny + ic) * g.nx + i
    rows = np.arange(geo.M, dtype=np.int32)
    psf = to_np(geo.psf_batch([v], [rows], mode=0)).reshape(g.nz, g.ny, g.nx)
    vert_idx = np.array([(k * g.ny + ic) * g.nx + i for k in range(g.nz)])
    horz_idx = np.array([(kc * g.ny + ic) * g.nx + ii for ii in range(g.nx)])
    og = oracle.Geometry.from_workload(w)
    ref = og.psf(np.array([v]), [rows], np.concatenate([vert_idx, horz_idx]))[0, 0]
    vert, horz = psf[:, ic, i], psf[kc, ic, :]
    assert rel_l2(vert, ref[:g.nz]) <= 1e-5
    assert rel_l2(horz, ref[g.nz:]) <= 1e-5
    return vert, kc


@pytest.mark.parametrize("x_mm", [0, 40])
def test_overlapping_elevations_reduce_tradeoffs(fg, x_mm):
    v3, kc = _profiles(fg, 3e-3, 11, x_mm)
    v8, _ = _profiles(fg, 8e-3, 7, x_mm)
    assert v3[kc] > 2.0 * v8[kc]                      # more overlapping data: stronger response
    lobe3, lobe8 = -v3.min() / v3[kc], -v8.min() / v8[kc]
    assert lobe8 > 0.3 and lobe3 < 0.5 * lobe8        # oscillating trade-offs with 8 mm spacing
