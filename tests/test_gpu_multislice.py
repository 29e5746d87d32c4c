"""A slice-by-slice acquisition of the slices3d kind at a size the FP64 oracle solves in
seconds: the 32-element ring stepped to 4 slices, the three bands of slices3d (the 1.4 MHz
band keeps a few per cent of Phi's peak at its cut-off, so the sharp-cut kernels run), 48 x 48
x 24 voxels at 2 mm. Against the oracle:

* the 20-iteration damped CGLS solve replayed from its CUDA graph (Sec. II-D, Eq.
  leastSquare_misfit): model within relative L2 1e-4, residual history within 1e-3;
* Hessian PSFs (Eq. resolution_2) for 6 spikes x 3 nested ring subsets (every 4th, every 2nd
  and every element of each ring, all slices and bands): the BF16 tensor-core path within
  relative L2 1e-2 per PSF, both FP32 paths (one PSF at a time, and four columns per J^T)
  within 1e-5.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_common import gpu_geometry, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def slices32():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = wl.slices32()
    geo, _ = gpu_geometry(w)
    return w, oracle.Geometry.from_workload(w), geo


def test_slices32_cg_matches_oracle(slices32):
    w, og, geo = slices32
    d = og.J(wl.model_for(w)) + wl.noise(og.M, w.noise_seed)
    m_ref, hist_ref, rc = og.cgls(d, og.lambda_abs(w.lambda_rel), w.cg_iters)
    assert rc == 0
    # the damping is relative to |J|_F^2, which each side computes on its own
    assert geo.frob2() == pytest.approx(og.frob2(), rel=1e-5)
    m, hist = geo.cg_solve(to_dev(d), w.lambda_rel, w.cg_iters, with_history=True)
    err = rel_l2(to_np(m), m_ref)
    print(f"slices32 CG(20) rel-L2 vs oracle {err:.2e}")
    assert err <= 1e-4
    assert np.allclose(hist, hist_ref, rtol=1e-3)
    assert torch.equal(geo.cg_solve(to_dev(d), w.lambda_rel, w.cg_iters), m)


def test_psf_sharp_three_band_all_modes(slices32):
    w, og, geo = slices32
    spikes = wl.random_voxels(w.grid, 6, 8, rho_max=0.035, z_max=0.01)
    subsets = wl.ring_subsets(n_tx=32, n_slices=4, n_bands=3)
    ref = og.psf(spikes, subsets)
    fp = to_np(geo.psf_batch(spikes, subsets, mode=0))
    fp4 = to_np(geo.psf_batch(spikes, subsets, mode=2))
    tc = to_np(geo.psf_batch(spikes, subsets, mode=1))
    errs = {"fp32": [], "fp32x4": [], "tc": []}
    for s in range(len(subsets)):
        for k in range(len(spikes)):
            assert np.linalg.norm(ref[s, k]) > 0
            errs["fp32"].append(rel_l2(fp[s, k], ref[s, k]))
            errs["fp32x4"].append(rel_l2(fp4[s, k], ref[s, k]))
            errs["tc"].append(rel_l2(tc[s, k], ref[s, k]))
    print("PSF rel-L2 vs oracle, max over 18:", {k: f"{max(v):.2e}" for k, v in errs.items()})
    assert max(errs["fp32"]) <= 1e-5
    assert abs(geo.support_evals - og.count_support()) <= 1e-4 * og.count_support()
    assert max(errs["fp32x4"]) <= 1e-5
    assert max(errs["tc"]) <= 1e-2
