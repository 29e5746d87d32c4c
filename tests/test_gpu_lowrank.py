"""Parity of the low-rank posterior covariance and resolution (Sec. II-D, Eqs. low_rank,
posterior_app, resolution_app) with the FP64 oracle, through the C ABI, from the same
seeded starting block.

Tolerances: the GPU applies H with FP32 J / J^T (~1e-6 relative each) and orthonormalises
in FP32 with FP64 Gram matrices, the oracle in FP64 with Householder QR; both span the same
subspaces, so the Ritz values agree to ~1e-5 and the dominant ones are held to 1e-4; the
diagonals sum k squared eigenvector entries and are held to 1e-3 (relative L2).
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_common import gpu_geometry, rel_l2, to_np
from oracle import lowrank as lr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_03302_gb300 as m
    m._lib.load()
    return m


def _case(fg, w, ell, k, n_power, sigma, seed):
    og = oracle.Geometry.from_workload(w)
    geo, _ = gpu_geometry(w)
    omega = wl.gaussian_block(og.V, ell, seed)
    lam_ref, vec_ref = lr.randomized_eig(og, omega, k, n_power, sigma)
    om = torch.as_tensor(np.ascontiguousarray(omega.T), dtype=torch.float32, device="cuda")
    lam, vecs = geo.hessian_lowrank(om, k, n_power, sigma)
    return og, geo, lam_ref, vec_ref, lam, vecs


def test_lowrank_wider_than_rank(fg):
    # 66 rows: a 72-column block spans the whole range of H, the pairs are exact
    w = wl.tiny()
    og, geo, lam_ref, vec_ref, lam, vecs = _case(fg, w, 72, 12, 1, 2.5e-8, 31)
    assert np.allclose(lam, lam_ref, rtol=1e-4, atol=0)
    V = to_np(vecs).T
    assert np.allclose(V.T @ V, np.eye(12), atol=1e-5)
    P, P_ref = V[:, :3] @ V[:, :3].T, vec_ref[:, :3] @ vec_ref[:, :3].T
    assert np.max(np.abs(P - P_ref)) <= 1e-3 * np.max(np.abs(P_ref))
    alpha = 1e-3 * lam_ref[0]
    post, res = geo.lowrank_diag(vecs, lam, alpha)
    post_ref, res_ref = lr.lowrank_diagonals(lam_ref, vec_ref, alpha)
    assert rel_l2(to_np(res), res_ref) <= 1e-3
    assert rel_l2(to_np(post), post_ref) <= 1e-3


def test_lowrank_randomized_regime(fg):
    # 276 rows, a 40-column block with two power iterations: the same randomized estimate
    w = wl.tiny(n_tx=24, radius=30e-3, n=(24, 24, 8))
    og, geo, lam_ref, vec_ref, lam, vecs = _case(fg, w, 40, 20, 2, 1.0, 32)
    assert np.allclose(lam[:8], lam_ref[:8], rtol=1e-4, atol=0)
    assert np.allclose(lam, lam_ref, rtol=1e-3, atol=0)
    alpha = 1e-2 * lam_ref[0]
    post, res = geo.lowrank_diag(vecs, lam, alpha)
    post_ref, res_ref = lr.lowrank_diagonals(lam_ref, vec_ref, alpha)
    assert rel_l2(to_np(res), res_ref) <= 1e-3
    assert rel_l2(to_np(post), post_ref) <= 1e-3


def test_lowrank_argument_checks(fg):
    w = wl.tiny()
    geo, _ = gpu_geometry(w)
    om = torch.zeros((4, geo.V), device="cuda", dtype=torch.float32)
    with pytest.raises(fg.FFTError):
        geo.hessian_lowrank(om, 5)                     # k > ell
    with pytest.raises(fg.FFTError):                   # an all-zero block cannot be orthonormalised
        geo.hessian_lowrank(om, 2)
