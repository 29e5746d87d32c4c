"""Pins for the oracle's low-rank posterior covariance and resolution (Sec. II-D, Eqs.
low_rank, posterior_app, resolution_app):

* with k = N (every eigenpair) the low-rank formulas equal the dense definitions
  Gamma_post = (H + alpha I)^{-1} and R = (H + alpha I)^{-1} H (Eqs. posterior, resolution);
* the randomized subspace iteration recovers the dominant eigenpairs of the dense Hessian
  F^T F / sigma^2 (numpy eigh) on a tiny ring: exactly (1e-10) when the block is wider than
  the rank, and converging with the power iterations when it is narrower;
* its diagonals from k < N eigenpairs approach the dense ones as k grows (the truncation
  the paper applies) and bound them: diag R from k pairs never exceeds the exact one.
"""
import numpy as np

import oracle
import workloads as wl
from oracle import lowrank as lr


def _tiny():
    w = wl.tiny()
    og = oracle.Geometry.from_workload(w)
    F = og.dense()
    return w, og, F


def test_full_rank_formulas_are_exact():
    w, og, F = _tiny()
    sigma = 2.5e-8
    H = F.T @ F / sigma ** 2
    lam, U = np.linalg.eigh(H)
    alpha = 1e-3 * np.trace(H) / H.shape[0]
    post, res = lr.lowrank_diagonals(lam, U, alpha)
    A = H + alpha * np.eye(H.shape[0])
    post_ref = np.diag(np.linalg.inv(A))
    res_ref = np.diag(np.linalg.solve(A, H))
    assert np.max(np.abs(post - post_ref)) <= 1e-8 * np.max(np.abs(post_ref))
    assert np.max(np.abs(res - res_ref)) <= 1e-8


def test_randomized_iteration_recovers_dominant_eigenpairs():
    w, og, F = _tiny()
    sigma = 2.5e-8
    H = F.T @ F / sigma ** 2
    lam_ref, U_ref = np.linalg.eigh(H)
    lam_ref, U_ref = lam_ref[::-1], U_ref[:, ::-1]
    rank = og.M                                  # H = F^T F has rank <= M (66 rows)
    # a block wider than the rank spans the whole range of H: exact up to rounding
    omega = wl.gaussian_block(og.V, rank + 6, seed=21)
    lam, vecs = lr.randomized_eig(og, omega, k=12, n_power=1, sigma=sigma)
    assert np.allclose(lam, lam_ref[:12], rtol=1e-10, atol=0)
    # eigenvectors: the spectral projector of the leading cluster (0.645 is a double eigenvalue)
    P, P_ref = vecs[:, :3] @ vecs[:, :3].T, U_ref[:, :3] @ U_ref[:, :3].T
    assert np.max(np.abs(P - P_ref)) < 1e-9 * np.max(np.abs(P_ref))
    assert abs(abs(vecs[:, 0] @ U_ref[:, 0]) - 1.0) < 1e-10
    assert np.allclose(vecs.T @ vecs, np.eye(12), atol=1e-12)
    # a narrower block converges with the power iterations (flat spectrum: slowly)
    omega = wl.gaussian_block(og.V, 24, seed=22)
    errs = [abs(lr.randomized_eig(og, omega, k=1, n_power=q, sigma=sigma)[0][0] - lam_ref[0]) / lam_ref[0]
            for q in (0, 2, 4)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-5, errs


def test_truncated_diagonals_approach_the_dense_ones():
    w, og, F = _tiny()
    H = F.T @ F
    lam, U = np.linalg.eigh(H)
    lam, U = lam[::-1], U[:, ::-1]
    alpha = 1e-3 * np.trace(H) / H.shape[0]
    _, res_ref = lr.lowrank_diagonals(lam, U, alpha)
    prev = None
    for k in (4, 16, 32, 64):
        _, res = lr.lowrank_diagonals(lam[:k], U[:, :k], alpha)
        assert np.all(res <= res_ref + 1e-9 * np.max(res_ref))
        err = np.linalg.norm(res - res_ref)
        if prev is not None:
            assert err <= prev + 1e-15
        prev = err
