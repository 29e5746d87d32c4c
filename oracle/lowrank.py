"""Low-rank posterior covariance and resolution (Sec. II-D, Eqs. low_rank, posterior_app,
resolution_app) in FP64 with numpy: TEST INFRASTRUCTURE ONLY (see the package docstring).

With Gamma_pr = I and Gamma_n^{-1} = I / sigma^2 (the reading of Sec. IV's noise model), the
prior-preconditioned misfit Hessian is H = J^T J / sigma^2. Its dominant eigenpairs come from
the randomized subspace iteration of Halko, Martinsson and Tropp (SIAM Review 53, 2011,
Algorithms 4.4 and 5.3), in the order the CUDA path takes them:

  Y = H Omega                      (Omega: V x ell, given)
  repeat n_power times:  Q = orth(Y),  Y = H Q
  Q = orth(Y);  T = Q^T (H Q);  T = U diag(lambda) U^T;  V_k = Q U[:, :k]   (largest first)

orth is numpy's QR (any orthonormal basis of the same span gives the same eigenpairs). Then
  diag(R)       ~ sum_i d_i v_i^2,               d_i = lambda_i / (lambda_i + alpha)
  diag(Gamma_post) ~ (1 - sum_i d_i v_i^2) / alpha
which are exact when k = N (the full spectrum).
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def hessian_apply(og, X: np.ndarray, sigma: float = 1.0) -> np.ndarray:
    """H X = J^T (J X) / sigma^2 for the columns of X (V x b), FP64 oracle J and J^T."""
    out = np.empty_like(X)
    for j in range(X.shape[1]):
        out[:, j] = og.JT(og.J(X[:, j])) / sigma ** 2
    return out


def randomized_eig(og, omega: np.ndarray, k: int, n_power: int, sigma: float = 1.0) -> Tuple[np.ndarray, np.ndarray]:
    """(lambda_1 >= ... >= lambda_k, V_k) of H by randomized subspace iteration from omega."""
    Y = hessian_apply(og, np.asarray(omega, dtype=np.float64), sigma)
    for _ in range(n_power):
        Q, _ = np.linalg.qr(Y)
        Y = hessian_apply(og, Q, sigma)
    Q, _ = np.linalg.qr(Y)
    T = Q.T @ hessian_apply(og, Q, sigma)
    T = 0.5 * (T + T.T)
    lam, U = np.linalg.eigh(T)
    order = np.argsort(lam)[::-1][:k]
    return lam[order], Q @ U[:, order]


def lowrank_diagonals(lam: np.ndarray, vecs: np.ndarray, alpha: float) -> Tuple[np.ndarray, np.ndarray]:
    """(diag Gamma_post, diag R) from k eigenpairs (Eqs. posterior_app, resolution_app)."""
    d = lam / (lam + alpha)
    s = (vecs ** 2) @ d
    return (1.0 - s) / alpha, s
