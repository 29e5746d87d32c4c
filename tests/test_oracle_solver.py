"""Pins for the oracle's damped CGLS and Hessian PSFs (Sec. II-D, Eqs. leastSquare_misfit,
resolution_2) against dense linear algebra on a tiny problem.

* CGLS run to convergence equals numpy.linalg.solve(F^T F + lambda I, F^T d);
* a fixed number of CGLS iterations equals the same number of textbook CG iterations on
  the dense damped normal equations (the iterates agree in exact arithmetic);
* PSFs equal columns of F_S^T F_S for each row subset S;
* the relative damping lambda = lambda_rel |F|_F^2 / N equals the mean diagonal of F^T F.
"""
import numpy as np
import pytest

import oracle
import workloads as wl


@pytest.fixture(scope="module")
def tiny():
    w = wl.tiny()
    geo = oracle.Geometry.from_workload(w)
    F = geo.dense()
    return w, geo, F


def test_frobenius_and_lambda(tiny):
    w, geo, F = tiny
    assert geo.frob2() == pytest.approx(np.sum(F * F), rel=1e-12)
    lam = geo.lambda_abs(1e-3)
    assert lam == pytest.approx(1e-3 * np.mean(np.diag(F.T @ F)), rel=1e-12)


def test_cgls_converges_to_damped_solution(tiny):
    w, geo, F = tiny
    rng = np.random.default_rng(21)
    d = F @ rng.normal(size=geo.V) * 10 + rng.normal(scale=1e-9, size=geo.M)
    lam = geo.lambda_abs(0.1)
    ref = np.linalg.solve(F.T @ F + lam * np.eye(geo.V), F.T @ d)
    m, hist, rc = geo.cgls(d, lam, 400)
    assert rc == 0
    assert np.linalg.norm(m - ref) <= 1e-10 * np.linalg.norm(ref)
    assert hist[-1] < 1e-20 * hist[0]


def test_cgls_fixed_iterations_match_dense_cg(tiny):
    w, geo, F = tiny
    rng = np.random.default_rng(22)
    d = rng.normal(scale=1e-7, size=geo.M)
    lam = geo.lambda_abs(1e-3)
    A = F.T @ F + lam * np.eye(geo.V)
    b = F.T @ d
    x = np.zeros(geo.V)
    r = b.copy()
    p = r.copy()
    rs = r @ r
    for _ in range(10):
        Ap = A @ p
        al = rs / (p @ Ap)
        x += al * p
        r -= al * Ap
        rn = r @ r
        p = r + (rn / rs) * p
        rs = rn
    m, hist, rc = geo.cgls(d, lam, 10)
    assert rc == 0
    assert np.linalg.norm(m - x) <= 1e-8 * np.linalg.norm(x)
    assert hist[0] == pytest.approx(b @ b, rel=1e-12)


def test_cgls_zero_gradient_is_converged(tiny):
    # d = 0 and m0 = 0: the gradient of the damped misfit vanishes, m = 0 is its minimiser
    w, geo, F = tiny
    m, hist, rc = geo.cgls(np.zeros(geo.M), 0.0, 3)
    assert rc == 0
    assert np.all(m == 0.0) and np.all(hist == 0.0)
    # m0 = the damped solution itself: J^T (d - J m0) = lambda m0 up to rounding, so CGLS
    # stays within rounding of it
    rng = np.random.default_rng(23)
    d = F @ rng.normal(size=geo.V)
    lam = geo.lambda_abs(0.1)
    ref = np.linalg.solve(F.T @ F + lam * np.eye(geo.V), F.T @ d)
    m, hist, rc = geo.cgls(d, lam, 3, m0=ref)
    assert rc == 0
    assert np.linalg.norm(m - ref) <= 1e-10 * np.linalg.norm(ref)


def test_cgls_breakdown_status(tiny):
    # a curvature |J p|^2 + lambda |p|^2 <= 0 (damping far below -|J|^2) or a non-finite
    # datum is a breakdown
    w, geo, F = tiny
    rng = np.random.default_rng(24)
    d = F @ rng.normal(size=geo.V)
    m, hist, rc = geo.cgls(d, -1e3 * np.linalg.norm(F, 2) ** 2, 3)
    assert rc == -4
    d[5] = np.nan
    m, hist, rc = geo.cgls(d, 0.0, 3)
    assert rc == -4


def test_psf_dense(tiny):
    w, geo, F = tiny
    spikes = np.array([200, 611, 950], dtype=np.int64)
    subsets = [np.arange(0, geo.M, 3, dtype=np.int32), np.arange(geo.M, dtype=np.int32)]
    out = geo.psf(spikes, subsets)
    for s, S in enumerate(subsets):
        H = F[S].T @ F[S]
        for k, v in enumerate(spikes):
            ref = H[:, v]
            assert np.max(np.abs(out[s, k] - ref)) <= 1e-12 * np.max(np.abs(ref))
    vox = np.array([3, 200, 700], dtype=np.int64)
    part = geo.psf(spikes, subsets, vox)
    assert np.array_equal(part, out[:, :, vox])
