"""Pins for the oracle's 2-D approximation (Sec. II-B, Eq. forward_2D): the kernel integrated
over z by the midpoint rule on the grid's layers, acting on a plane map.

* the midpoint z rule agrees with an adaptive quadrature of the z integral of K0
  (scipy.integrate.quad on the oracle's own K0) once its layers resolve the Fresnel zones,
  in the first three zones;
* symmetry of the in-plane geometry: K0(z) = K0(-z);
* J2 = F E and J2^T = E^T F^T with the dense 3-D operator F (assembled column by column)
  and the extrusion E of a plane map along the layers.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

scipy_integrate = pytest.importorskip("scipy.integrate")

C0 = 1500.0


def test_midpoint_z_rule_converges():
    fc, fs = 1.0e6, 0.3e6
    dtm = 3.0 / fc
    tab = oracle.phi_table_gauss(fc, fs, 4096, dtm)
    xs, xr = np.array([-0.05, 0.0, 0.0]), np.array([0.05, 0.0, 0.0])
    L = 0.1
    zmax = np.sqrt(((L + C0 * dtm) / 2) ** 2 - (L / 2) ** 2) * 1.05   # beyond the truncated support
    for y in (0.4e-3, 1.5e-3, 3.0e-3):
        x = 0.01
        f = lambda z: oracle.k0(xs, xr, np.array([x, y, z]), C0, tab, dtm)
        ref, _ = scipy_integrate.quad(f, -zmax, zmax, limit=4000, epsabs=0, epsrel=1e-12, points=[0.0])
        err = lambda nz: abs(oracle.k2_midpoint(xs, xr, x, y, -zmax, 2 * zmax / nz, nz, C0, tab, dtm) - ref) / abs(ref)
        # the integrand is smooth and dies out at both ends: the midpoint rule is accurate once
        # the layers resolve the Fresnel zones (~1.4 mm here) and converges fast beyond that,
        # down to the table's interpolation level
        assert err(16) > 1e-3
        assert err(32) < 5e-6 and err(64) < 2e-6 and err(256) < 2e-6
        # in-plane symmetry: the half-range integral is half of the full one
        half = oracle.k2_midpoint(xs, xr, x, y, 0.0, zmax / 256, 256, C0, tab, dtm)
        full = oracle.k2_midpoint(xs, xr, x, y, -zmax, zmax / 256, 512, C0, tab, dtm)
        assert half == pytest.approx(0.5 * full, rel=1e-12)


def test_J2_is_the_dense_operator_times_extrusion():
    w = wl.tiny()
    og = oracle.Geometry.from_workload(w)
    g = w.grid
    F = og.dense()
    n2 = g.nx * g.ny
    E = np.tile(np.eye(n2), (g.nz, 1))             # (V, n2): voxel (k, j, i) <- pixel (j, i)
    rng = np.random.default_rng(8)
    m2 = rng.normal(size=n2)
    ref = F @ (E @ m2)
    assert np.max(np.abs(og.J2d(m2) - ref)) <= 1e-12 * np.max(np.abs(ref))
    d = rng.normal(size=og.M)
    refT = E.T @ (F.T @ d)
    assert np.max(np.abs(og.JT2d(d) - refT)) <= 1e-12 * np.max(np.abs(refT))
    pix = np.array([0, 7, n2 // 2, n2 - 1])
    assert np.allclose(og.JT2d(d, pix), og.JT2d(d)[pix], rtol=1e-13, atol=0)
    rows = np.array([1, 5, og.M - 1])
    assert np.allclose(og.J2d(m2, rows), og.J2d(m2)[rows], rtol=1e-13, atol=0)
