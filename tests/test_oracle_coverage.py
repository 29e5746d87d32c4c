"""Pins for the oracle's sensitivity coverage (Sec. III-A: the absolute values of the
operator's entries summed over the rows, per voxel).

* against the dense operator: cov = |F|^T |w| (the dense F is assembled column by column
  through J, a different loop than the coverage's per-voxel gather);
* additivity over disjoint row masks and the triangle inequality cov >= |J^T w|;
* the ring's symmetry: a 32-element ring on a centred square grid is invariant under a
  quarter turn, and so is its coverage (to rounding);
* the paper's observation for ring arrays: coverage is lower at the centre than towards the
  ring.
"""
import numpy as np

import oracle
import workloads as wl


def test_coverage_matches_dense_operator():
    w = wl.tiny()
    og = oracle.Geometry.from_workload(w)
    F = og.dense()
    cov = og.coverage()
    ref = np.abs(F).sum(axis=0)
    assert np.max(np.abs(cov - ref)) <= 1e-12 * np.max(ref)
    wt = np.random.default_rng(1).normal(size=og.M)
    assert np.allclose(og.coverage(wt), np.abs(F).T @ np.abs(wt), rtol=1e-12, atol=1e-12 * np.max(ref))
    vox = np.array([0, 5, og.V // 2, og.V - 1])
    assert np.array_equal(og.coverage(wt, vox), og.coverage(wt)[vox])


def test_coverage_additive_and_bounds_the_adjoint():
    w = wl.ring32()
    og = oracle.Geometry.from_workload(w)
    rng = np.random.default_rng(4)
    m1 = (rng.random(og.M) < 0.5).astype(float)
    m2 = 1.0 - m1
    vox = np.arange(0, og.V, 37)
    c1, c2, c = og.coverage(m1, vox), og.coverage(m2, vox), og.coverage(None, vox)
    assert np.allclose(c1 + c2, c, rtol=1e-12, atol=0)
    d = rng.normal(size=og.M)
    assert np.all(og.coverage(d, vox) >= np.abs(og.JT(d, vox)) * (1 - 1e-12))


def test_coverage_ring_symmetry_and_centre():
    w = wl.ring32()
    og = oracle.Geometry.from_workload(w)
    g = w.grid
    k = g.nz // 2
    idx = lambda i, j: (k * g.ny + j) * g.nx + i
    ii, jj = np.meshgrid(np.arange(g.nx), np.arange(g.ny), indexing="ij")
    # a quarter turn about the ring centre maps (i, j) -> (n-1-j, i) on the centred grid
    a = np.array([idx(i, j) for i, j in zip(ii.ravel(), jj.ravel())])
    b = np.array([idx(g.nx - 1 - j, i) for i, j in zip(ii.ravel(), jj.ravel())])
    ca, cb = og.coverage(None, a), og.coverage(None, b)
    assert np.max(np.abs(ca - cb)) <= 1e-9 * np.max(ca)
    # lower at the centre than at 60 % of the ring radius
    c = g.nx // 2
    centre = og.coverage(None, np.array([idx(c, c)]))[0]
    r = int(round(0.6 * 50e-3 / g.h))
    mid = og.coverage(None, np.array([idx(c + r, c)]))[0]
    assert centre < mid
