"""The stored expected results under tests/golden/ belong to the seeded workloads they claim
to: each file's inputs are recomputed here from `workloads` and the FP64 oracle on a sample
(no GPU), so a stale or mislabelled file fails before any GPU test compares against it."""
import os

import numpy as np
import pytest

import oracle
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_ring256_cgls_golden_inputs():
    ref = np.load(os.path.join(GOLDEN, "ring256_cgls30.npz"))
    w = wl.ring256()
    og = oracle.Geometry.from_workload(w)
    assert ref["d"].shape == (og.M,) and ref["m"].shape == (og.V,) and ref["hist"].shape == (w.cg_iters + 1,)
    # the data: oracle J of the nested-cylinder model plus the seeded noise, on sampled rows
    rows = np.sort(np.random.default_rng(77).choice(og.M, 48, replace=False)).astype(np.int64)
    d = og.J(wl.model_for(w), rows) + wl.noise(og.M, w.noise_seed)[rows]
    assert np.allclose(ref["d"][rows], d, rtol=1e-12, atol=0.0)
    # the damping is the relative one of the workload
    assert float(ref["lam"]) == pytest.approx(w.lambda_rel * float(ref["frob2"]) / og.V, rel=1e-14)
    # the stored solve made progress: the normal-equations residual fell by orders of magnitude
    assert ref["hist"][-1] < 1e-2 * ref["hist"][0]
    assert np.all(np.isfinite(ref["m"])) and np.linalg.norm(ref["m"]) > 0
