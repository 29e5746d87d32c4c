"""Batched Hessian PSFs on the tensor cores (BF16 operands, FP32 accumulation in TMEM)
against the FP64 oracle (relative L2 <= 1e-2 per PSF) and against the FP32 CUDA-core path:
nested ring subsets (one row group per subset, PSFs as prefix sums of the groups), overlapping
subsets that are not nested (a row group per combination of subsets), more subset
combinations than one launch takes (subsets one at a time), and more spikes than one launch
takes (spike blocks)."""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_common import gpu_geometry, oracle_geometry, rel_l2, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def ring_subsets32(M_pairs):
    local = wl.unordered_pairs(range(32))
    out = []
    for st in (4, 2, 1):
        out.append(np.flatnonzero((local[:, 0] % st == 0) & (local[:, 1] % st == 0)).astype(np.int32))
    return out


@pytest.fixture(scope="module")
def ring32():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w, og = oracle_geometry("ring32")
    geo, tabs = gpu_geometry(w)
    return w, og, geo


def test_psf_tc_matches_oracle(ring32):
    w, og, geo = ring32
    spikes = wl.random_voxels(w.grid, 6, 8, rho_max=0.035, z_max=0.012)
    subsets = ring_subsets32(og.M)
    ref = og.psf(spikes, subsets)
    tc = to_np(geo.psf_batch(spikes, subsets, mode=1))
    fp = to_np(geo.psf_batch(spikes, subsets, mode=0))
    for s in range(len(subsets)):
        for k in range(len(spikes)):
            assert rel_l2(fp[s, k], ref[s, k]) <= 1e-5
            assert rel_l2(tc[s, k], ref[s, k]) <= 1e-2


@pytest.mark.parametrize("n_spike", [100, 200])
def test_psf_tc_many_rhs(ring32, n_spike):
    # 3 nested subsets x 100 spikes: one launch (3 row groups x 112 accumulator columns);
    # 3 x 200: two spike blocks
    w, og, geo = ring32
    spikes = wl.random_voxels(w.grid, n_spike, 9, rho_max=0.04, z_max=0.014)
    subsets = ring_subsets32(og.M)
    tc = to_np(geo.psf_batch(spikes, subsets, mode=1))
    fp = to_np(geo.psf_batch(spikes, subsets, mode=0))
    errs = [rel_l2(tc[s, k], fp[s, k]) for s in range(3) for k in range(n_spike)
            if np.linalg.norm(fp[s, k]) > 0]
    assert len(errs) > 0 and max(errs) <= 1e-2


def test_psf_tc_ragged_tiny(fg_tiny=None):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w, og = oracle_geometry("tiny")
    geo, _ = gpu_geometry(w)
    spikes = np.array([200, 611, 950], dtype=np.int64)
    subsets = [np.arange(0, og.M, 3, dtype=np.int32), np.arange(og.M, dtype=np.int32)]
    ref = og.psf(spikes, subsets)
    tc = to_np(geo.psf_batch(spikes, subsets, mode=1))
    for s in range(2):
        for k in range(3):
            assert rel_l2(tc[s, k], ref[s, k]) <= 1e-2


def test_psf_tc_transducer_on_a_voxel_centre():
    # the guarded tensor-core kernel: a transducer exactly on a voxel centre of a ragged grid
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_03302_gb300 as fg
    w = wl.tiny()
    g = w.grid
    tx = w.tx.copy()
    tx[0] = [g.origin[0] + 3 * g.h, g.origin[1] + 5 * g.h, g.origin[2] + 2 * g.h]
    geo = fg.Geometry(tx, w.row_pairs(), g, w.c0, [fg.Table(1e6, 0.3e6, 4096, 3e-6)])
    og = oracle.Geometry(tx, w.row_pairs(), None, [oracle.phi_table_gauss(1e6, 0.3e6, 4096, 3e-6)], [3e-6], g, w.c0)
    spikes = np.array([(2 * g.ny + 5) * g.nx + 4, 611, 950], dtype=np.int64)   # one next to the transducer
    subsets = [np.arange(0, og.M, 2, dtype=np.int32), np.arange(og.M, dtype=np.int32)]
    ref = og.psf(spikes, subsets)
    tc = to_np(geo.psf_batch(spikes, subsets, mode=1))
    fp = to_np(geo.psf_batch(spikes, subsets, mode=0))
    for s in range(2):
        for k in range(3):
            assert rel_l2(fp[s, k], ref[s, k]) <= 1e-5
            assert rel_l2(tc[s, k], ref[s, k]) <= 1e-2


def test_psf_tc_overlapping_subsets(ring32):
    # two overlapping subsets, neither inside the other: rows of the first only, of the second
    # only and of both form three groups; each PSF sums the two groups of its subset
    w, og, geo = ring32
    local = wl.unordered_pairs(range(32))
    even = np.flatnonzero((local[:, 0] % 2 == 0) & (local[:, 1] % 2 == 0)).astype(np.int32)
    low = np.flatnonzero(local[:, 1] < 20).astype(np.int32)
    assert 0 < len(np.intersect1d(even, low)) < min(len(even), len(low))
    spikes = wl.random_voxels(w.grid, 5, 21, rho_max=0.035, z_max=0.012)
    subsets = [even, low]
    ref = og.psf(spikes, subsets)
    tc = to_np(geo.psf_batch(spikes, subsets, mode=1))
    for s in range(2):
        for k in range(len(spikes)):
            assert rel_l2(tc[s, k], ref[s, k]) <= 1e-2


def test_psf_tc_many_subset_combinations(ring32):
    # six random halves of the rows: up to 63 distinct combinations, more than one launch
    # groups, so the subsets are taken one at a time
    w, og, geo = ring32
    rng = np.random.default_rng(22)
    subsets = [np.flatnonzero(rng.random(og.M) < 0.5).astype(np.int32) for _ in range(6)]
    member = np.zeros(og.M, dtype=np.int64)
    for s, rows in enumerate(subsets):
        member[rows] |= 1 << s
    assert len(np.unique(member[member > 0])) > 32
    spikes = wl.random_voxels(w.grid, 4, 23, rho_max=0.035, z_max=0.012)
    tc = to_np(geo.psf_batch(spikes, subsets, mode=1))
    fp = to_np(geo.psf_batch(spikes, subsets, mode=0))
    for s in range(len(subsets)):
        for k in range(len(spikes)):
            assert rel_l2(tc[s, k], fp[s, k]) <= 1e-2


def test_psf_tc_many_nested_groups(ring32):
    # eight nested subsets (rows whose two elements lie in the first 4, 8, ..., 32 elements of
    # a seeded order): eight row groups of at most 64 accumulator columns each (512 / 8), so
    # 100 spikes run in two launches (64 + 36), and each PSF sums up to eight groups
    w, og, geo = ring32
    local = wl.unordered_pairs(range(32))
    order = np.random.default_rng(24).permutation(32)
    rank = np.empty(32, dtype=np.int64)
    rank[order] = np.arange(32)
    top = np.maximum(rank[local[:, 0]], rank[local[:, 1]])
    subsets = [np.flatnonzero(top < n).astype(np.int32) for n in range(4, 33, 4)]
    spikes = wl.random_voxels(w.grid, 100, 25, rho_max=0.035, z_max=0.012)
    tc = to_np(geo.psf_batch(spikes, subsets, mode=1))
    fp = to_np(geo.psf_batch(spikes, subsets, mode=0))
    checked = 0
    for s in range(len(subsets)):
        for k in range(len(spikes)):
            if np.linalg.norm(fp[s, k]) > 0:
                assert rel_l2(tc[s, k], fp[s, k]) <= 1e-2
                checked += 1
    assert checked > len(spikes)


def test_psf_tc_bitwise_repeatable(ring32):
    # the K order of every MMA chain is fixed (groups in order, candidates in order), so two
    # calls give the same bits
    w, og, geo = ring32
    spikes = wl.random_voxels(w.grid, 24, 26, rho_max=0.035, z_max=0.012)
    subsets = ring_subsets32(og.M)
    a = geo.psf_batch(spikes, subsets, mode=1).cpu().numpy()
    b = geo.psf_batch(spikes, subsets, mode=1).cpu().numpy()
    assert np.linalg.norm(a) > 0
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_psf_tc_rejects_a_row_listed_twice(ring32):
    import paper_1908_03302_gb300 as fg
    w, og, geo = ring32
    rows = np.arange(0, og.M, 3, dtype=np.int32)
    bad = np.sort(np.concatenate([rows, rows[5:6]])).astype(np.int32)
    spikes = wl.random_voxels(w.grid, 2, 27, rho_max=0.035, z_max=0.012)
    with pytest.raises(fg.FFTError) as ei:
        geo.psf_batch(spikes, [rows, bad], mode=1)
    assert ei.value.status == fg._lib.FFT_ERR_ARG
