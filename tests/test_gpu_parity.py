"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

Tolerances (relative L2 against the oracle, FP32 kernels): J and J^T <= 1e-5; CG model
after the fixed iterations <= 1e-4; dot-product test <= 1e-6. The 32-element ring
(48 x 48 x 16 voxels) spans several tiles with a ragged z edge; the 12-element tiny ring has
a grid that is not a multiple of the tile in any axis.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_common import gpu_geometry, oracle_geometry, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_03302_gb300 as m
    m._lib.load()
    return m


@pytest.fixture(scope="module")
def ring32(fg):
    w, og = oracle_geometry("ring32")
    geo, tabs = gpu_geometry(w)
    return w, og, geo


def test_table_matches_oracle(fg):
    for fc, fs in [(1e6, 0.3e6), (1e6, 0.4e6), (0.6e6, 0.2e6), (1.4e6, 0.2e6)]:
        t = fg.Table(fc, fs, 4096, 3.0 / fc, keep_host=True)
        ref = oracle.phi_table_gauss(fc, fs, 4096, 3.0 / fc)
        assert np.max(np.abs(t.host - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_sampled_table_matches_oracle(fg):
    w0, s = 2 * math.pi * 1e6, 2 * math.pi * 0.3e6
    om = np.linspace(0, w0 + 12 * s, 6001)
    W = np.exp(-0.5 * ((om - w0) / s) ** 2) * (1 + 0.3 * np.sin(om / w0))
    t = fg.Table(omega=om, weight=W, n=1024, dt_max=3e-6, keep_host=True)
    ref = oracle.phi_table_sampled(om, W, 1024, 3e-6)
    assert np.max(np.abs(t.host - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_J_and_JT_ring32(ring32):
    w, og, geo = ring32
    m = wl.model_for(w)
    d_ref = og.J(m)
    d = to_np(geo.J(to_dev(m)))
    assert rel_l2(d, d_ref) <= 1e-5
    rng = np.random.default_rng(7)
    dd = rng.normal(size=og.M) * 1e-8
    g_ref = og.JT(dd)
    g = to_np(geo.JT(to_dev(dd)))
    assert rel_l2(g, g_ref) <= 1e-5


def test_support_count(ring32):
    w, og, geo = ring32
    n_ref = og.count_support()
    assert abs(geo.support_evals - n_ref) <= 1e-4 * n_ref


def test_tiny_ragged_grid_and_dense_matrix(fg):
    w, og = oracle_geometry("tiny")
    geo, _ = gpu_geometry(w)
    F = og.dense()
    rng = np.random.default_rng(3)
    m = rng.normal(size=og.V)
    d = rng.normal(size=og.M)
    assert rel_l2(to_np(geo.J(to_dev(m))), F @ m) <= 1e-5
    assert rel_l2(to_np(geo.JT(to_dev(d))), F.T @ d) <= 1e-5
    # single columns and rows of J through unit vectors
    for v in (0, 137, og.V - 1):
        e = np.zeros(og.V)
        e[v] = 1.0
        col = to_np(geo.J(to_dev(e)))
        assert np.max(np.abs(col - F[:, v])) <= 1e-5 * np.max(np.abs(F))


def test_dot_product_and_determinism(ring32):
    # <J m, d> = <m, J^T d> over 16 seeded (m, d) pairs
    w, og, geo = ring32
    rng = np.random.default_rng(5)
    rel = []
    for _ in range(16):
        m = to_dev(rng.normal(size=og.V))
        d = to_dev(rng.normal(size=og.M) * 1e-8)
        Jm = geo.J(m)
        JTd = geo.JT(d)
        lhs = float(torch.dot(Jm.double(), d.double()))
        rhs = float(torch.dot(m.double(), JTd.double()))
        rel.append(abs(lhs - rhs) / float(Jm.double().norm() * d.double().norm()))
        assert rel[-1] <= 1e-6
        assert torch.equal(geo.J(m), Jm)
        assert torch.equal(geo.JT(d), JTd)
    print(f"dot-product test over 16 pairs: |<Jm,d> - <m,J^T d>| / (|Jm||d|) max {max(rel):.2e}, "
          f"median {np.median(rel):.2e}")


def test_dt_modes(fg, ring32):
    w, og, _ = ring32
    m = wl.model_for(w)
    d_ref = og.J(m)
    errs = {}
    for mode in (fg.FFT_DT_STABLE, fg.FFT_DT_NAIVE, fg.FFT_DT_FP64):
        geo, _ = gpu_geometry(w, dt_mode=mode)
        errs[mode] = rel_l2(to_np(geo.J(to_dev(m))), d_ref)
    print("J m rel-L2 vs the FP64 oracle by detour mode: "
          f"FP64 {errs[fg.FFT_DT_FP64]:.2e}, stable FP32 {errs[fg.FFT_DT_STABLE]:.2e}, "
          f"naive FP32 {errs[fg.FFT_DT_NAIVE]:.2e}")
    assert errs[fg.FFT_DT_FP64] <= 1e-6
    assert errs[fg.FFT_DT_STABLE] <= 1e-5
    assert errs[fg.FFT_DT_NAIVE] <= 1e-3


def test_cg_matches_oracle(ring32):
    w, og, geo = ring32
    m_true = wl.model_for(w)
    d = og.J(m_true) + wl.noise(og.M, w.noise_seed)
    lam = og.lambda_abs(w.lambda_rel)
    m_ref, hist_ref, rc = og.cgls(d, lam, w.cg_iters)
    assert rc == 0
    assert geo.frob2() == pytest.approx(og.frob2(), rel=1e-5)
    m, hist = geo.cg_solve(to_dev(d), w.lambda_rel, w.cg_iters, with_history=True)
    err = rel_l2(to_np(m), m_ref)
    print(f"ring32 CG(10) rel-L2 vs oracle {err:.2e}")
    assert err <= 1e-4
    assert np.allclose(hist, hist_ref, rtol=1e-3)
    # the same call again reuses the captured graph and reproduces the result bit for bit
    m2 = geo.cg_solve(to_dev(d), w.lambda_rel, w.cg_iters)
    assert torch.equal(m, m2)


def test_cg_breakdown_status(fg, ring32):
    # a non-finite datum makes gamma non-finite: a breakdown, reported by the synchronous call
    # with a history and by fft_cg_status after the asynchronous one
    w, og, geo = ring32
    d = torch.zeros(og.M, device="cuda")
    d[17] = float("nan")
    with pytest.raises(fg.FFTError) as ei:
        geo.cg_solve(d, 1e-3, 3)
    assert ei.value.status == fg._lib.FFT_ERR_BREAKDOWN
    with pytest.raises(fg.FFTError) as ei:
        geo.cg_solve(d, 1e-3, 3, with_history=True)
    assert ei.value.status == fg._lib.FFT_ERR_BREAKDOWN
    geo.cg_solve(d, 1e-3, 3, check_status=False)
    with pytest.raises(fg.FFTError) as ei:
        geo.cg_status()
    assert ei.value.status == fg._lib.FFT_ERR_BREAKDOWN


def test_cg_zero_data_is_converged(fg, ring32):
    # d = 0, m0 = 0: the gradient of the damped misfit vanishes; m = 0 is the minimiser and the
    # solve reports success (the oracle does the same)
    w, og, geo = ring32
    m_ref, hist_ref, rc = og.cgls(np.zeros(og.M), og.lambda_abs(w.lambda_rel), 3)
    assert rc == 0 and np.all(m_ref == 0.0)
    m, hist = geo.cg_solve(torch.zeros(og.M, device="cuda"), w.lambda_rel, 3, with_history=True)
    assert torch.count_nonzero(m) == 0
    assert np.all(hist == 0.0)
    geo.cg_status()


def test_cg_asynchronous_call(fg, ring32):
    # without a history the call only enqueues the solve; fft_cg_status waits and reports it
    w, og, geo = ring32
    d = to_dev(og.J(wl.model_for(w)) + wl.noise(og.M, w.noise_seed))
    m_sync = geo.cg_solve(d, w.lambda_rel, w.cg_iters)
    m_async = geo.cg_solve(d, w.lambda_rel, w.cg_iters, check_status=False)
    geo.cg_status()
    assert torch.equal(m_sync, m_async)


def test_autograd_gradient(fg, ring32):
    w, og, geo = ring32
    rng = np.random.default_rng(4)
    m0 = wl.model_for(w)
    dobs = og.J(m0) + wl.noise(og.M, 2)
    m = to_dev(m0 * 0.5).requires_grad_(True)
    dT = fg.jacobian_apply(m, geo)
    loss = 0.5 * ((dT.double() - torch.as_tensor(dobs, device="cuda")) ** 2).sum()
    loss.backward()
    r = og.J(m0 * 0.5) - dobs
    g_ref = og.JT(r)
    err_jt = rel_l2(to_np(m.grad), g_ref)
    assert err_jt <= 1e-5
    # central finite differences of the FP64 oracle misfit on 64 voxels agree with autograd
    vox = rng.choice(og.V, 64, replace=False)
    fd = []
    for v in vox:
        e = np.zeros(og.V)
        e[v] = 1e-3
        fp = 0.5 * np.sum((og.J(m0 * 0.5 + e) - dobs) ** 2)
        fm = 0.5 * np.sum((og.J(m0 * 0.5 - e) - dobs) ** 2)
        fd.append((fp - fm) / 2e-3)
    err_fd = rel_l2(to_np(m.grad)[vox], np.array(fd))
    print(f"autograd gradient rel-L2: vs oracle J^T {err_jt:.2e}, vs central FD on 64 voxels {err_fd:.2e}")
    assert err_fd <= 1e-3


def test_psf_matches_oracle(fg):
    w, og = oracle_geometry("tiny")
    geo, _ = gpu_geometry(w)
    spikes = np.array([200, 611, 950], dtype=np.int64)
    subsets = [np.arange(0, og.M, 3, dtype=np.int32), np.arange(og.M, dtype=np.int32)]
    ref = og.psf(spikes, subsets)
    out = to_np(geo.psf_batch(spikes, subsets))
    for s in range(2):
        for k in range(3):
            assert rel_l2(out[s, k], ref[s, k]) <= 1e-5


def test_rows_outside_grid_and_single_voxel(fg):
    # a pair far from a small grid gives d = 0; a 1-voxel grid is a valid operator
    tx = np.array([[0.0, 0.5, 0.0], [0.1, 0.5, 0.0], [-0.01, 0.0, 0.0], [0.01, 0.0, 0.0]])
    rows = np.array([[0, 1], [2, 3]], dtype=np.int32)
    grid = wl.Grid(1, 1, 1, 1e-3, (0.0, 0.0005, 0.0003))
    tab = [fg.Table(1e6, 0.3e6, 4096, 3e-6)]
    geo = fg.Geometry(tx, rows, grid, 1500.0, tab)
    og = oracle.Geometry(tx, rows, None, [oracle.phi_table_gauss(1e6, 0.3e6, 4096, 3e-6)], [3e-6], grid, 1500.0)
    d = to_np(geo.J(to_dev(np.array([2.0]))))
    ref = og.J(np.array([2.0]))
    assert d[0] == 0.0 and ref[0] == 0.0
    assert d[1] == pytest.approx(ref[1], rel=1e-5)


def test_invalid_arguments(fg):
    tab = [fg.Table(1e6, 0.3e6, 4096, 3e-6)]
    grid = wl.Grid.centred(8, 8, 8, 1e-3)
    tx = wl.ring(4, 0.02)
    with pytest.raises(fg.FFTError) as ei:
        fg.Geometry(tx, np.array([[0, 0]]), grid, 1500.0, tab)
    assert ei.value.status == fg._lib.FFT_ERR_ARG
    with pytest.raises(fg.FFTError):
        fg.Geometry(tx, np.array([[0, 9]]), grid, 1500.0, tab)
    with pytest.raises(fg.FFTError):
        fg.Table(-1.0, 0.3e6, 4096, 3e-6)
    with pytest.raises(fg.FFTError):
        fg.Table(1e6, 0.3e6, 1, 3e-6)
