"""fft_psf_noalloc: the point-spread-function entry point that allocates no device memory.

It serves callers that may not call the device allocator while running (memory reserved up
front, or another framework's memory pool). Its scratch is a fixed array inside the library,
shared by all calls and left holding the previous call's values, so two calls in a row with
different spikes and row subsets check that each call clears what it uses. The references are
the allocating fft_psf_batch on the same geometry and the FP64 oracle, with the parity
tolerance used throughout the GPU tests (relative L2 <= 1e-5). The device's free memory and
PyTorch's allocated bytes must not change across a call, and row indices outside [0, M) are
skipped and reported.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ring32():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_03302_gb300 as fg
    import workloads as wl

    w = wl.ring32()
    b = w.bands[0]
    table = fg.Table(b.f_center_hz, b.f_sigma_hz, b.n_samples, b.dt_max)
    geo = fg.Geometry(w.tx, w.pairs, w.grid, w.c0, [table])

    def vox(i, j, k):
        return int((k * w.grid.ny + j) * w.grid.nx + i)

    return fg, w, geo, table, vox


def test_psf_noalloc_matches_psf_batch_twice(ring32):
    import oracle
    fg, w, geo, table, vox = ring32
    og = oracle.Geometry.from_workload(w)
    # spikes inside the 50 mm ring: one near the centre, one off-centre in another slice
    cases = [
        (vox(24, 24, 8), np.arange(geo.M, dtype=np.int32)),              # all rows
        (vox(31, 18, 5), np.arange(0, geo.M, 5, dtype=np.int32)),        # a fifth of them
    ]
    for spike, rows in cases:
        ref = geo.psf_batch([spike], [rows])[0, 0].double().cpu().numpy()
        got = geo.psf_noalloc(spike, torch.as_tensor(rows, device="cuda")).double().cpu().numpy()
        assert np.linalg.norm(ref) > 0
        assert rel_l2(got, ref) <= 1e-5
        assert rel_l2(got, og.psf(np.array([spike]), [rows])[0, 0]) <= 1e-5


def test_psf_noalloc_allocates_nothing(ring32):
    fg, w, geo, table, vox = ring32
    rows = torch.arange(0, geo.M, 3, dtype=torch.int32, device="cuda")
    out = torch.empty(geo.V, dtype=torch.float32, device="cuda")
    geo.psf_noalloc(vox(20, 26, 9), rows, out=out)      # warm-up
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    geo.psf_noalloc(vox(27, 21, 6), rows, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_psf_noalloc_rows_outside_are_skipped_and_reported(ring32):
    fg, w, geo, table, vox = ring32
    spike = vox(22, 25, 7)
    valid = np.arange(1, geo.M, 2, dtype=np.int32)
    rows = torch.as_tensor(np.concatenate([valid, [geo.M]]).astype(np.int32), device="cuda")
    out = torch.empty(geo.V, dtype=torch.float32, device="cuda")
    with pytest.raises(fg.FFTError) as ei:
        geo.psf_noalloc(spike, rows, out=out)
    assert ei.value.status == fg._lib.FFT_ERR_ARG
    ref = geo.psf_batch([spike], [valid])[0, 0].double().cpu().numpy()
    assert rel_l2(out.double().cpu().numpy(), ref) <= 1e-5
