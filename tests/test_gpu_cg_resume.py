"""CG checkpoint and resume (fft_cg_continue, fft_cg_save / fft_cg_load): a solve of k
iterations continued for n gives the same bits as one solve of k + n, also when its state is
saved to host memory and loaded into another handle of the same geometry; a handle without a
state, or a foreign or damaged state, is refused with a status code."""
import numpy as np
import pytest

import workloads as wl
from gpu_common import gpu_geometry, oracle_geometry, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ring32():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w, og = oracle_geometry("ring32")
    geo, _ = gpu_geometry(w)
    d = og.J(wl.model_for(w)) + wl.noise(og.M, w.noise_seed)
    return w, og, geo, to_dev(d)


def bits(t):
    return t.detach().cpu().numpy().view(np.uint32)


def test_continue_equals_one_solve(ring32):
    w, og, geo, d = ring32
    m10, h10 = geo.cg_solve(d, w.lambda_rel, 10, with_history=True)
    m10 = m10.clone()
    geo.cg_solve(d, w.lambda_rel, 5)
    m, h = geo.cg_continue(5, with_history=True)
    assert np.array_equal(bits(m), bits(m10))
    assert np.array_equal(h, h10[5:])
    # and in two steps of 2 and 3
    geo.cg_solve(d, w.lambda_rel, 5)
    geo.cg_continue(2)
    m = geo.cg_continue(3)
    assert np.array_equal(bits(m), bits(m10))


def test_save_load_resume_in_another_handle(ring32):
    w, og, geo, d = ring32
    m10 = geo.cg_solve(d, w.lambda_rel, 10).clone()
    geo.cg_solve(d, w.lambda_rel, 4)
    state = geo.cg_save()
    assert state.size == 64 + 4 * (2 * geo.V + geo.M)
    geo2, _ = gpu_geometry(w)
    geo2.cg_load(state)
    m = geo2.cg_continue(6)
    assert np.array_equal(bits(m), bits(m10))
    # the saved state also resumes the handle it came from after other work on it
    geo.cg_solve(d, w.lambda_rel, 7)
    geo.cg_load(state)
    assert np.array_equal(bits(geo.cg_continue(6)), bits(m10))
    geo2.close()


def test_refused_states(ring32):
    import paper_1908_03302_gb300 as fg
    w, og, geo, d = ring32
    fresh, _ = gpu_geometry(w)
    with pytest.raises(fg.FFTError) as ei:
        fresh.cg_continue(2)
    assert ei.value.status == fg._lib.FFT_ERR_STATE
    with pytest.raises(fg.FFTError) as ei:
        fresh.cg_save()
    assert ei.value.status == fg._lib.FFT_ERR_STATE
    geo.cg_solve(d, w.lambda_rel, 3)
    state = geo.cg_save()
    damaged = state.copy()
    damaged[0] ^= 0xFF                    # magic
    short = state[: state.size - 4]
    for bad in (damaged, short):
        with pytest.raises(fg.FFTError) as ei:
            fresh.cg_load(bad)
        assert ei.value.status == fg._lib.FFT_ERR_ARG
    wt, _ = oracle_geometry("tiny")
    other, _ = gpu_geometry(wt)           # another number of rows and voxels
    with pytest.raises(fg.FFTError) as ei:
        other.cg_load(state)
    assert ei.value.status == fg._lib.FFT_ERR_ARG
    other.close()
    fresh.close()
