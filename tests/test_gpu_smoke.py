"""The repository's smoke entry point (one small J, J^T and 3-iteration CG on ring32 against
the FP64 oracle) runs and passes its own checks."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_smoke_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.smoke()
