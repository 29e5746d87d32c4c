"""The tensor-core (tcgen05) operand layout and descriptors: a 128 x n x k BF16 product with
integer-valued operands must be exact."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n,k", [(128, 64), (256, 64), (32, 16), (64, 128)])
def test_tc_selftest_exact(n, k):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_03302_gb300 as fg
    assert fg.tc_selftest(n, k) == 0.0
