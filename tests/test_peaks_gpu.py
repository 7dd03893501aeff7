"""The random-gather microbenchmark behind the gather roofline: it runs and
reports rates in a plausible range for one GPU."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cgo():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19163_gb300 import cgo as C
    return C


def test_shared_and_l2_gather_rates(cgo):
    smem, ms = cgo.gather_peak(0, 16)
    assert ms > 0
    # at most one 32-lane wavefront per clock per SM (200 SMs at 3 GHz bounds any part)
    assert 1e10 < smem < 200 * 3e9 * 32
    l2, _ = cgo.gather_peak(1, 18)
    assert 1e9 < l2 < smem * 4
