"""The measured FP64 rate used as the FP64 roofline's peak: positive, within
a factor of two of the nominal GB300 figure (152 SMs x 2 FP64 FMA per clock x
2 flops x 2.07 GHz = 1.26 TFLOP/s), and stable between calls."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1310_7087_gb300 import build
    build.build()
    import paper_1310_7087_gb300 as q
    return q


def test_fp64_probe_rate(q):
    a, b = q.qcd_probe_fp64_rate(), q.qcd_probe_fp64_rate()
    assert 0.6e12 < a < 2.6e12, a
    assert abs(a - b) < 0.1 * a, (a, b)
