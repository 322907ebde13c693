"""The roofline denominators the library measures on the device
(rom_measure_peak): each microbenchmark runs, and its figure lies in the
range the GB300's unit counts and clocks allow (nominal rates at the 2070 MHz
maximum SM clock: FP32 80.5 and BF16 2250 TFLOP/s dense, TF32 half of BF16,
FP64 about 1.25 TFLOP/s; L2 reads well above the HBM copy rate)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rom():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_11742_gb300 import build
    build.build()
    from paper_2009_11742_gb300 import rom as R
    return R


@pytest.mark.parametrize("kind,lo,hi", [("fp32", 20.0, 90.0), ("fp64", 0.2, 3.0),
                                        ("tf32", 150.0, 1300.0), ("bf16", 300.0, 2600.0),
                                        ("l2", 5000.0, 80000.0)])
def test_measured_peak_in_range(rom, kind, lo, hi):
    v, ms = rom.measure_peak(kind)
    assert lo <= v <= hi, (kind, v)
    assert ms > 0.5


def test_measure_peak_rejects_unknown_kind(rom):
    st, _, _ = rom.rom_measure_peak(9)
    assert st == rom.ROM_E_INVAL
