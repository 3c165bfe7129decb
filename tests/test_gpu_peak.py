"""The FMA microbenchmark: plausible rates and clock on the device it runs
on. Bounds come from the unit counts (128 FP32 lanes per multiprocessor,
an FMA = 2 FLOP) at the clock the kernel itself reads."""
import pytest

from paper_2603_19764_b300 import build, sph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_fma_peak_fp32_and_fp64():
    f32 = sph.measure_fma_peak(1, launches=5)
    f64 = sph.measure_fma_peak(0, launches=2)
    assert 500 < f32["sm_mhz"] < 3000, f32
    unit = 128 * 2 * f32["n_sm"] * f32["sm_mhz"] * 1e6 / 1e12
    # issue-bound chains reach most of the unit-count rate, never above it
    assert 0.5 * unit < f32["tflops"] < 1.05 * unit, (f32, unit)
    assert 0 < f64["tflops"] < f32["tflops"], (f64, f32)
