"""Peak microbenchmarks run and report plausible rates (GPU); the measured
values are printed for the roofline denominators."""
import pytest

from tests.gpu_util import lib_ready

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,work,lo,hi", [
    ("dfma", 2000, 1e11, 2e14), ("dmma", 2000, 1e11, 2e14), ("imma", 2000, 1e12, 2e16),
    ("hmma_bf16", 2000, 1e12, 5e15), ("tc05_bf16", 20000, 1e14, 5e15), ("copy", 1024, 1e12, 2e13),
    ("tc05_bf16_pair", 20000, 1e14, 5e15),
])
def test_peak(kind, work, lo, hi):
    hs = lib_ready()
    r = hs.peak(kind, work)
    print(f"PEAK {kind} {r:.4e}")
    assert lo < r < hi
