"""Peak microbenchmarks run and report plausible rates (GPU); the measured
values are printed for the roofline denominators."""
import pytest

from tests.gpu_util import lib_ready

pytestmark = pytest.mark.gpu


# The tcgen05 rates must show every SM busy at the full tensor rate (8192 bf16
# flops per cycle and SM: about 2.4e15 at 1.95 GHz); 1.5e15 leaves room for a
# power-capped clock and stays above what half of the SMs could reach.
@pytest.mark.parametrize("kind,work,lo,hi", [
    ("dfma", 2000, 1e11, 2e14), ("dmma", 2000, 1e11, 2e14), ("imma", 2000, 1e12, 2e16),
    ("hmma_bf16", 2000, 1e12, 5e15), ("tc05_bf16", 200000, 1.5e15, 3e15),
    ("copy", 1024, 1e12, 2e13), ("tc05_bf16_pair", 200000, 1.5e15, 3e15),
])
def test_peak(kind, work, lo, hi):
    hs = lib_ready()
    r = hs.peak(kind, work)
    print(f"PEAK {kind} {r:.4e}")
    assert lo < r < hi
