"""The seeded generator: SplitMix64 against its published reference values, the
distributions' ranges, and numpy/torch agreement (no GPU)."""
import numpy as np
import pytest

import workloads


def test_splitmix64_reference_values():
    # Reference outputs of SplitMix64 seeded with 1234567 (the values printed
    # with Vigna's reference implementation, splitmix64.c)
    x = workloads.splitmix64(1234567, 0, 5)
    assert [int(v) for v in x] == [6457827717110365317, 3203168211198807973,
                                   9817491932198370423, 4593380528125082431,
                                   16408922859458223821]


def test_stream_offsets_consistent():
    a = workloads.splitmix64(7, 0, 100)
    b = workloads.splitmix64(7, 40, 60)
    assert np.array_equal(a[40:], b)


def test_ranges():
    u = workloads.matrix(64, 65, 1, "uniform")
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.05
    s = workloads.matrix(64, 65, 2, "smallint")
    assert set(np.unique(s)) == set(range(-8, 9))
    w = workloads.matrix(64, 65, 3, "wide")
    _, e = np.frexp(np.abs(w[w != 0]))
    assert e.min() >= -21 - 30 and e.max() <= 21
    n = workloads.matrix(200, 100, 4, "normal_spiked")
    big = np.abs(n).max(axis=0) > 1e4
    assert big.sum() == 1


def test_chunking_does_not_change_values():
    a = workloads.matrix(37, 29, 5, "wide")
    b = workloads.matrix(37, 29, 5, "wide", chunk_rows=4)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("dist", ["uniform", "smallint", "wide"])
def test_torch_matches_numpy(dist):
    torch = pytest.importorskip("torch")
    a = workloads.matrix(19, 23, 77, dist)
    b = workloads.matrix_torch(19, 23, 77, dist).numpy()
    assert np.array_equal(a, b)


def test_normal_distributions_and_torch_generator():
    torch = pytest.importorskip("torch")
    a = workloads.matrix(400, 300, 19, "normal")
    assert abs(a.mean()) < 0.02 and abs(a.std() - 1.0) < 0.02
    s = workloads.matrix(400, 300, 19, "normal_spiked")
    spiked = np.nonzero(np.abs(s).max(axis=0) > 1e4)[0]
    assert spiked.size == 3                                  # round(0.01 * 300)
    assert np.array_equal(np.delete(s, spiked, axis=1), np.delete(a, spiked, axis=1))
    t = workloads.matrix_torch(400, 300, 19, "normal_spiked").numpy()
    assert np.allclose(t, s, rtol=1e-14, atol=0)             # same draws, libm rounding apart
