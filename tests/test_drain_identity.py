"""The integer identity the bf16 kernels' drain uses (no GPU).

An fp32 accumulator of exact digit products holds an integer x, |x| <= 2^24.
The drain adds it to an int32 sum as bits(x + 1.5 * 2^23) - bits(1.5 * 2^23)
when |x| <= 2^22, and with the float-to-int conversion otherwise (after a
check that flags any |x| >= 2^22).  Here the identity is checked with IEEE
binary32 arithmetic on the CPU (round to nearest even, as the GPU's add):
exact on the whole range it is used for, wrong just past it (so the check
is needed), and the fix-up (conversion minus the fast value) exact for every
x the accumulator can hold."""
import numpy as np

MAGIC = np.float32(12582912.0)          # 1.5 * 2^23
MAGIC_BITS = np.uint32(0x4B400000)


def fast(x: np.ndarray) -> np.ndarray:
    """The drain's add-based conversion, modulo 2^32, as int64."""
    y = (x.astype(np.float32) + MAGIC).astype(np.float32)
    return ((y.view(np.uint32) - MAGIC_BITS).astype(np.uint32)).astype(np.int64)


def as_int32(v: np.ndarray) -> np.ndarray:
    v = np.asarray(v, dtype=np.int64) & 0xFFFFFFFF
    return np.where(v >= 2 ** 31, v - 2 ** 32, v)


def test_magic_bits():
    assert np.array(MAGIC, dtype=np.float32).view(np.uint32) == MAGIC_BITS


def test_exact_up_to_two_to_the_22():
    rng = np.random.default_rng(1)
    edges = np.array([0, 1, -1, 2, -2, 2 ** 21, -(2 ** 21), 2 ** 22 - 1, -(2 ** 22 - 1),
                      2 ** 22, -(2 ** 22)], dtype=np.int64)
    xs = np.concatenate([edges, rng.integers(-(2 ** 22), 2 ** 22 + 1, 200000),
                         np.arange(-70000, 70001)])
    assert np.array_equal(as_int32(fast(xs)), xs)
    # -0.0 (an empty chunk's sum may be either zero)
    assert as_int32(fast(np.array([-0.0])))[0] == 0


def test_wrong_past_two_to_the_22():
    # every odd x above 2^22 in magnitude rounds (x + 1.5 * 2^23 needs 25 bits),
    # and large negative ones fall below 2^23: the check is needed
    xs = np.array([2 ** 22 + 1, 2 ** 22 + 3, 2 ** 23 + 1, -(2 ** 22) - 1, -(2 ** 23) - 5,
                   2 ** 24 - 1], dtype=np.int64)
    assert np.all(as_int32(fast(xs)) != xs)


def test_fix_up_restores_every_value():
    # the fix-up adds conversion(x) - fast(x) to a sum that already holds
    # fast(x): the total is x, modulo 2^32, for every |x| <= 2^24
    rng = np.random.default_rng(2)
    xs = np.concatenate([rng.integers(-(2 ** 24), 2 ** 24 + 1, 200000),
                         np.array([2 ** 24, -(2 ** 24), 2 ** 22 + 1, -(2 ** 22) - 1])])
    conv = np.rint(xs.astype(np.float32).astype(np.float64)).astype(np.int64)
    assert np.array_equal(conv, xs)                      # integers <= 2^24 are exact in fp32
    acc = fast(xs) + (conv - fast(xs))
    assert np.array_equal(as_int32(acc), xs)


def test_flag_bound_is_sufficient():
    # the drain flags a warp's values when their largest magnitude reaches
    # 2^22; below that every value converts exactly (the boundary included)
    xs = np.array([2 ** 22 - 1, -(2 ** 22 - 1)], dtype=np.int64)
    assert np.all(np.abs(xs) < 2 ** 22)
    assert np.array_equal(as_int32(fast(xs)), xs)


def test_exact_chunk_bounds():
    # digit products of width w are at most 2^(2w - 2) in magnitude; a chunk of
    # 2^(26 - 2w) of them stays within 2^24, where fp32 holds every integer
    for w, chunk in ((9, 256), (8, 1024)):
        assert chunk * (2 ** (w - 1)) ** 2 == 2 ** 24
        assert float(np.float32(2 ** 24)) == 2 ** 24
        assert float(np.float32(2 ** 24 - 1)) == 2 ** 24 - 1
    # 127 such chunks fit int32, 128 would not in the worst case
    assert 127 * 2 ** 24 < 2 ** 31 <= 128 * 2 ** 24
