"""Pins of the split-precision oracle (no GPU): exact reconstruction of the
digits, digit and exponent ranges, special cases that reduce to exact results
(small integers, identity and permutation right factors), and accuracy within
the 2 K u bound against the compensated reference."""
from fractions import Fraction

import numpy as np
import pytest

import workloads
from oracle import native, split


@pytest.mark.parametrize("kind", ["int8", "bf16"])
@pytest.mark.parametrize("dist", ["uniform", "wide", "smallint"])
def test_digits_reconstruct_exactly(kind, dist):
    w = split.SLICE_BITS[kind]
    A = workloads.matrix(6, 11, 3, dist)
    A[2, :] = 0.0                          # an all-zero row
    A[3, 4] = 2.0 ** -1060                 # a subnormal next to normal values
    e = split.row_exponents(A)
    S = 9
    D = split.split_rows(A, e, S, w)
    # rebuild the remainder of the last step and check
    # A_ik = 2^e_i (sum_s t_s 2^-ws + r_S 2^-wS) with |r_S| <= 1/2 exactly
    for i in range(A.shape[0]):
        for k in range(A.shape[1]):
            x = Fraction(float(A[i, k])) / Fraction(2) ** int(e[i])
            approx = sum(Fraction(int(D[s, i, k])) / Fraction(2) ** (w * (s + 1)) for s in range(S))
            rem = (x - approx) * Fraction(2) ** (w * S)
            assert abs(rem) <= Fraction(1, 2)
            assert all(abs(D[s, i, k]) <= 2 ** (w - 1) for s in range(S))
    assert np.all(D[:, 2, :] == 0)


def test_exponent_range():
    A = workloads.matrix(40, 30, 8, "wide")
    A[5] = 0.0
    e = split.row_exponents(A)
    mu = np.abs(A).max(axis=1)
    nz = mu > 0
    s = mu[nz] * 2.0 ** (-e[nz].astype(float))
    assert np.all(s >= 0.25) and np.all(s < 0.5)
    assert e[5] == 0
    assert np.array_equal(split.col_exponents(A.T), e)


def test_tie_rounds_to_even():
    # row max 0.25 = 2^-2 -> e = ilogb + 2 = 0, so r = A.  With w = 8:
    #   0.25 * 256 = 64 exactly;  (2.5/256) * 256 = 2.5 -> 2 (even), remainder
    #   +0.5 -> next digit 128;  (3.5/256) * 256 = 3.5 -> 4 (even), remainder
    #   -0.5 -> next digit -128
    A = np.array([[0.25, 2.5 / 256.0, 3.5 / 256.0]])
    e = split.row_exponents(A)
    assert e[0] == 0
    D = split.split_rows(A, e, 3, 8)
    assert D[:, 0, 0].tolist() == [64, 0, 0]
    assert D[:, 0, 1].tolist() == [2, 128, 0]
    assert D[:, 0, 2].tolist() == [4, -128, 0]
    # the same with w = 9 (bf16 up to six slices): 0.25 * 512 = 128;
    # 2.5 -> 2 with remainder +0.5 -> 256; 3.5 -> 4 with remainder -0.5 -> -256,
    # the extreme digits 2^(w-1) that bfloat16 still holds exactly
    A9 = np.array([[0.25, 2.5 / 512.0, 3.5 / 512.0]])
    D9 = split.split_rows(A9, split.row_exponents(A9), 3, 9)
    assert D9[:, 0, 0].tolist() == [128, 0, 0]
    assert D9[:, 0, 1].tolist() == [2, 256, 0]
    assert D9[:, 0, 2].tolist() == [4, -256, 0]


def test_slice_widths():
    # the widest width whose digits (|t| <= 2^(w-1)) the slice type holds,
    # capped so that w S <= 56
    assert [split.slice_bits("bf16", S) for S in range(1, 8)] == [9, 9, 9, 9, 9, 9, 8]
    assert [split.slice_bits("int8", S) for S in range(1, 9)] == [7] * 8
    for S in range(1, 8):
        w = split.slice_bits("bf16", S)
        assert w * S <= 56
        # every digit magnitude up to 2^(w-1) survives a round trip through
        # bfloat16 (8 significant bits: truncate the binary64 pattern to its top
        # 16 bits after round to nearest even), and 2^(w-1) + 1 would not
        for t in range(2 ** (w - 1) + 1):
            assert _bf16(float(t)) == float(t)
    assert _bf16(257.0) != 257.0
    assert 2 ** (split.slice_bits("int8", 1) - 1) <= 127 < 2 ** split.slice_bits("int8", 1)


def _bf16(x: float) -> float:
    """x rounded to bfloat16 (round to nearest, ties to even), by the float32
    bit pattern: bfloat16 is the top 16 bits of a float32."""
    b = int(np.array(x, dtype=np.float32).view(np.uint32))
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return float(np.array(b, dtype=np.uint32).view(np.float32))


@pytest.mark.parametrize("kind,S", [("int8", 1), ("int8", 3), ("bf16", 1), ("bf16", 4)])
def test_small_integers_exact_for_any_S(kind, S):
    A = workloads.matrix(13, 21, 51, "smallint")
    B = workloads.matrix(21, 9, 52, "smallint")
    C = split.split_gemm(A, B, S, kind)
    assert np.array_equal(C, native.dgemm(A, B))


@pytest.mark.parametrize("kind,S", [("bf16", 6), ("bf16", 7), ("int8", 8)])
def test_identity_right_factor_returns_A(kind, S):
    # B = I: f_j = 2, the only nonzero digit of column j is 2^(w-2) at row j, so
    # C^ = 2^e_i sum_s t_s 2^-ws, the first S digits of A; w S >= 54 > 53 bits
    # relative to the row maximum captures A exactly
    A = workloads.matrix(17, 12, 61, "uniform")
    C = split.split_gemm(A, np.eye(12), S, kind)
    assert np.array_equal(C, A)


def test_permutation_right_factor():
    A = workloads.matrix(9, 14, 62, "uniform")
    perm = np.array(workloads.splitmix64(3, 0, 14).argsort())
    Pm = np.eye(14)[:, perm]
    C = split.split_gemm(A, Pm, 7, "bf16")
    assert np.array_equal(C, A[:, perm])


def test_truncation_changes_with_S():
    # with fewer slices the identity product keeps only the top w S bits of each
    # row (relative to the row maximum), within half a unit of the last digit
    A = workloads.matrix(5, 8, 63, "uniform")
    e = split.row_exponents(A)
    for S in (2, 3, 4):
        C = split.split_gemm(A, np.eye(8), S, "bf16")
        w = split.slice_bits("bf16", S)
        bound = 0.5 * 2.0 ** (e[:, None].astype(float) - w * S)
        assert np.all(np.abs(C - A) <= bound * (1 + 2.0 ** -50) + np.abs(A) * 2.0 ** -53)


def test_pairs_triangle():
    assert split.kept_pairs(3) == [(1, 1), (1, 2), (2, 1), (1, 3), (2, 2), (3, 1)]
    assert len(split.kept_pairs(6)) == 21


@pytest.mark.parametrize("kind,S", [("bf16", 5), ("bf16", 6), ("int8", 6), ("int8", 7)])
def test_accuracy_bound_uniform(kind, S):
    # FP64-accurate: max |C - C^| / (|A||B|) <= 2 K u on uniform[-1, 1] inputs.
    # The slicing error relative to |A||B| hardly depends on K while the bound
    # grows with K, so the smallest passing S depends on K; K = 4096 here.
    M, N, K = 16, 16, 4096
    A = workloads.matrix(M, K, 1002, "uniform")
    B = workloads.matrix(K, N, 2002, "uniform")
    C = split.split_gemm(A, B, S, kind)
    ref, absab = native.dot2_full(A, B)
    assert split.max_rel_error(C, ref, absab) <= split.tolerance(K)


def test_accuracy_improves_with_S():
    M, N, K = 16, 16, 128
    A = workloads.matrix(M, K, 1002, "wide")
    B = workloads.matrix(K, N, 2002, "wide")
    ref, absab = native.dot2_full(A, B)
    errs = [split.max_rel_error(split.split_gemm(A, B, S, "bf16"), ref, absab) for S in (2, 3, 4, 5)]
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_entries_match_full():
    A = workloads.matrix(10, 40, 71, "wide")
    B = workloads.matrix(40, 12, 72, "uniform")
    C = split.split_gemm(A, B, 4, "int8")
    rows, cols = np.array([0, 9, 3, 3]), np.array([11, 0, 5, 6])
    assert np.array_equal(split.split_entries(A, B, rows, cols, 4, "int8"), C[rows, cols])


def test_round_scaled_is_correctly_rounded():
    # ties to even, subnormal results and overflow
    assert split.round_scaled(2 ** 53 + 1, 0) == 2.0 ** 53
    assert split.round_scaled(2 ** 53 + 3, 0) == 2.0 ** 53 + 4
    assert split.round_scaled(3, -1075) == 2.0 ** -1074 * 2      # 1.5 ulp -> 2 ulp
    assert split.round_scaled(1, -1075) == 0.0                    # half ulp -> even 0
    assert split.round_scaled(3, 1023) == float("inf")
    assert split.round_scaled(-3, 1023) == float("-inf")


def test_metric_zero_denominator():
    assert split.max_rel_error(np.zeros(2), np.zeros(2), np.zeros(2)) == 0.0
    assert split.max_rel_error(np.array([1e-300]), np.zeros(1), np.zeros(1)) == float("inf")


@pytest.mark.parametrize("S", [2, 3, 4, 5])
def test_diagonal_products_form_exactly_the_triangle(S):
    # one entry, K = 1, digits chosen so that every slice pair contributes its
    # own power of two: a_s = 2^(s-1), b_t = 2^(S (t-1)), so a_s b_t = 2^(s-1+S(t-1))
    # has a distinct exponent for each of the S^2 pairs and D_d, read in binary,
    # names exactly the pairs summed into it.  A dropped or extra pair, a square
    # pair set or a wrong diagonal changes the diagonals or their bits.
    Ad = np.array([[[2.0 ** (s - 1)]] for s in range(1, S + 1)])      # S x 1 x 1
    Bd = np.array([[[2.0 ** (S * (t - 1))]] for t in range(1, S + 1)])
    D = split.diagonal_products(Ad, Bd, S, 8)
    assert sorted(D) == list(range(2, S + 2))
    for d, v in D.items():
        bits = {(b % S + 1, b // S + 1) for b in range(S * S) if (int(v[0, 0]) >> b) & 1}
        assert bits == {(s, d - s) for s in range(1, d)}, (d, bits)
    assert sum(bin(int(v[0, 0])).count("1") for v in D.values()) == S * (S + 1) // 2


def _exact_from_digits(A, B, S, kind, square=False):
    """C^ from the digits of step 2 with exact rationals: the sum over the slice
    pairs (all S^2 of them if `square`, else s + t <= S + 1) of
    a_s[i,k] b_t[k,j] 2^(e_i + f_j - w (s + t)), rounded once (float(Fraction) is
    correctly rounded, ties to even)."""
    w = split.slice_bits(kind, S)
    e, f = split.row_exponents(A), split.col_exponents(B)
    Ad, Bd = split.split_rows(A, e, S, w), split.split_cols(B, f, S, w)
    M, K = A.shape
    N = B.shape[1]
    C = np.empty((M, N))
    for i in range(M):
        for j in range(N):
            x = Fraction(0)
            for s in range(1, S + 1):
                for t in range(1, S + 1):
                    if not square and s + t > S + 1:
                        continue
                    dot = sum(int(Ad[s - 1, i, k]) * int(Bd[t - 1, k, j]) for k in range(K))
                    x += Fraction(dot) * Fraction(2) ** (int(e[i]) + int(f[j]) - w * (s + t))
            C[i, j] = float(x)
    return C


@pytest.mark.parametrize("kind", ["int8", "bf16"])
@pytest.mark.parametrize("S", [2, 3, 4])
def test_split_gemm_is_the_rounded_exact_triangle_sum(kind, S):
    # the whole split path against its definition: the exact sum of the kept
    # slice-pair products (Ozaki et al.: pairs with s + t <= S + 1), rounded
    # once; and the square pair set gives a different result on the same inputs,
    # so a path that formed extra pairs would fail here
    A = workloads.matrix(5, 6, 90 + S, "wide")
    B = workloads.matrix(6, 4, 190 + S, "wide")
    got = split.split_gemm(A, B, S, kind)
    assert np.array_equal(got, _exact_from_digits(A, B, S, kind))
    assert not np.array_equal(got, _exact_from_digits(A, B, S, kind, square=True))
    rows, cols = np.array([0, 4, 2, 1]), np.array([3, 0, 1, 2])
    assert np.array_equal(split.split_entries(A, B, rows, cols, S, kind), got[rows, cols])
