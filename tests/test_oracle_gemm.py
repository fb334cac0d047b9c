"""Pins of the binary64 GEMM oracle and the Dot2 reference against exact
rational arithmetic, closed forms and invariants (no GPU)."""
from fractions import Fraction

import numpy as np
import pytest

import workloads
from oracle import native

U = 2.0 ** -53


def exact_product(A, B):
    M, K = A.shape
    N = B.shape[1]
    Af = [[Fraction(float(x)) for x in row] for row in A]
    Bf = [[Fraction(float(x)) for x in row] for row in B]
    return [[sum((Af[i][k] * Bf[k][j] for k in range(K)), Fraction(0)) for j in range(N)]
            for i in range(M)]


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (3, 5, 7), (8, 8, 8), (5, 2, 9)])
def test_small_integer_exact(M, N, K):
    # every partial sum is an integer below 2^53: the result is exact
    A = workloads.matrix(M, K, 11, "smallint")
    B = workloads.matrix(K, N, 12, "smallint")
    C = native.dgemm(A, B)
    E = exact_product(A, B)
    assert all(C[i, j] == float(E[i][j]) for i in range(M) for j in range(N))


@pytest.mark.parametrize("M,N,K", [(4, 6, 8), (7, 3, 16)])
def test_float_within_textbook_bound(M, N, K):
    # recursive summation: |C - AB| <= gamma_K |A||B|, gamma_K = K u / (1 - K u)
    A = workloads.matrix(M, K, 21, "uniform")
    B = workloads.matrix(K, N, 22, "wide")
    C = native.dgemm(A, B)
    E = exact_product(A, B)
    g = K * U / (1 - K * U)
    for i in range(M):
        for j in range(N):
            absab = sum(abs(Fraction(float(A[i, k])) * Fraction(float(B[k, j]))) for k in range(K))
            assert abs(Fraction(float(C[i, j])) - E[i][j]) <= Fraction(g) * absab


def test_identity_and_permutation_exact():
    A = workloads.matrix(33, 17, 5, "wide")
    I = np.eye(17)
    assert np.array_equal(native.dgemm(A, I), A)
    perm = np.array(workloads.splitmix64(9, 0, 17).argsort())
    Pm = np.eye(17)[:, perm]            # A @ Pm permutes the columns of A
    assert np.array_equal(native.dgemm(A, Pm), A[:, perm])
    Pl = np.eye(33)[perm[:1].tolist() + [i for i in range(33) if i != perm[0]]]
    assert np.array_equal(native.dgemm(Pl, A), Pl @ A)


def test_summation_order_is_ascending_k():
    # (1 + 2^-53) + (-1): ascending order gives 2^-53 * 0 ... check a case where
    # the order of the three terms decides the rounded result
    A = np.array([[1.0, 2.0 ** -53, -1.0]])
    B = np.array([[1.0], [1.0], [1.0]])
    # ((0 + 1) + 2^-53) + (-1) = (1) + (-1) = 0 (1 + 2^-53 rounds to 1)
    assert native.dgemm(A, B)[0, 0] == 0.0


def test_empty_shapes():
    C = native.dgemm(np.zeros((3, 0)), np.zeros((0, 4)))
    assert C.shape == (3, 4) and np.all(C == 0)


@pytest.mark.parametrize("K", [1, 5, 64])
def test_dot2_within_its_bound(K):
    # Ogita-Rump-Oishi: |Dot2 - x.y| <= u |x.y| + gamma_K^2 sum |x_i y_i|
    A = workloads.matrix(3, K, 31, "wide")
    B = workloads.matrix(K, 4, 32, "wide")
    rows, cols = np.repeat(np.arange(3), 4), np.tile(np.arange(4), 3)
    c, ab = native.dot2_entries(A, B, rows, cols)
    E = exact_product(A, B)
    g = K * U / (1 - K * U)
    for t in range(rows.size):
        e = E[rows[t]][cols[t]]
        absab = sum(abs(Fraction(float(A[rows[t], k])) * Fraction(float(B[k, cols[t]]))) for k in range(K))
        assert abs(Fraction(float(c[t])) - e) <= Fraction(U) * abs(e) + Fraction(g * g) * absab
        # the |A||B| entry: a plain sum of nonnegative terms, relative error <= gamma_K
        assert abs(Fraction(float(ab[t])) - absab) <= Fraction(g) * absab


def test_dot2_cancellation():
    # 1e16 + 1 - 1e16 = 1 exactly; the naive sum loses the 1
    A = np.array([[1e16, 1.0, -1e16]])
    B = np.array([[1.0], [1.0], [1.0]])
    c, ab = native.dot2_entries(A, B, [0], [0])
    assert c[0] == 1.0
    assert native.dgemm(A, B)[0, 0] == 0.0


def test_dot2_full_matches_entries():
    A = workloads.matrix(5, 9, 41)
    B = workloads.matrix(9, 6, 42)
    c, ab = native.dot2_full(A, B)
    c2, ab2 = native.dot2_entries(A, B, [4, 0], [5, 2])
    assert c[4, 5] == c2[0] and c[0, 2] == c2[1] and ab[4, 5] == ab2[0]
