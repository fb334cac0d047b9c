"""Oracle for the split-precision (Ozaki-style) path of C = A x B.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper itself only multiplies in binary64 (Section II-A: the local update is
a DGEMM).  The split path is the error-free splitting of Ozaki, Ogita, Oishi and
Rump ("Error-free transformations of matrix multiplication by using fast
routines of matrix multiplication and its applications", Numer. Algorithms
59, 2012), with integer-valued slices as in Ootomo, Ozaki and Yokota ("DGEMM on
integer matrix multiplication unit", IJHPCA 2024).  The steps below are written
from those definitions; where they leave a choice, the reading taken is stated
at the step.

Steps, for slice width w bits and S slices:
  1. scaling: e_i = ilogb(max_k |A_ik|) + 2 (0 for an all-zero row), so that
     |A_ik| 2^-e_i < 1/2; likewise f_j over the columns of B.
  2. splitting: r <- A_ik 2^-e_i; for s = 1..S:  y <- r 2^w;  t_s <- rint(y)
     (round half to even);  r <- y - t_s.  Every operation is exact in
     binary64, |t_s| <= 2^(w-1), and A_ik = 2^e_i (sum_s t_s 2^(-w s) + r 2^(-wS)).
  3. products: for every kept pair (s, t), s + t <= S + 1, the integer matrix
     P_st = A_s B_t, grouped by diagonal d = s + t:  D_d = sum_{s+t=d} P_st.
  4. recombination: C^_ij = RN( 2^(e_i + f_j) sum_d D_d,ij 2^(-w d) ), the
     exact sum of the kept terms rounded once to binary64 (round to nearest,
     ties to even).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

# Widest slice width w (bits) per slice type: a digit |t| <= 2^(w-1) must be
# exact in it.  INT8 holds [-128, 127], so w = 7 (digits in [-64, 64]); every
# integer of magnitude <= 256 is exact in bfloat16's 8-bit significand, so
# w = 9 (digits in [-256, 256]).
SLICE_BITS = {"int8": 7, "bf16": 9}
SLICE_RANGE = {"int8": (3, 8), "bf16": (3, 6)}
# The S slices of an operand hold at most this many bits (w S).  This is the
# library's definition, which the oracle follows: its digit extraction works
# from a 64-bit fixed-point image of each scaled value and needs the last
# digit's rounding bit well above the image's bottom.
MAX_SLICED_BITS = 56


def slice_bits(kind: str, S: int) -> int:
    """The slice width used with S slices of type `kind`: the widest exact one,
    narrowed where S of them would pass MAX_SLICED_BITS (bf16 with S = 7 takes
    w = 8)."""
    return min(SLICE_BITS[kind], MAX_SLICED_BITS // S)


def row_exponents(A: np.ndarray) -> np.ndarray:
    """Step 1 for the rows of A: e_i with max_k |A_ik| 2^-e_i in [1/4, 1/2)."""
    A = np.asarray(A, dtype=np.float64)
    if not np.all(np.isfinite(A)):
        raise ValueError("split path needs finite inputs")
    mu = np.abs(A).max(axis=1) if A.shape[1] else np.zeros(A.shape[0])
    _, ex = np.frexp(mu)          # mu = m 2^ex, m in [1/2, 1)  =>  ilogb = ex - 1
    return np.where(mu > 0, ex + 1, 0).astype(np.int64)


def col_exponents(B: np.ndarray) -> np.ndarray:
    """Step 1 for the columns of B."""
    return row_exponents(np.asarray(B, dtype=np.float64).T)


def split_rows(A: np.ndarray, e: np.ndarray, S: int, w: int) -> np.ndarray:
    """Step 2 for the rows of A: returns digits t[s, i, k], s = 0..S-1, as float64."""
    r = np.ldexp(np.asarray(A, dtype=np.float64), -e[:, None])
    out = np.empty((S,) + r.shape, dtype=np.float64)
    for s in range(S):
        y = np.ldexp(r, w)
        t = np.rint(y)
        r = y - t
        out[s] = t
    return out


def split_cols(B: np.ndarray, f: np.ndarray, S: int, w: int) -> np.ndarray:
    """Step 2 for the columns of B: digits u[t, k, j]."""
    return np.transpose(split_rows(np.asarray(B).T, f, S, w), (0, 2, 1))


def kept_pairs(S: int):
    """Step 3's pairs (s, t), 1-based, with s + t <= S + 1, by diagonal d = s + t."""
    return [(s, d - s) for d in range(2, S + 2) for s in range(1, d)]


def diagonal_products(Ad: np.ndarray, Bd: np.ndarray, S: int, w: int) -> dict:
    """Step 3: D_d = sum_{s+t=d} A_s B_t as exact int64 matrices, over the pairs
    kept_pairs(S) gives (so the diagonals are d = 2..S+1).

    The float64 library matmul is exact here: every product of two digits is an
    integer of magnitude <= 2^(2w-2) and every partial sum of the (d-1) K terms
    stays below 2^53 (asserted), so no rounding happens in any order."""
    K = Ad.shape[2]
    acc = {}
    for s, t in kept_pairs(S):
        d = s + t
        assert (d - 1) * K * 2 ** (2 * w - 2) < 2 ** 53, "exactness bound"
        if d not in acc:
            acc[d] = np.zeros((Ad.shape[1], Bd.shape[2]), dtype=np.float64)
        acc[d] += Ad[s - 1] @ Bd[t - 1]
    return {d: v.astype(np.int64) for d, v in acc.items()}


def round_scaled(X: int, k: int) -> float:
    """RN(X * 2^k) for an integer X: exact rational, rounded once (CPython's
    int -> float and int / int are correctly rounded, ties to even)."""
    if X == 0:
        return 0.0
    try:
        if k >= 0:
            return float(X << k)
        return X / (1 << -k)
    except OverflowError:
        return float("inf") if X > 0 else float("-inf")


def recombine(D: dict, e: np.ndarray, f: np.ndarray, S: int, w: int) -> np.ndarray:
    """Step 4: C^_ij = RN(2^(e_i+f_j) sum_d D_d,ij 2^(-w d))."""
    M, N = e.size, f.size
    X = np.zeros((M, N), dtype=object)
    for d in sorted(D):
        X = X + (D[d].astype(object) * (1 << (w * (S + 1 - d))))
    C = np.empty((M, N), dtype=np.float64)
    base = -w * (S + 1)
    for i in range(M):
        ei = int(e[i]) + base
        row = X[i]
        for j in range(N):
            C[i, j] = round_scaled(int(row[j]), ei + int(f[j]))
    return C


def split_gemm(A: np.ndarray, B: np.ndarray, S: int, kind: str = "bf16",
               return_parts: bool = False):
    """The whole split path on the CPU: C^ ~= A x B from S slices of type `kind`."""
    w = slice_bits(kind, S)
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    e = row_exponents(A)
    f = col_exponents(B)
    Ad = split_rows(A, e, S, w)
    Bd = split_cols(B, f, S, w)
    D = diagonal_products(Ad, Bd, S, w)
    C = recombine(D, e, f, S, w)
    if return_parts:
        return C, dict(e=e, f=f, Ad=Ad, Bd=Bd, D=D, w=w)
    return C


def split_entries(A: np.ndarray, B: np.ndarray, rows, cols, S: int,
                  kind: str = "bf16") -> np.ndarray:
    """C^ at listed entries only (for full-size checks): same steps, restricted
    to the rows of A and columns of B that the entries use."""
    w = slice_bits(kind, S)
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    ur, ir = np.unique(rows, return_inverse=True)
    uc, ic = np.unique(cols, return_inverse=True)
    Ar = np.asarray(A, dtype=np.float64)[ur]
    Bc = np.asarray(B, dtype=np.float64)[:, uc]
    e = row_exponents(Ar)
    f = col_exponents(Bc)
    Ad = split_rows(Ar, e, S, w)
    Bd = split_cols(Bc, f, S, w)
    K = Ar.shape[1]
    out = np.empty(rows.size, dtype=np.float64)
    base = -w * (S + 1)
    pairs = kept_pairs(S)
    for n in range(rows.size):
        a, b = ir[n], ic[n]
        Dd = {}
        for s, t in pairs:
            d = s + t
            assert (d - 1) * K * 2 ** (2 * w - 2) < 2 ** 53
            Dd[d] = Dd.get(d, 0.0) + float(Ad[s - 1, a, :] @ Bd[t - 1, :, b])
        X = sum(int(v) << (w * (S + 1 - d)) for d, v in Dd.items())
        out[n] = round_scaled(X, int(e[a]) + int(f[b]) + base)
    return out


def max_rel_error(C_hat, C_ref, absab) -> float:
    """Accuracy metric max_ij |C - C^|_ij / (|A||B|)_ij.  Reading for a zero
    denominator: 0/0 counts as 0, x/0 with x != 0 as infinity."""
    C_hat = np.asarray(C_hat, dtype=np.float64)
    num = np.abs(np.asarray(C_ref, dtype=np.float64) - C_hat)
    den = np.asarray(absab, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(den > 0, num / np.where(den > 0, den, 1.0),
                     np.where(num == 0, 0.0, np.inf))
    r = np.where(np.isnan(num), np.inf, r)
    return float(r.max()) if r.size else 0.0


def tolerance(K: int) -> float:
    """Accuracy bound 2 K u with u = 2^-53 ~= 1.11e-16 for both paths."""
    return 2.0 * K * 1.11e-16
