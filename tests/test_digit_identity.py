"""The fixed-point digit identity the slicing kernels use (no GPU).

With F = floor(|x| 2^-e 2^64) and p = 63 - w s, the kernels form digit s as
  t_s = (q_s mod 2^w) + c_s - 2^w c_(s-1),   q_s = floor(F / 2^(p+1)),
  c_s = (bit p of F) and (a lower bit of F, a bit dropped below F, or bit p+1),
which must equal the oracle's digits t_s = RN(r 2^(ws)) - 2^w RN(r 2^(w(s-1)))
(r = x 2^-e, round half to even).  This restates the kernels' integer steps
bit for bit (32-bit window, trailing-zero test) and compares them with
oracle.split on random values over the whole exponent range, subnormals,
zeros, and exact ties at every slice boundary, for every slice width."""
import random
import struct

import numpy as np
import pytest

from oracle import split

M64 = (1 << 64) - 1


def kernel_digits(x, e, S, w):
    bits = struct.unpack("<Q", struct.pack("<d", x))[0]
    neg = bits >> 63
    E = (bits >> 52) & 0x7FF
    m = bits & ((1 << 52) - 1)
    if E > 0:
        m |= 1 << 52
        lsb = E - 1075
    else:
        lsb = -1074
    sh = lsb - e + 64
    if sh >= 0:
        F, sticky = (m << min(sh, 63)) & M64, False
    elif sh > -64:
        F, sticky = m >> -sh, ((m << (64 + sh)) & M64) != 0
    else:
        F, sticky = 0, m != 0
    assert F < 2 ** 63                      # |x| 2^-e < 1/2
    tz = -1 if sticky else ((F & -F).bit_length() - 1 if F else 64)
    cprev, out = 0, []
    for s in range(1, S + 1):
        p = 63 - w * s
        win = (F >> p) & 0xFFFFFFFF
        field = (win >> 1) & ((1 << w) - 1)
        c = (win & 1) & int(tz < p or (field & 1) == 1)
        t = field + c - (cprev << w)
        cprev = c
        out.append(-t if neg else t)
    return out


def awkward_rows(seed):
    rnd = random.Random(seed)
    rows = []
    for _ in range(300):
        ex = rnd.randint(-1070, 1000)
        rows.append([rnd.uniform(-1, 1) * 2.0 ** (ex + rnd.randint(-70, 0)) for _ in range(16)])
    for w in (7, 8, 9):
        for s in range(1, 9):
            q = 2.0 ** (-2 - w * s)            # a tie at slice s of a row whose maximum is 0.49
            rows.append([0.49, 0.25 + q, -(0.25 + q), 0.25 + 3 * q, 0.125 + q / 2, 0.0, -0.0,
                         2.0 ** -1074, 1.5e-323, 2.0 ** -1060, 0.3, -0.3, 1e-5, 0.26, 0.126,
                         2.0 ** -30])
    rows.append([2.0 ** -1074 * k for k in range(1, 17)])
    rows.append([0.0] * 16)
    rows.append([2.0 ** 1023 * 1.9] + [2.0 ** (1023 - 8 * k) for k in range(15)])
    return np.array(rows)


@pytest.mark.parametrize("kind,S", [("bf16", 6), ("bf16", 7), ("int8", 8)])
def test_kernel_digit_identity_equals_oracle(kind, S):
    w = split.slice_bits(kind, S)
    A = awkward_rows(11 + w)
    e = split.row_exponents(A)
    ref = split.split_rows(A, e, S, w)          # S x M x K
    for i in range(A.shape[0]):
        for k in range(A.shape[1]):
            got = kernel_digits(float(A[i, k]), int(e[i]), S, w)
            assert got == [int(ref[s, i, k]) for s in range(S)], (A[i, k], e[i])
