"""Launch policies of the CTA-pair bf16 kernel (GPU): one launch for all slice
pairs, one launch per diagonal, and persistent clusters that sweep several
group tiles each give the oracle's exact diagonal sums and the closed-form
counters; and the benchmark's own launch (n = 16384, S = 4, 2 x 1 groups,
B = 512, one launch per diagonal by the library's rule) gives the oracle's
C bit for bit on sampled entries."""
import numpy as np
import pytest

import workloads
from oracle import gpu_schedule as gsched
from oracle import split
from tests.gpu_util import lib_ready, pair, sample_entries, torch_cuda

pytestmark = pytest.mark.gpu


_ORACLE = {}


def _oracle_diagonals(A, B, S):
    key = (A.shape, B.shape, S, A[:2].tobytes(), B[:, :2].tobytes())
    if key in _ORACLE:
        return _ORACLE[key]
    w = split.slice_bits("bf16", S)
    e, f = split.row_exponents(A), split.col_exponents(B)
    _ORACLE.clear()
    _ORACLE[key] = split.diagonal_products(split.split_rows(A, e, S, w),
                                           split.split_cols(B, f, S, w), S, w)
    return _ORACLE[key]


@pytest.mark.parametrize("policy", ["one", "per_diagonal"])
@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("M,N,K,P,Q,G,S,Bo", [
    (1030, 1100, 700, 8, 4, 16, 3, 1024),     # 2 x 1 groups, ragged blocks, B longer than K
    (4096, 4096, 192, 32, 16, 256, 3, 128),   # 2 x 1 groups, 256 tiles: several per cluster
    (600, 1100, 700, 4, 4, 4, 3, 256),        # 2 x 2 groups (two pairs per cluster), ragged
    (4096, 4096, 320, 32, 16, 128, 2, 64),    # 2 x 2 groups, 128 tiles
])
def test_pair_launch_policies_exact(policy, persistent, M, N, K, P, Q, G, S, Bo):
    hs = lib_ready()
    torch = torch_cuda()
    I, J, cm, cn = hs.group_shape(P, Q, G)
    assert (cm, cn) in ((2, 1), (2, 2))
    A, B, dA, dB = pair(M, N, K, 61, "wide", "uniform")
    e, f = hs.split_exponents(dA, dB)
    As, Bs = hs.split_slices(dA, dB, e, f, "bf16", S)
    was_pair = hs.pair_kernel(True)
    was = hs.pair_launch(policy, persistent)
    try:
        n0 = hs.launches()
        D = hs.split_diagonals(As, Bs, M, N, K, "bf16", S, P=P, Q=Q, G=G, b=64, Bouter=Bo)
        hs.sync()
        nl = hs.launches() - n0
        c = hs.counters()
    finally:
        hs.pair_launch(*was)
        hs.pair_kernel(was_pair)
    assert nl == (S if policy == "per_diagonal" else 1)
    want = _oracle_diagonals(A, B, S)
    Dg = D.to(torch.int64).sum(dim=1).cpu().numpy()
    for d in range(2, S + 2):
        assert np.array_equal(Dg[d - 2], want[d]), d
    npairs = S * (S + 1) // 2
    cw = gsched.counters_closed_form(M, N, K, P, Q, cm, cn, 128, 256, Bo, npairs)
    for k, v in cw.items():
        assert c[k] == v, (k, c[k], v)


def test_pair_launch_rejects_unknown_policy():
    hs = lib_ready()
    with pytest.raises(KeyError):
        hs.pair_launch("sideways")
    assert hs.lib().hsumma_pair_launch(0x7) == -1        # split code out of range
    assert hs.lib().hsumma_pair_launch(0x100) == -1      # unknown bit
    assert hs.pair_launch() == ("auto", True)            # unchanged, the default


@pytest.mark.parametrize("S", [4, 5])
def test_bench_launch_bit_exact_at_16384(S):
    # bench.py's split step as it runs: M = N = K = 16384, uniform[-1, 1], bf16
    # S = 4 (S = 5 beside it), a 128 x 64 grid of 128 x 256 blocks, G = 4096
    # groups of 2 x 1 (one CTA pair each), b = 64, B = 512; persistent pair
    # clusters, and at this size the library's rule makes one launch per
    # diagonal (exponent scan 2, slicing 2, products S, recombination 1
    # launches).  Sampled entries, including every corner and tile border, bit
    # for bit against the oracle.
    hs = lib_ready()
    torch = torch_cuda()
    n = 16384
    assert hs.pair_launch() == ("auto", True) and hs.pair_kernel() is True
    dA = workloads.matrix_torch(n, n, 1002, "uniform", device="cuda")
    dB = workloads.matrix_torch(n, n, 2002, "uniform", device="cuda")
    n0 = hs.launches()
    C = hs.gemm(dA, dB, P=128, Q=64, G=4096, b=64, Bouter=512, kind="bf16", slices=S)
    hs.sync()
    assert hs.launches() - n0 == 2 + 2 + S + 1
    rows, cols = sample_entries(n, n, 48, 123)
    ur, uc = np.unique(rows), np.unique(cols)
    A = dA[torch.as_tensor(ur, device="cuda")].cpu().numpy()
    B = dB[:, torch.as_tensor(uc, device="cuda")].cpu().numpy()
    # whole rows of A and whole columns of B: their exponents are the full ones
    want = split.split_entries(A, B, np.searchsorted(ur, rows), np.searchsorted(uc, cols), S,
                               "bf16")
    got = C[torch.as_tensor(rows, device="cuda"),
            torch.as_tensor(cols, device="cuda")].cpu().numpy()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("kind,S,K,P,Q,G,pair_kernel", [
    ("bf16", 3, 43328, 2, 1, 1, True),    # CTA pair: diagonal 4 has five segments
    ("bf16", 3, 43328, 2, 1, 2, False),   # one CTA each: diagonal 4 has four
    ("bf16", 3, 16384, 2, 1, 1, True),    # diagonal 2 has one segment, 3 and 4 two
    ("int8", 3, 87360, 2, 2, 4, False),   # int8: diagonal 4 has two segments
])
def test_planes_past_a_diagonals_segments_are_zero(kind, S, K, P, Q, G, pair_kernel):
    # K large enough for several int32 planes per diagonal; the shorter
    # diagonals fill only their first ones, and the kernels must write the rest
    # as zeros (a caller of step 3 may add every plane).  The sums' buffer
    # starts out dirty.  (The 128-column stages of the CTA pairs pad a pair's
    # odd last panel: at K = 43328 that gives diagonal 4 one segment more than
    # the 64-column stages of one CTA.)
    import ctypes
    hs = lib_ready()
    torch = torch_cuda()
    M, N = 256, 256
    A, B, dA, dB = pair(M, N, K, 71, "uniform", "wide")
    e, f = hs.split_exponents(dA, dB)
    As, Bs = hs.split_slices(dA, dB, e, f, kind, S)
    planes = hs.split_planes(K, kind, S)
    assert planes == {43328: 5, 16384: 2, 87360: 2}[K]
    D = torch.full((S, planes, M, N), 0x3f3f3f3f, dtype=torch.int32, device="cuda")
    was = hs.pair_kernel(pair_kernel)
    try:
        hs._check(hs.lib().hsumma_split_diagonals(M, N, K, hs.KINDS[kind], S, As.data_ptr(),
                                                  Bs.data_ptr(), D.data_ptr(), P, Q, G, 128,
                                                  256, None))
        hs.sync(None)
    finally:
        hs.pair_kernel(was)
    w = split.slice_bits(kind, S)
    ee, ff = split.row_exponents(A), split.col_exponents(B)
    want = split.diagonal_products(split.split_rows(A, ee, S, w), split.split_cols(B, ff, S, w),
                                   S, w)
    Dg = D.to(torch.int64).sum(dim=1).cpu().numpy()
    for d in range(2, S + 2):
        assert np.array_equal(Dg[d - 2], want[d]), d
    # each diagonal's own segments: (d - 1) pairs of the kernel's k-stages,
    # segments of 127 exact fp32 chunks (bf16: 2^(26 - 2w) products each) or of
    # 2^18 products (int8); every plane past them is zero
    stage = 64 if kind == "bf16" and not pair_kernel else 128
    seg = 127 * 2 ** (26 - 2 * w) // stage if kind == "bf16" else 2 ** 18 // stage
    nk = -(-(-(-K // 64) * 64) // stage)
    zero_planes = 0
    for d in range(2, S + 2):
        own = -(-((d - 1) * nk) // seg)
        assert own <= planes
        if own < planes:
            assert int(D[d - 2, own:].abs().max()) == 0, d
            zero_planes += planes - own
    assert zero_planes > 0
