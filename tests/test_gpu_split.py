"""Parity of the split-precision path with the oracle (GPU), step by step and
end to end: exponents, digits and recombination bit for bit, diagonal sums
exactly, C bit for bit (the recombination rounds an exact sum once), accuracy
within 2 K u against the compensated reference, and the counters."""
import numpy as np
import pytest

import workloads
from oracle import gpu_schedule as gsched
from oracle import native, split
from tests.gpu_util import lib_ready, pair, sample_entries, torch_cuda

pytestmark = pytest.mark.gpu


def awkward(M, K, seed):
    """Wide-range values with zero rows, subnormals and exact ties."""
    A = workloads.matrix(M, K, seed, "wide")
    A[min(2, M - 1), :] = 0.0
    if M > 4 and K > 3:
        A[4, 1] = 2.0 ** -1070
        A[4, 2] = -(2.0 ** -1074)
        A[3, :] = 2.0 ** -1060 * np.sign(A[3, :])     # a subnormal-scale row
        A[1, 0] = 0.5 + 2.0 ** -9                       # ties in the digits
    return A


@pytest.mark.parametrize("kind", ["bf16", "int8"])
def test_exponents_and_slices_bit_exact(kind):
    hs = lib_ready()
    torch = torch_cuda()
    M, N, K = 70, 90, 130
    A = awkward(M, K, 11)
    B = awkward(N, K, 12).T.copy()
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    e, f = hs.split_exponents(dA, dB)
    hs.sync()
    e_o, f_o = split.row_exponents(A), split.col_exponents(B)
    assert np.array_equal(e.cpu().numpy(), e_o)
    assert np.array_equal(f.cpu().numpy(), f_o)
    S = 8 if kind == "int8" else 7
    As, Bs = hs.split_slices(dA, dB, e, f, kind, S)
    hs.sync()
    w = split.slice_bits(kind, S)
    Ad = split.split_rows(A, e_o, S, w)
    Bd = split.split_cols(B, f_o, S, w)
    Kp = As.shape[2]
    got_a = As.float().cpu().numpy()
    got_b = Bs.float().cpu().numpy()
    assert np.array_equal(got_a[:, :, :K], Ad)
    assert np.all(got_a[:, :, K:] == 0)
    assert np.array_equal(got_b[:, :, :K], np.transpose(Bd, (0, 2, 1)))
    assert np.all(got_b[:, :, K:] == 0)


def bit_patterns(M, K, seed):
    """Rows mixing the cases the digit arithmetic treats apart: values far below
    the row's largest (bits dropped below the 64-bit fixed-point form), raw
    random finite bit patterns, subnormals, exact ties at digit boundaries,
    signed zeros, rows scaled into the subnormal range and all-zero rows."""
    rng = np.random.default_rng(seed)
    A = np.empty((M, K))
    for i in range(M):
        c = rng.random(K)
        row = rng.uniform(-1, 1, K) * np.exp2(rng.integers(-80, 3, K).astype(float))
        raw = rng.integers(0, 2 ** 63, K, dtype=np.int64).view(np.float64)
        raw[~np.isfinite(raw)] = 1.0
        raw *= np.where(rng.random(K) < 0.5, -1.0, 1.0)
        sub = (rng.integers(0, 2 ** 52, K, dtype=np.int64) >> rng.integers(0, 52, K)).view(np.float64)
        tie = (rng.integers(1, 600, K) + 0.5) * np.exp2(rng.integers(-70, -8, K).astype(float))
        special = rng.choice(np.array([0.0, -0.0, 0.5 - 2.0 ** -60, 2.0 ** -1074, -(2.0 ** -1074),
                                       2.0 ** -1022]), K)
        row = np.where(c < 0.55, row, np.where(c < 0.65, raw, np.where(c < 0.75, sub, np.where(
            c < 0.9, tie * np.sign(rng.uniform(-1, 1, K)), special))))
        if i % 7 == 3:
            row = row * 2.0 ** -1000
        if i % 11 == 5:
            row[:] = 0.0
        A[i] = row
    return A


@pytest.mark.parametrize("kind", ["bf16", "int8"])
def test_slices_bit_patterns(kind):
    # every branch of the slicing arithmetic (shifts by less than 0, 0..31 and
    # 32 or more bits; dropped and sticky bits; ties) against the oracle's digits
    hs = lib_ready()
    torch = torch_cuda()
    M, N, K = 96, 80, 200
    A = bit_patterns(M, K, 41)
    B = bit_patterns(N, K, 42).T.copy()
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    e, f = hs.split_exponents(dA, dB)
    S = 8 if kind == "int8" else 7
    As, Bs = hs.split_slices(dA, dB, e, f, kind, S)
    hs.sync()
    w = split.slice_bits(kind, S)
    e_o, f_o = split.row_exponents(A), split.col_exponents(B)
    assert np.array_equal(e.cpu().numpy(), e_o) and np.array_equal(f.cpu().numpy(), f_o)
    got_a = As.float().cpu().numpy()[:, :, :K]
    got_b = Bs.float().cpu().numpy()[:, :, :K]
    assert np.array_equal(got_a, split.split_rows(A, e_o, S, w))
    assert np.array_equal(got_b, np.transpose(split.split_cols(B, f_o, S, w), (0, 2, 1)))


@pytest.mark.parametrize("K,N", [(1, 1), (3, 65), (7, 200), (130, 64), (1000, 130), (4099, 7)])
def test_column_exponents_split_over_k(K, N):
    # the column scan splits k over a cluster of up to 8 CTAs (fewer when K is
    # smaller); the largest entry of a column sits in any of the slices
    hs = lib_ready()
    torch = torch_cuda()
    rng = np.random.default_rng(K + N)
    B = rng.uniform(-1, 1, (K, N)) * np.exp2(rng.integers(-30, 30, (K, N)).astype(float))
    B[rng.integers(0, K, N), np.arange(N)] = 2.0 ** 40 * rng.uniform(0.5, 1, N)
    A = np.ones((2, K))
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    e, f = hs.split_exponents(dA, dB)
    hs.sync()
    assert np.array_equal(f.cpu().numpy(), split.col_exponents(B))
    assert np.array_equal(e.cpu().numpy(), split.row_exponents(A))


def test_nonfinite_is_reported():
    hs = lib_ready()
    torch = torch_cuda()
    A = np.ones((8, 8))
    A[3, 5] = np.inf
    dA = torch.from_numpy(A).cuda()
    with pytest.raises(hs.HsummaError) as ei:
        hs.gemm(dA, dA, P=1, Q=1, G=1, b=64, Bouter=64, kind="bf16", slices=3)
        hs.sync()
    assert ei.value.status == -6
    hs.sync()          # the error word was cleared


@pytest.mark.parametrize("M,N,K,P,Q,G,S", [
    (300, 600, 1000, 3, 3, 9, 3),       # flat, ragged everywhere
    (300, 600, 1000, 3, 3, 1, 2),       # one 3 x 3 cluster: 8-row pieces
    (256, 512, 512, 2, 2, 1, 4),        # one 2 x 2 cluster: contiguous shares
    (512, 1024, 4096, 4, 4, 4, 3),      # 2 x 2 groups, several chunks per diagonal
    (130, 260, 64, 1, 1, 1, 5),         # one CTA, 2 x 2 sub-tiles, ragged
])
def test_bf16_diagonals_exact(M, N, K, P, Q, G, S):
    hs = lib_ready()
    torch = torch_cuda()
    A, B, dA, dB = pair(M, N, K, 21, "uniform", "wide")
    e, f = hs.split_exponents(dA, dB)
    As, Bs = hs.split_slices(dA, dB, e, f, "bf16", S)
    D = hs.split_diagonals(As, Bs, M, N, K, "bf16", S, P=P, Q=Q, G=G, b=64, Bouter=128)
    hs.sync()
    _, parts = split.split_gemm(A, B, S, "bf16", return_parts=True)
    Dg = D.to(torch.int64).sum(dim=1).cpu().numpy()
    for d in range(2, S + 2):
        assert np.array_equal(Dg[d - 2], parts["D"][d]), d
    npairs = S * (S + 1) // 2
    I, J, cm, cn = hs.group_shape(P, Q, G)
    want = gsched.counters_closed_form(M, N, K, P, Q, cm, cn, 128, 256, 128, npairs)
    c = hs.counters()
    for k, v in want.items():
        assert c[k] == v, (k, c[k], v)


@pytest.mark.parametrize("S", [2, 7])
@pytest.mark.parametrize("P", [1, 2])
def test_bf16_exact_at_the_fp32_bound(S, P):
    # every digit at its largest magnitude 2^(w-1) (256 with w = 9 at S = 2,
    # 128 with w = 8 at S = 7): products 2^(2w-2), chunk sums reach exactly
    # 2^24 -- the fp32 accumulator must still be exact, and the drain's
    # add-based conversion (exact below 2^22) must give way to the conversion
    # instruction.  P = 1: one CTA; P = 2: one CTA pair.
    hs = lib_ready()
    torch = torch_cuda()
    M, N, K = 256, 256, 2048
    w = split.slice_bits("bf16", S)
    A = np.full((M, K), 0.5 - 2.0 ** -20)          # r 2^w rounds to 2^(w-1)
    A[1::2] *= -1.0
    B = np.full((K, N), 0.5 - 2.0 ** -20)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    e, f = hs.split_exponents(dA, dB)
    As, Bs = hs.split_slices(dA, dB, e, f, "bf16", S)
    assert As.float().abs().max().item() == 2.0 ** (w - 1)
    D = hs.split_diagonals(As, Bs, M, N, K, "bf16", S, P=P, Q=1, G=1, b=64, Bouter=64)
    hs.sync()
    _, parts = split.split_gemm(A, B, S, "bf16", return_parts=True)
    Dg = D.to(torch.int64).sum(dim=1).cpu().numpy()
    assert abs(int(parts["D"][2][0, 0])) == K * 4 ** (w - 1)
    for d in range(2, S + 2):
        assert np.array_equal(Dg[d - 2], parts["D"][d]), d


@pytest.mark.parametrize("kind,S,dist", [("bf16", 3, "uniform"), ("bf16", 5, "wide"),
                                         ("bf16", 6, "uniform")])
def test_gemm_bit_exact_with_oracle(kind, S, dist):
    hs = lib_ready()
    M, N, K = 200, 300, 700
    A, B, dA, dB = pair(M, N, K, 31, dist)
    C = hs.gemm(dA, dB, P=2, Q=2, G=1, b=64, Bouter=128, kind=kind, slices=S)
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), split.split_gemm(A, B, S, kind))


def test_recombine_special_values():
    # exact integer digits chosen to make the rounding interesting: ties,
    # subnormal and overflowing results
    hs = lib_ready()
    torch = torch_cuda()
    M, N, S = 4, 3, 3
    D = np.zeros((S, 1, M, N), dtype=np.int32)
    D[0, 0] = [[1, 3, -5], [2 ** 30, -(2 ** 30), 7], [0, 1, 1], [123456789, -987654321, 5]]
    D[1, 0] = [[1, 0, 1], [255, 256, -1], [0, 0, 1], [77, 1, -2 ** 31 + 1]]
    D[2, 0] = [[-1, 2 ** 20, 0], [1, -1, 2 ** 31 - 1], [1, 0, -1], [0, 0, 0]]
    e = np.array([0, 2000, -1060, 5], dtype=np.int32)
    f = np.array([0, -3, 1000], dtype=np.int32)
    dD = torch.from_numpy(D).cuda()
    de, df = torch.from_numpy(e).cuda(), torch.from_numpy(f).cuda()
    C = hs.split_recombine(dD, de, df, M, N, 64, "bf16", S)
    hs.sync()
    Dd = {d: D[d - 2, 0].astype(np.int64) for d in range(2, S + 2)}
    want = split.recombine(Dd, e, f, S, split.slice_bits("bf16", S))
    got = C.cpu().numpy()
    assert np.array_equal(np.isinf(got), np.isinf(want))
    fin = np.isfinite(want)
    assert np.array_equal(got[fin], want[fin])


@pytest.mark.parametrize("kind,S", [("bf16", 5), ("bf16", 6), ("int8", 6), ("int8", 7)])
def test_recombine_64_and_128_bit_paths(kind, S):
    # one segment plane per diagonal (K = 64): most entries take the 64-bit
    # path; |D_2| near 2^31 and the int32 extremes in the other diagonals force
    # the 128-bit one (bf16 S = 6 and int8 S = 7 always take it), alone and
    # next to 64-bit entries in the same group of four columns
    hs = lib_ready()
    torch = torch_cuda()
    M, N = 9, 37
    rng = np.random.default_rng(S * 10 + len(kind))
    D = rng.integers(-2 ** 24, 2 ** 24, size=(S, 1, M, N)).astype(np.int32)
    D[0, 0, 1, 5] = 2 ** 31 - 1
    D[0, 0, 2, 0:4] = -(2 ** 31)
    D[0, 0, 3, 9] = 2 ** 28 + 12345
    D[1:, 0, 4, :] = 2 ** 31 - 1
    D[1:, 0, 5, :] = -(2 ** 31)
    D[0, 0, 6, 12:16] = 2 ** 27 - 1
    e = rng.integers(-40, 40, M).astype(np.int32)
    f = rng.integers(-40, 40, N).astype(np.int32)
    dD = torch.from_numpy(D).cuda()
    de, df = torch.from_numpy(e).cuda(), torch.from_numpy(f).cuda()
    C = hs.split_recombine(dD, de, df, M, N, 64, kind, S)
    hs.sync()
    w = split.slice_bits(kind, S)
    want = split.recombine({d: D[d - 2, 0].astype(np.int64) for d in range(2, S + 2)}, e, f, S, w)
    assert np.array_equal(C.cpu().numpy(), want)


def _own_planes(K, kind, S, d):
    """Segment planes diagonal d fills: (d - 1) pairs of K rounded up to the
    128-column stages, cut into segments of 127 exact fp32 chunks (bf16:
    2^(26 - 2w) products each) or of 2^18 products (int8)."""
    k128 = -(-(-(-K // 64) * 64) // 128) * 128
    seg = 127 * 2 ** (26 - 2 * split.slice_bits(kind, S)) if kind == "bf16" else 2 ** 18
    return max(1, -(-((d - 1) * k128) // seg))


@pytest.mark.parametrize("kind,S,K,M,N", [
    ("bf16", 3, 70000, 5, 37),     # diagonals fill 3 / 5 / 7 planes; ragged rows of C
    ("bf16", 4, 40000, 4, 64),     # 2 / 3 / 4 / 5 planes; 16-byte rows
    ("bf16", 6, 33000, 3, 20),     # every diagonal past one plane; 128-bit path only
    ("int8", 3, 300000, 4, 36),    # 2 / 3 / 4 planes
])
def test_recombine_several_planes_per_diagonal(kind, S, K, M, N):
    # a diagonal's exact sum spread over several int32 planes, the first
    # diagonal's too: the recombination must add exactly its own planes (the
    # planes past them hold garbage here, which it must not read), on the 64-
    # and the 128-bit path
    hs = lib_ready()
    torch = torch_cuda()
    planes = hs.split_planes(K, kind, S)
    own = [_own_planes(K, kind, S, d) for d in range(2, S + 2)]
    assert own[-1] == planes and own[0] >= 2
    rng = np.random.default_rng(K + S)
    D = np.full((S, planes, M, N), 0x3F3F3F3F, dtype=np.int32)
    for i, n in enumerate(own):
        D[i, :n] = rng.integers(-2 ** 20, 2 ** 20, size=(n, M, N))
    # full-range planes in one row: sums past 2^31 (the 128-bit path at S = 6,
    # where the other diagonals alone can pass 2^63)
    D[:, :, 1, :] = rng.integers(-2 ** 31, 2 ** 31, size=(S, planes, N))
    D[0, 0, 2, :] = 2 ** 31 - 1
    e = rng.integers(-40, 40, M).astype(np.int32)
    f = rng.integers(-40, 40, N).astype(np.int32)
    dD = torch.from_numpy(D).cuda()
    de, df = torch.from_numpy(e).cuda(), torch.from_numpy(f).cuda()
    C = hs.split_recombine(dD, de, df, M, N, K, kind, S)
    hs.sync()
    sums = {d: D[d - 2, :own[d - 2]].astype(np.int64).sum(axis=0) for d in range(2, S + 2)}
    want = split.recombine(sums, e, f, S, split.slice_bits(kind, S))
    got = C.cpu().numpy()
    assert np.array_equal(np.isinf(got), np.isinf(want))
    fin = np.isfinite(want)
    assert np.array_equal(got[fin], want[fin])


def test_accuracy_within_bound_bf16_S5():
    hs = lib_ready()
    M, N, K = 256, 256, 4096
    A, B, dA, dB = pair(M, N, K, 1002, "uniform")
    C = hs.gemm(dA, dB, P=2, Q=1, G=1, b=64, Bouter=256, kind="bf16", slices=5)
    hs.sync()
    ref, absab = native.dot2_full(A, B)
    assert split.max_rel_error(C.cpu().numpy(), ref, absab) <= split.tolerance(K)


def test_full_size_16384_sampled():
    # the bench workload: M = N = K = 16384, bf16 S = 5, 128 x 64 grid of
    # 128 x 256 blocks in 2 x 2 groups; sampled entries bit for bit against the
    # oracle, and within 2 K u of the compensated reference
    hs = lib_ready()
    torch = torch_cuda()
    n, S = 16384, 5
    dA = workloads.matrix_torch(n, n, 1002, "uniform", device="cuda")
    dB = workloads.matrix_torch(n, n, 2002, "uniform", device="cuda")
    C = hs.gemm(dA, dB, P=128, Q=64, G=2048, b=64, Bouter=256, kind="bf16", slices=S)
    hs.sync()
    rows, cols = sample_entries(n, n, 40, 99)
    ur = np.unique(rows)
    uc = np.unique(cols)
    A = dA[torch.as_tensor(ur, device="cuda")].cpu().numpy()
    B = dB[:, torch.as_tensor(uc, device="cuda")].cpu().numpy()
    ri = np.searchsorted(ur, rows)
    ci = np.searchsorted(uc, cols)
    # the exponents use whole rows of A and whole columns of B: the sampled
    # rows/columns carry them entirely
    want = split.split_entries(A, B, ri, ci, S, "bf16")
    got = C[torch.as_tensor(rows, device="cuda"), torch.as_tensor(cols, device="cuda")].cpu().numpy()
    assert np.array_equal(got, want)
    ref, absab = native.dot2_entries(A, B, ri, ci)
    assert split.max_rel_error(got, ref, absab) <= split.tolerance(n)


@pytest.mark.parametrize("M,N,K,P,Q,G,S", [
    (300, 600, 1000, 3, 3, 9, 3),
    (300, 600, 1000, 3, 3, 1, 2),
    (512, 512, 4096, 4, 4, 4, 6),
    (130, 260, 64, 1, 1, 1, 8),
])
def test_int8_diagonals_exact(M, N, K, P, Q, G, S):
    hs = lib_ready()
    torch = torch_cuda()
    A, B, dA, dB = pair(M, N, K, 23, "wide", "uniform")
    e, f = hs.split_exponents(dA, dB)
    As, Bs = hs.split_slices(dA, dB, e, f, "int8", S)
    D = hs.split_diagonals(As, Bs, M, N, K, "int8", S, P=P, Q=Q, G=G, b=128, Bouter=256)
    hs.sync()
    _, parts = split.split_gemm(A, B, S, "int8", return_parts=True)
    Dg = D.to(torch.int64).sum(dim=1).cpu().numpy()
    for d in range(2, S + 2):
        assert np.array_equal(Dg[d - 2], parts["D"][d]), d
    npairs = S * (S + 1) // 2
    I, J, cm, cn = hs.group_shape(P, Q, G)
    want = gsched.counters_closed_form(M, N, K, P, Q, cm, cn, 128, 128, 256, npairs)
    c = hs.counters()
    for k, v in want.items():
        assert c[k] == v, (k, c[k], v)


@pytest.mark.parametrize("S,dist", [(6, "uniform"), (8, "wide")])
def test_int8_gemm_bit_exact_with_oracle(S, dist):
    hs = lib_ready()
    M, N, K = 200, 300, 700
    A, B, dA, dB = pair(M, N, K, 37, dist)
    C = hs.gemm(dA, dB, P=2, Q=2, G=1, b=128, Bouter=256, kind="int8", slices=S)
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), split.split_gemm(A, B, S, "int8"))


def test_odd_leading_dimensions():
    hs = lib_ready()
    torch = torch_cuda()
    M, N, K = 37, 41, 53
    A, B, _, _ = pair(M, N, K, 41, "smallint")
    # views with odd leading dimensions and an 8-byte (not 16-byte) aligned base
    bigA = torch.zeros((M, K + 2), dtype=torch.float64, device="cuda")
    bigB = torch.zeros((K, N + 2), dtype=torch.float64, device="cuda")
    dA = bigA[:, 1:K + 1]
    dB = bigB[:, 1:N + 1]
    dA.copy_(torch.from_numpy(A))
    dB.copy_(torch.from_numpy(B))
    C = hs.gemm(dA, dB, P=2, Q=2, G=1, b=16, Bouter=32)
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), native.dgemm(A, B))
    C = hs.gemm(dA, dB, P=2, Q=2, G=4, b=64, Bouter=64, kind="bf16", slices=2)
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), split.split_gemm(A, B, 2, "bf16"))


@pytest.mark.parametrize("M,N,K,P,Q,G,S,Bo", [
    (256, 256, 1024, 2, 1, 1, 3, 128),        # one CTA pair
    (600, 700, 640, 4, 3, 6, 2, 128),         # 2 x 1 groups, ragged blocks and sub-tiles
    (1030, 1100, 700, 8, 4, 16, 3, 1024),     # 2 x 1 groups, B longer than K
    (512, 2048, 4096, 2, 4, 4, 4, 256),       # several chunks per diagonal
    (256, 512, 640, 2, 2, 1, 3, 128),         # one 2 x 2 group: two pairs, A multicast
    (600, 1100, 700, 4, 4, 4, 3, 256),        # 2 x 2 groups, ragged blocks and sub-tiles
    (1030, 1000, 900, 8, 4, 8, 2, 1024),      # 2 x 2 groups, B longer than K
    (512, 1024, 4096, 2, 2, 1, 4, 512),       # 2 x 2, several chunks per diagonal
])
def test_bf16_pair_kernel_exact(M, N, K, P, Q, G, S, Bo):
    # groups realised as 2 x 1 or 2 x 2 clusters run on CTA pairs when asked
    hs = lib_ready()
    torch = torch_cuda()
    I, J, cm, cn = hs.group_shape(P, Q, G)
    assert (cm, cn) in ((2, 1), (2, 2))
    A, B, dA, dB = pair(M, N, K, 29, "wide", "uniform")
    e, f = hs.split_exponents(dA, dB)
    As, Bs = hs.split_slices(dA, dB, e, f, "bf16", S)
    was = hs.pair_kernel(True)
    try:
        D = hs.split_diagonals(As, Bs, M, N, K, "bf16", S, P=P, Q=Q, G=G, b=64, Bouter=Bo)
        hs.sync()
        c = hs.counters()
    finally:
        hs.pair_kernel(was)
    _, parts = split.split_gemm(A, B, S, "bf16", return_parts=True)
    Dg = D.to(torch.int64).sum(dim=1).cpu().numpy()
    for d in range(2, S + 2):
        assert np.array_equal(Dg[d - 2], parts["D"][d]), d
    npairs = S * (S + 1) // 2
    want = gsched.counters_closed_form(M, N, K, P, Q, cm, cn, 128, 256, Bo, npairs)
    for k, v in want.items():
        assert c[k] == v, (k, c[k], v)


def test_pair_kernel_gemm_matches_single_cta_kernel():
    hs = lib_ready()
    torch = torch_cuda()
    A, B, dA, dB = pair(1500, 1300, 900, 33, "uniform", "wide")
    cfg = dict(P=12, Q=6, G=36, b=64, Bouter=256, kind="bf16", slices=5)
    assert hs.group_shape(12, 6, 36)[2:] == (2, 1)
    was = hs.pair_kernel(True)
    try:
        C2 = hs.gemm(dA, dB, **cfg)
        hs.pair_kernel(False)
        C1 = hs.gemm(dA, dB, **cfg)
        hs.sync()
    finally:
        hs.pair_kernel(was)
    assert torch.equal(C1, C2)
    assert np.array_equal(C2.cpu().numpy(), split.split_gemm(A, B, 5, "bf16"))


def test_stage_timing_records_each_call():
    hs = lib_ready()
    torch = torch_cuda()
    A, B, dA, dB = pair(512, 768, 640, 41)
    hs.stage_timing(True)
    hs.gemm(dA, dB, P=4, Q=3, G=1, b=64, Bouter=256, kind="bf16", slices=3)
    hs.gemm(dA, dB, P=4, Q=6, G=4, b=32, Bouter=128)
    hs.stage_timing(False)
    hs.gemm(dA, dB, P=4, Q=6, G=4, b=32, Bouter=128)       # not recorded
    ms, calls = hs.stage_times()
    hs.sync()
    assert calls == 2
    assert all(t > 0 for t in ms)                           # every split stage ran
    hs.stage_timing(True)
    hs.gemm(dA, dB, P=4, Q=6, G=4, b=32, Bouter=128)
    hs.stage_timing(False)
    ms, calls = hs.stage_times()
    assert calls == 1 and ms[2] > 0
    assert ms[0] < 0.01 and ms[1] < 0.01 and ms[3] < 0.01   # binary64: one kernel


@pytest.mark.parametrize("kind,S,M,N,K,P,Q,G,pinned", [
    ("fp64", 0, 4000, 900, 640, 16, 4, 16, False),     # 4 row blocks of 1000 rows
    ("fp64", 0, 3001, 700, 512, 12, 4, 12, True),      # 3 blocks, the last one short
    ("bf16", 5, 4100, 1000, 900, 32, 4, 32, True),     # split path, 4 blocks, ragged
    ("int8", 6, 2100, 520, 700, 16, 4, 16, False),     # 2 blocks
])
def test_host_entry_pipelined_by_row_blocks(kind, S, M, N, K, P, Q, G, pinned):
    hs = lib_ready()
    torch = torch_cuda()
    dist = "smallint" if kind == "fp64" else "uniform"
    A = workloads.matrix(M, K, 51, dist)
    B = workloads.matrix(K, N, 52, "wide" if kind != "fp64" else dist)
    big = np.full((M, N + 8), 7.0)                   # C with padding the call must not touch
    hC = big[:, :N]
    if pinned:
        A = torch.from_numpy(A).pin_memory()
        B = torch.from_numpy(B).pin_memory()
    b = 32 if kind == "fp64" else (64 if kind == "bf16" else 128)
    hs.gemm_host(A, B, hC, P=P, Q=Q, G=G, b=b, Bouter=4 * b, kind=kind, slices=S)
    An = A.numpy() if pinned else A
    Bn = B.numpy() if pinned else B
    if kind == "fp64":
        want = (An.astype(np.int64) @ Bn.astype(np.int64)).astype(np.float64)
    else:
        want = split.split_gemm(An, Bn, S, kind)
    assert np.array_equal(hC, want)
    assert np.all(big[:, N:] == 7.0)


def test_a_wait_that_runs_out_is_reported_and_cleared():
    # the bounded-wait machinery itself: a barrier nothing arrives on, a 2 ms
    # limit, the status word read and cleared by hsumma_sync, the context usable
    hs = lib_ready()
    torch = torch_cuda()
    hs._check(hs.lib().hsumma_selftest_timeout(2_000_000, None))
    with pytest.raises(hs.HsummaError) as ei:
        hs.sync(None)
    assert ei.value.status == -4
    assert "self-test wait" in str(ei.value)
    hs.sync(None)                                   # cleared
    with pytest.raises(hs.HsummaError):
        hs._check(hs.lib().hsumma_selftest_timeout(2_000_000_000, None))   # limit too long
    A, B, dA, dB = pair(200, 300, 700, 31, "uniform")
    C = hs.gemm(dA, dB, P=2, Q=2, G=1, b=64, Bouter=128, kind="bf16", slices=3)
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), split.split_gemm(A, B, 3, "bf16"))


@pytest.mark.parametrize("kind,S,P,Q,G,dist", [
    ("bf16", 3, 16, 8, 64, "wide"),        # 2 x 1 groups on CTA pairs
    ("fp64", 0, 16, 16, 16, "smallint"),   # 4 x 4 clusters
])
def test_host_entry_pipelined_in_two_dimensions(kind, S, P, Q, G, dist):
    # 4 row blocks x 2 column blocks: B_0 and A_0 first, each block after its
    # own operands; the timeline lists every phase in order and C is the
    # unblocked product bit for bit
    hs = lib_ready()
    torch = torch_cuda()
    M, N = 2048, 1032          # ragged column blocks (the second one is shorter)
    K = 700 if kind == "bf16" else 512
    A = torch.from_numpy(workloads.matrix(M, K, 57, dist)).pin_memory()
    B = torch.from_numpy(workloads.matrix(K, N, 58, dist)).pin_memory()
    big = np.full((M, N + 8), 7.0)
    hC = big[:, :N]
    b = 64 if kind == "bf16" else 32
    hs.stage_timing(True)
    try:
        hs.gemm_host(A, B, hC, P=P, Q=Q, G=G, b=b, Bouter=4 * b, kind=kind, slices=S)
        tl = hs.host_timeline()
    finally:
        hs.stage_timing(False)
    names = [(nm, r, c) for nm, r, c, _, _ in tl]
    assert names[:6] == [("B in", -1, 0), ("B in", -1, 1), ("A in", 0, -1), ("A in", 1, -1),
                         ("A in", 2, -1), ("A in", 3, -1)]
    prods = [(r, c) for nm, r, c in names if nm == "product"]
    assert prods == [(r, c) for r in range(4) for c in range(2)]
    assert len(tl) == 2 + 4 + 2 * 8
    t = {(nm, r, c): (a, e) for nm, r, c, a, e in tl}
    # the first block starts once B_0 is in (its scan and slicing overlap A_0's
    # copy) and cannot finish before A_0 is in
    assert t[("product", 0, 0)][0] >= t[("B in", -1, 0)][1] - 1e-3
    assert t[("product", 0, 0)][1] >= t[("A in", 0, -1)][1] - 1e-3
    if kind == "fp64":
        want = (A.numpy().astype(np.int64) @ B.numpy().astype(np.int64)).astype(np.float64)
    else:
        want = split.split_gemm(A.numpy(), B.numpy(), S, kind)
    assert np.array_equal(hC, want)
    assert np.all(big[:, N:] == 7.0)


def test_host_entry_row_blocks_in_whole_rounds():
    # bf16 on persistent CTA pairs (2 x 1 groups): the row blocks after the
    # first span whole rounds of the resident pair clusters and the first
    # takes the remaining tile rows; with 40 x 8 processors, two column blocks
    # of 4 and 76 resident clusters that is 2 + 38 processor rows (256 + 4864
    # rows).  Every row block of A is copied before B_1, the products sweep
    # column block 0 down and column block 1 back up (the small first row
    # block's product last), and C matches the oracle bit for bit
    # on sampled entries (every block border among them).
    hs = lib_ready()
    torch_cuda()
    import torch
    M, N, K, S = 5120, 2048, 320, 3
    A = torch.from_numpy(workloads.matrix(M, K, 91, "wide")).pin_memory()
    B = torch.from_numpy(workloads.matrix(K, N, 92, "wide")).pin_memory()
    hC = torch.empty((M, N), dtype=torch.float64).pin_memory()
    hs.stage_timing(True)
    try:
        hs.gemm_host(A, B, hC, P=40, Q=8, G=160, b=64, Bouter=128, kind="bf16", slices=S)
        tl = hs.host_timeline()
    finally:
        hs.stage_timing(False)
    row0 = hs.host_row_blocks()
    assert len(row0) >= 2 and row0[0] == 0
    assert all(r % 256 == 0 for r in row0) and row0 == sorted(row0)
    sizes = [b - a for a, b in zip(row0, row0[1:] + [M])]
    assert sizes[0] < sizes[1] and all(s == sizes[1] for s in sizes[1:-1])
    t = {(nm, r, c): (a, e) for nm, r, c, a, e in tl}
    R = len(row0)
    assert t[("A in", R - 1, -1)][1] <= t[("B in", -1, 1)][0] + 1e-3
    sweep = [(r, 0) for r in range(R)] + [(r, 1) for r in reversed(range(R))]
    starts = [t[("product", r, c)][0] for r, c in sweep]
    assert starts == sorted(starts)
    rows, cols = sample_entries(M, N, 64, 93)
    edges = np.array([min(M - 1, max(0, r + d)) for r in row0 for d in (-1, 0, 1)])
    rows = np.concatenate([rows, edges])
    cols = np.concatenate([cols, np.resize(np.array([0, 1023, 1024, 2047]), len(edges))])
    want = split.split_entries(A.numpy(), B.numpy(), rows, cols, S, "bf16")
    assert np.array_equal(hC.numpy()[rows, cols], want)


@pytest.mark.parametrize("kind,S", [("bf16", 3), ("int8", 4)])
def test_empty_and_zero_k_split_and_host(kind, S):
    # K = 0 gives C = 0 (every sum empty); M = 0 or N = 0 gives an empty C;
    # the same through the host-buffer entry
    hs = lib_ready()
    torch = torch_cuda()
    cfg = dict(P=2, Q=2, G=2, b=64, Bouter=128, kind=kind, slices=S)
    dA = torch.zeros((256, 0), dtype=torch.float64, device="cuda")
    dB = torch.zeros((0, 512), dtype=torch.float64, device="cuda")
    C = torch.full((256, 512), 5.0, dtype=torch.float64, device="cuda")
    hs.gemm(dA, dB, out=C, **cfg)
    hs.sync()
    assert torch.all(C == 0)
    for M, N in ((0, 512), (256, 0)):
        dA = torch.ones((M, 64), dtype=torch.float64, device="cuda")
        dB = torch.ones((64, N), dtype=torch.float64, device="cuda")
        C = hs.gemm(dA, dB, **cfg)
        hs.sync()
        assert C.shape == (M, N)
    hA = torch.zeros((256, 0), dtype=torch.float64).pin_memory()
    hB = torch.zeros((0, 512), dtype=torch.float64).pin_memory()
    hC = np.full((256, 512), 5.0)
    hs.gemm_host(hA, hB, hC, **cfg)
    assert np.all(hC == 0)
    # one row and one column: a 1 x 1 C from a 1 x K by K x 1 product
    A, B, dA, dB = pair(1, 1, 300, 97, "wide")
    C = hs.gemm(dA, dB, P=1, Q=1, G=1, b=64, Bouter=64, kind=kind, slices=S)
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), split.split_gemm(A, B, S, kind))


@pytest.mark.parametrize("kind,P,Q,G,pair_kernel", [
    ("bf16", 4, 2, 4, True),      # 2 x 1 groups on CTA pairs
    ("bf16", 4, 2, 8, False),     # one CTA per processor
    ("int8", 4, 4, 4, False),
])
def test_one_slice_and_slice_count_limits(kind, P, Q, G, pair_kernel):
    # S = 1: the single pair (1, 1), one diagonal, bit for bit; S = 0 and one
    # more than the kind allows are rejected
    hs = lib_ready()
    A, B, dA, dB = pair(500, 400, 300, 101, "wide")
    was = hs.pair_kernel(pair_kernel)
    try:
        C = hs.gemm(dA, dB, P=P, Q=Q, G=G, b=64 if kind == "bf16" else 128,
                    Bouter=128 if kind == "bf16" else 256, kind=kind, slices=1)
        hs.sync()
    finally:
        hs.pair_kernel(was)
    assert np.array_equal(C.cpu().numpy(), split.split_gemm(A, B, 1, kind))
    top = 7 if kind == "bf16" else 8
    for S in (0, top + 1):
        with pytest.raises(hs.HsummaError) as ei:
            hs.gemm(dA, dB, P=P, Q=Q, G=G, b=64 if kind == "bf16" else 128,
                    Bouter=128 if kind == "bf16" else 256, kind=kind, slices=S)
        assert ei.value.status == -1
