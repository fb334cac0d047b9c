"""The block-cyclic layout of the virtual grid (GPU): the distribution the
paper's conclusion (Section VI) leaves to future work, with the sub-tile as the
distribution block.  Every element is the same k-ascending sum in both
layouts, so C must equal the oracle bit for bit on integer inputs (binary64)
and on any finite inputs (split kinds: exact sums, one rounding), and equal the
block layout's C bit for bit on float inputs; the panel-load counters must
equal the oracle's block-cyclic counter model, including clusters that lie
wholly outside the matrix and are skipped."""
import numpy as np
import pytest

from oracle import gpu_schedule as gsched
from oracle import native, split
from tests.gpu_util import lib_ready, pair, torch_cuda

pytestmark = pytest.mark.gpu


def cyclic_counters(hs, M, N, K, P, Q, G, Bo, tm, tn, npairs=1):
    I, J, cm, cn = hs.group_shape(P, Q, G)
    return gsched.counters_closed_form(M, N, K, P, Q, cm, cn, tm, tn, Bo, npairs, cyclic=True)


def check_counters(hs, want):
    c = hs.counters()
    for k, v in want.items():
        assert c[k] == v, (k, c[k], v)


@pytest.mark.parametrize("M,N,K,P,Q,G,b,Bo", [
    (300, 520, 700, 3, 4, 2, 16, 64),        # ragged tiles and K, 3 x 2 clusters
    (1152, 700, 96, 5, 4, 5, 16, 48),        # 5 x 1 groups: 1 x 4 clusters
    (130, 900, 64, 4, 6, 6, 16, 64),         # 2 x 2 clusters, some wholly outside M and N
    (640, 640, 256, 8, 2, 4, 16, 64),        # a cluster whose second row lies outside M
    (9, 10, 5, 4, 4, 4, 16, 16),             # one tile: every other CTA skips
    (257, 129, 1000, 1, 1, 1, 64, 128),      # one CTA sweeping 3 x 2 sub-tiles
    (2000, 1500, 512, 6, 5, 30, 32, 128),    # flat, several tiles per processor
])
def test_fp64_integers_bit_exact_and_counters(M, N, K, P, Q, G, b, Bo):
    hs = lib_ready()
    A, B, dA, dB = pair(M, N, K, 501, "smallint")
    C = hs.gemm(dA, dB, P=P, Q=Q, G=G, b=b, Bouter=Bo, layout="cyclic")
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), native.dgemm(A, B))
    check_counters(hs, cyclic_counters(hs, M, N, K, P, Q, G, Bo, 128, 128))


@pytest.mark.parametrize("G", [1, 16, 144])
def test_fp64_floats_same_bits_as_block_layout(G):
    # 2048 over 12 processor rows: blocks of 171 rows (a 43-row second
    # sub-tile each) against 16 tiles dealt 2, 2, 2, 2, 1, ... (one software
    # group, 3 x 3 clusters, flat)
    hs = lib_ready()
    torch = torch_cuda()
    n = 2048
    _, _, dA, dB = pair(n, n, n, 502, "uniform", "wide")
    cfg = dict(P=12, Q=12, G=G, b=32, Bouter=128)
    Cb = hs.gemm(dA, dB, **cfg)
    Cc = hs.gemm(dA, dB, layout="cyclic", **cfg)
    hs.sync()
    assert torch.equal(Cb, Cc)
    check_counters(hs, cyclic_counters(hs, n, n, n, 12, 12, G, 128, 128, 128))


@pytest.mark.parametrize("M,N,K,P,Q,G,S,pairs", [
    (300, 600, 1000, 3, 3, 9, 3, False),     # flat, ragged everywhere
    (300, 600, 1000, 3, 3, 1, 2, False),     # one 3 x 3 cluster
    (600, 700, 640, 4, 3, 6, 2, True),       # 2 x 1 groups on CTA pairs
    (600, 1100, 700, 4, 4, 4, 3, True),      # 2 x 2 groups: two pairs per cluster
    (130, 1100, 700, 4, 4, 4, 2, True),      # pairs wholly outside M are skipped
    (1030, 1000, 900, 8, 4, 8, 2, False),    # 2 x 2 groups on the single-CTA kernel
])
def test_bf16_bit_exact_and_counters(M, N, K, P, Q, G, S, pairs):
    hs = lib_ready()
    torch = torch_cuda()
    A, B, dA, dB = pair(M, N, K, 503, "wide", "uniform")
    cfg = dict(P=P, Q=Q, G=G, b=64, Bouter=128, kind="bf16", slices=S)
    was = hs.pair_kernel(pairs)
    try:
        Cc = hs.gemm(dA, dB, layout="cyclic", **cfg)
        hs.sync()
        c_cyc = hs.counters()
        Cb = hs.gemm(dA, dB, **cfg)
        hs.sync()
    finally:
        hs.pair_kernel(was)
    assert torch.equal(Cb, Cc)
    assert np.array_equal(Cc.cpu().numpy(), split.split_gemm(A, B, S, "bf16"))
    want = cyclic_counters(hs, M, N, K, P, Q, G, 128, 128, 256, S * (S + 1) // 2)
    for k, v in want.items():
        assert c_cyc[k] == v, (k, c_cyc[k], v)


@pytest.mark.parametrize("M,N,K,P,Q,G,S", [
    (300, 600, 1000, 3, 3, 9, 4),
    (512, 520, 1024, 4, 4, 4, 6),            # 2 x 2 clusters, a column tile short
    (130, 260, 64, 1, 1, 1, 8),
])
def test_int8_bit_exact_and_counters(M, N, K, P, Q, G, S):
    hs = lib_ready()
    A, B, dA, dB = pair(M, N, K, 504, "uniform", "wide")
    C = hs.gemm(dA, dB, P=P, Q=Q, G=G, b=128, Bouter=256, kind="int8", slices=S,
                layout="cyclic")
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), split.split_gemm(A, B, S, "int8"))
    check_counters(hs, cyclic_counters(hs, M, N, K, P, Q, G, 256, 128, 128, S * (S + 1) // 2))


@pytest.mark.parametrize("kind,S,b", [("fp64", 0, 32), ("bf16", 4, 64)])
def test_host_buffers_pipelined(kind, S, b):
    # row blocks of the host-buffer entry each deal their tiles over their own
    # processor rows; the result is the device entry's, bit for bit
    hs = lib_ready()
    torch = torch_cuda()
    M, N, K = 2100, 1000, 700
    A, B, dA, dB = pair(M, N, K, 505, "uniform")
    cfg = dict(P=8, Q=4, G=16, b=b, Bouter=4 * b, kind=kind, slices=S, layout="cyclic")
    Cd = hs.gemm(dA, dB, **cfg)
    hs.sync()
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.empty((M, N), dtype=torch.float64).pin_memory()
    hs.gemm_host(hA, hB, hC, **cfg)
    assert torch.equal(hC, Cd.cpu())
