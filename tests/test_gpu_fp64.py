"""Parity of the native binary64 HSUMMA kernel with the oracle (GPU).

Integer inputs: every partial sum is an integer below 2^53, so C must equal the
oracle bit for bit whatever G, b, B and summation order.  Float inputs: the
accuracy metric max |C - C^| / (|A||B|) against the compensated reference must
stay within 2 K u.  The panel-load counters must equal the oracle's counter
model exactly."""
import numpy as np
import pytest

from oracle import gpu_schedule as gsched
from oracle import native, split
from tests.gpu_util import lib_ready, pair, sample_entries, torch_cuda

pytestmark = pytest.mark.gpu


def run(hs, dA, dB, **kw):
    C = hs.gemm(dA, dB, **kw)
    hs.sync()
    return C.cpu().numpy()


def expected_counters(hs, M, N, K, P, Q, G, Bo, tm=128, tn=128, npairs=1):
    I, J, cm, cn = hs.group_shape(P, Q, G)
    return gsched.counters_closed_form(M, N, K, P, Q, cm, cn, tm, tn, Bo, npairs)


@pytest.mark.parametrize("G", [1, 2, 4, 8, 16])
def test_cfg0_integers_bit_exact_every_G(G):
    hs = lib_ready()
    M = N = K = 512
    A, B, dA, dB = pair(M, N, K, 1000, "smallint")
    C = run(hs, dA, dB, P=4, Q=4, G=G, b=32, Bouter=64)
    assert np.array_equal(C, native.dgemm(A, B))
    c = hs.counters()
    want = expected_counters(hs, M, N, K, 4, 4, G, 64)
    for k, v in want.items():
        assert c[k] == v, (k, c[k], v)


def test_cfg0_uniform_within_bound():
    hs = lib_ready()
    M = N = K = 512
    A, B, dA, dB = pair(M, N, K, 1000, "uniform")
    C = run(hs, dA, dB, P=4, Q=4, G=4, b=32, Bouter=64)
    ref, absab = native.dot2_full(A, B)
    err = split.max_rel_error(C, ref, absab)
    assert err <= split.tolerance(K), err
    # and within the textbook bound of the triple loop's own result
    C0 = native.dgemm(A, B)
    assert np.max(np.abs(C - C0) / absab) <= 2 * K * 2.0 ** -53


@pytest.mark.parametrize("M,N,K,P,Q,G,b,Bo", [
    (300, 520, 700, 3, 4, 2, 16, 64),        # ragged blocks, sub-tiles and K
    (300, 520, 700, 3, 4, 12, 32, 32),       # G = p
    (1152, 700, 96, 5, 4, 5, 16, 48),        # ragged, 5 x 1 groups
    (9, 10, 5, 4, 4, 4, 16, 16),             # empty last block row
    (1, 1, 1, 1, 1, 1, 16, 16),
    (257, 129, 1000, 1, 1, 1, 64, 128),      # one CTA sweeping 3 x 2 sub-tiles
    (640, 640, 256, 8, 2, 4, 16, 64),        # in-group 2 x 2 clusters with 4-wide pieces
])
def test_ragged_integers_bit_exact(M, N, K, P, Q, G, b, Bo):
    hs = lib_ready()
    A, B, dA, dB = pair(M, N, K, 77, "smallint")
    C = run(hs, dA, dB, P=P, Q=Q, G=G, b=b, Bouter=Bo)
    assert np.array_equal(C, native.dgemm(A, B))
    c = hs.counters()
    want = expected_counters(hs, M, N, K, P, Q, G, Bo)
    for k, v in want.items():
        assert c[k] == v, (k, c[k], v)


def test_sixteen_cta_cluster_and_summa_equivalence():
    # 4 x 4 grid, G = 1: the whole grid is one group of 16 (one cluster);
    # G = 16: flat.  Both are SUMMA (Section III) and give identical C.
    hs = lib_ready()
    A, B, dA, dB = pair(512, 512, 512, 5, "smallint")
    C1 = run(hs, dA, dB, P=4, Q=4, G=1, b=16, Bouter=16)
    assert hs.group_shape(4, 4, 1)[2:] in ((4, 4), (1, 1))
    C16 = run(hs, dA, dB, P=4, Q=4, G=16, b=16, Bouter=16)
    assert np.array_equal(C1, C16)
    assert np.array_equal(C1, native.dgemm(A, B))


def test_empty_and_zero_k():
    hs = lib_ready()
    torch = torch_cuda()
    A, B, dA, dB = pair(8, 8, 0, 3, "uniform")
    dA = torch.zeros((8, 0), dtype=torch.float64, device="cuda")
    dB = torch.zeros((0, 8), dtype=torch.float64, device="cuda")
    C = hs.gemm(dA, dB, P=2, Q=2, G=1, b=16, Bouter=16)
    hs.sync()
    assert torch.all(C == 0)
    dA = torch.zeros((0, 8), dtype=torch.float64, device="cuda")
    dB = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    C = hs.gemm(dA, dB, P=2, Q=2, G=1, b=16, Bouter=16)
    hs.sync()
    assert C.shape == (0, 4)


def test_argument_errors():
    hs = lib_ready()
    torch = torch_cuda()
    _, _, dA, dB = pair(64, 64, 64, 3, "uniform")
    for kw, code in [(dict(P=4, Q=4, G=3, b=16, Bouter=16), -1),      # no factorisation
                     (dict(P=4, Q=4, G=4, b=24, Bouter=48), -1),      # b not a multiple of 16
                     (dict(P=4, Q=4, G=4, b=32, Bouter=48), -1),      # b does not divide B
                     (dict(P=0, Q=4, G=1, b=16, Bouter=16), -1)]:
        with pytest.raises(hs.HsummaError) as ei:
            hs.gemm(dA, dB, **kw)
        assert ei.value.status == code
    # a base that is not 8-byte aligned is rejected before any device access
    dC = torch.empty((64, 64), dtype=torch.float64, device="cuda")
    st = hs.lib().hsumma_gemm(64, 64, 64, dA.data_ptr() + 4, 64, dB.data_ptr(), 64,
                              dC.data_ptr(), 64, 1, 1, 1, 16, 16, 0, None)
    assert st == -1 and "aligned" in hs.last_error()
    # a leading dimension below the row length
    st = hs.lib().hsumma_gemm(64, 64, 64, dA.data_ptr(), 63, dB.data_ptr(), 64,
                              dC.data_ptr(), 64, 1, 1, 1, 16, 16, 0, None)
    assert st == -1


def test_host_buffers_entry():
    hs = lib_ready()
    torch = torch_cuda()
    A, B, _, _ = pair(200, 300, 128, 9, "smallint")
    C = np.zeros((200, 300))
    hs.gemm_host(A, B, C, P=2, Q=3, G=1, b=32, Bouter=64)
    assert np.array_equal(C, native.dgemm(A, B))


@pytest.mark.parametrize("G", [1, 4, 16, 64, 256])
def test_cfg1_8192_sampled_and_counters(G):
    # 8192^3 on the 16 x 16 grid: sampled entries against the compensated
    # reference, counters against the closed forms
    hs = lib_ready()
    torch = torch_cuda()
    import workloads
    n = 8192
    dA = workloads.matrix_torch(n, n, 1001, "uniform", device="cuda")
    dB = workloads.matrix_torch(n, n, 2001, "uniform", device="cuda")
    C = hs.gemm(dA, dB, P=16, Q=16, G=G, b=64, Bouter=128)
    hs.sync()
    c = hs.counters()
    want = expected_counters(hs, n, n, n, 16, 16, G, 128)
    for k, v in want.items():
        assert c[k] == v, (k, c[k], v)
    if G == 16:
        rows, cols = sample_entries(n, n, 48, 4242)
        A = dA[np.unique(rows)].cpu().numpy()
        rmap = {r: i for i, r in enumerate(np.unique(rows))}
        B = dB.cpu().numpy()
        ref, absab = native.dot2_entries(A, B, [rmap[r] for r in rows], cols)
        got = C[torch.as_tensor(rows, device="cuda"), torch.as_tensor(cols, device="cuda")].cpu().numpy()
        assert split.max_rel_error(got, ref, absab) <= split.tolerance(n)
