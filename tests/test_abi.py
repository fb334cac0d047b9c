"""The C-ABI library without a GPU: it builds for sm_103a, loads, exports every
function include/hsumma.h declares, and its host-side logic (group resolution,
workspace sizes, argument errors before initialisation) matches the oracle."""
import ctypes

import pytest

import paper_1306_4161_gb300 as hs
from paper_1306_4161_gb300 import _build
from oracle import gpu_schedule as gs


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return hs.lib()


def test_exports_every_declared_symbol(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", hs.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    declared = set(hs.declared_functions())
    assert declared, "no declarations parsed"
    assert declared <= exported, sorted(declared - exported)
    for name in declared:
        assert hasattr(lib, name)


def test_group_shape_matches_oracle(lib):
    for P, Q in [(4, 4), (16, 16), (12, 16), (5, 7), (128, 64), (2, 8), (1, 1)]:
        for G in range(1, min(P * Q, 300) + 1):
            want = gs.group_shape(P, Q, G)
            if want is None:
                with pytest.raises(hs.HsummaError) as ei:
                    hs.group_shape(P, Q, G)
                assert ei.value.status == -1
                continue
            I, J, cm, cn = hs.group_shape(P, Q, G)
            assert (I, J) == want, (P, Q, G)
            assert (cm, cn) == gs.cluster_shape(P, Q, I, J, limit=16), (P, Q, G)


def test_workspace_sizes(lib):
    assert hs.workspace_size(100, 100, 100, "fp64") == 0
    ws = hs.workspace_size(300, 520, 700, "bf16", 5)
    Kp = 704
    planes = hs.split_planes(700, "bf16", 5)
    assert planes == 1
    al = lambda x: (x + 255) // 256 * 256
    assert ws == al(300 * 4) + al(520 * 4) + al(5 * 300 * Kp * 2) + al(5 * 520 * Kp * 2) + \
        al(5 * planes * 300 * 520 * 4)
    # bf16 digits of 9 bits (S <= 6): a chunk is 256 products, a segment 127
    # chunks (32512 products), so a diagonal of 5 pairs over K = 32768 needs six
    # planes; with 7 slices the digits have 8 bits, a segment is 127 x 1024
    assert hs.split_planes(32768, "bf16", 5) == 6
    assert hs.split_planes(16384, "bf16", 4) == 3
    assert hs.split_planes(16384, "bf16", 7) == 1
    assert hs.split_planes(16384, "int8", 8) == 1


def test_planes_cover_every_kernel_segment(lib):
    # The product kernels cut a diagonal's exact sum into int32 segments of a
    # fixed number of k-stages: 127 chunks of exact fp32 sums for bf16 (a chunk
    # is 2^(26 - 2w) products: 256 for w = 9, 1024 for w = 8), that is 254 or
    # 1016 stages of 128 columns (CTA pairs), 508 or 2032 of 64 (one CTA); 2048
    # stages of 128 for int8; a pair's last stage padded to the stage width.
    # Every segment of the longest diagonal
    # (S pairs) must have a plane: a kernel writing more would write past the
    # sums' storage.  Odd panel counts (Kp / 64 odd) make the 128-column stages
    # longer than Kp; K = 43328, S = 3 and K = 87360, S = 3 are cases where
    # that padding adds a segment.
    cd = lambda a, b: -(-a // b)
    Ks = sorted({64, 700, 4096, 16384, 32768, 43328, 43392, 87360, 87296, 130048, 130112,
                 260032, 260096} | {64 * n for n in range(1, 4000, 37)})
    for K in Ks:
        Kp = cd(K, 64) * 64
        for S in range(1, 8):
            chunk = 2 ** (26 - 2 * (9 if S <= 6 else 8))
            for kind, stage, seg in (("bf16", 128, 127 * chunk // 128),
                                     ("bf16", 64, 127 * chunk // 64), ("int8", 128, 2048)):
                planes = hs.split_planes(K, kind, S)
                segs = cd(S * cd(Kp, stage), seg)
                assert segs <= planes, (K, S, kind, stage, segs, planes)
                # and no plane is wasted beyond one for the padding
                assert planes <= cd(S * Kp, seg * stage) + 1
    # 3 x 43328 = 129984 <= 4 x 32512 < 3 x 43392 (the 128-column stages)
    assert hs.split_planes(43328, "bf16", 3) == 5
    assert hs.split_planes(87360, "int8", 3) == 2


def test_errors_before_init(lib):
    st = lib.hsumma_gemm(4, 4, 4, None, 4, None, 4, None, 4, 1, 1, 1, 16, 16, 0, None)
    assert st == -5
    assert "hsumma_init" in hs.last_error()
    assert lib.hsumma_sync(None) == -5
    with pytest.raises(hs.HsummaError):
        hs.group_shape(0, 4, 1)
    with pytest.raises(hs.HsummaError):
        hs.workspace_size(4, 4, 4, "bf16", 0)       # S out of range
    with pytest.raises(hs.HsummaError):
        hs.workspace_size(4, 4, 4, "int8", 9)
    assert lib.hsumma_split_planes(10, 0, 3) == -1   # not a split kind


def test_mode_encoding():
    assert hs.mode_code("bf16", 5) == 2 | (5 << 8)
    assert hs.mode_code("fp64") == 0
    assert hs.mode_code("int8", 6, "cyclic") == 1 | (6 << 8) | 0x10000
    with pytest.raises(ValueError):
        hs.mode_code("fp64", 0, "diagonal")


def test_layout_bit_accepted_and_other_high_bits_rejected(lib):
    import ctypes
    out = ctypes.c_size_t()
    bf5 = hs.mode_code("bf16", 5)
    assert lib.hsumma_workspace_size(300, 520, 700, bf5 | 0x10000, ctypes.byref(out)) == 0
    assert out.value == hs.workspace_size(300, 520, 700, "bf16", 5)   # the layout adds none
    for bad in (0x20000, 0x40000000, 0x10000 | 0x100000):
        assert lib.hsumma_workspace_size(300, 520, 700, bf5 | bad, ctypes.byref(out)) == -1
        assert "mode" in hs.last_error()
