"""Pins of the group-resolution reading and the GPU counter model (no GPU):
hand-worked group shapes for the 12 x 16 grid, brute-force enumeration against
the closed forms (ragged shapes included), the hand-worked 512^3 counts
(tests/golden/counters_cfg0.txt), and the identity between the counters and the
paper's broadcast volumes at one sub-tile per CTA."""
import os

import pytest

from oracle import gpu_schedule as gs
from oracle import hsumma_sim as hs
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_group_shapes_12x16_worked_by_hand():
    # I*J = G, I | 12, J | 16, most square in-group grid, ties to smaller I
    expect = {1: (1, 1), 3: (3, 1), 4: (2, 2), 12: (3, 4), 16: (4, 4), 48: (6, 8),
              192: (12, 16)}
    for G, IJ in expect.items():
        assert gs.group_shape(12, 16, G) == IJ
    assert gs.group_shape(12, 16, 5) is None
    assert gs.group_shape(12, 16, 7) is None


def test_group_shape_square_grid():
    for G, IJ in {1: (1, 1), 4: (2, 2), 16: (4, 4), 64: (8, 8), 256: (16, 16),
                  2: (1, 2), 8: (2, 4)}.items():
        assert gs.group_shape(16, 16, G) == IJ


def test_group_shape_brute_force():
    import math
    for P, Q in [(4, 4), (6, 4), (12, 16), (5, 7), (8, 2)]:
        for G in range(1, P * Q + 1):
            cands = [(I, G // I) for I in range(1, G + 1)
                     if G % I == 0 and P % I == 0 and Q % (G // I) == 0]
            got = gs.group_shape(P, Q, G)
            if not cands:
                assert got is None
                continue
            I, J = got
            assert I * J == G and P % I == 0 and Q % J == 0
            best = min(abs(math.log((P / a) / (Q / b))) for a, b in cands)
            assert abs(math.log((P / I) / (Q / J))) == pytest.approx(best)


def test_cluster_realisation():
    assert gs.cluster_shape(4, 4, 2, 2) == (2, 2)
    assert gs.cluster_shape(16, 16, 16, 16) == (1, 1)     # G = p: flat
    assert gs.cluster_shape(16, 16, 1, 1) == (1, 1)       # G = 1, 256 CTAs: flat
    assert gs.cluster_shape(16, 16, 4, 4) == (4, 4)       # 16 CTAs per group
    assert gs.cluster_shape(16, 16, 4, 4, limit=8) == (1, 1)
    assert gs.cluster_shape(4, 4, 1, 1) == (4, 4)         # whole 4 x 4 grid fits


@pytest.mark.parametrize("M,N,K,P,Q,cm,cn,tm,tn,Bo", [
    (512, 512, 512, 4, 4, 2, 2, 128, 128, 64),
    (1152, 700, 96, 5, 4, 1, 2, 128, 128, 64),       # ragged blocks and sub-tiles
    (300, 520, 70, 3, 4, 3, 2, 128, 64, 32),
    (9, 10, 5, 4, 4, 2, 4, 128, 128, 16),              # an empty last block row
    (2048, 1024, 256, 4, 4, 4, 4, 256, 128, 64),
])
def test_counters_enumeration_equals_closed_form(M, N, K, P, Q, cm, cn, tm, tn, Bo):
    for npairs in (1, 15):
        e = gs.counters_enumerated(M, N, K, P, Q, cm, cn, tm, tn, Bo, npairs)
        c = gs.counters_closed_form(M, N, K, P, Q, cm, cn, tm, tn, Bo, npairs)
        assert e == c


def test_cfg0_counts_worked_by_hand():
    vals = {}
    for line in open(os.path.join(GOLDEN, "counters_cfg0.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = int(v)
    c = gs.counters_closed_form(512, 512, 512, 4, 4, 2, 2, 128, 128, 64)
    assert c["a_loaded"] == vals["a_loaded"]
    assert c["a_delivered"] - c["a_loaded"] == vals["a_saved"]
    flat = gs.counters_closed_form(512, 512, 512, 4, 4, 1, 1, 128, 128, 64)
    assert flat["a_loaded"] == vals["summa_flat"]


@pytest.mark.parametrize("P,Q,G", [(4, 4, 4), (4, 4, 1), (4, 4, 16), (2, 4, 2), (4, 2, 4)])
def test_identity_with_paper_volumes(P, Q, G):
    # one sub-tile per CTA, the group realised as one cluster: A loads = owner
    # copy + outer volume, multicast saving = inner volume; and the volumes are
    # the ones the distributed simulation counts with flat trees
    n = 32
    I, J = gs.group_shape(P, Q, G)
    cm, cn = gs.cluster_shape(P, Q, I, J)
    c = gs.counters_closed_form(n, n, n, P, Q, cm, cn, n // P, n // Q, 8)
    v = gs.paper_volumes(n, n, n, P, Q, I, J)
    A = workloads.matrix(n, n, 301, "smallint")
    B = workloads.matrix(n, n, 302, "smallint")
    sim = hs.hsumma(A, B, P, Q, I, J, b=4, Bo=8, tree="flat")
    assert v["a_outer"] == sim.stats["outer", "A"].words
    assert v["a_inner"] == sim.stats["inner", "A"].words
    assert v["b_outer"] == sim.stats["outer", "B"].words
    assert v["b_inner"] == sim.stats["inner", "B"].words
    if (cm, cn) == (P // I, Q // J):
        assert c["a_loaded"] == n * n + v["a_outer"]
        assert c["a_delivered"] - c["a_loaded"] == v["a_inner"]
        assert c["b_loaded"] == n * n + v["b_outer"]
        assert c["b_delivered"] - c["b_loaded"] == v["b_inner"]
    else:       # flat: every processor loads what SUMMA broadcasts to it
        assert c["a_loaded"] == n * n + v["a_outer"] + v["a_inner"]


# ---- block-cyclic layout (sub-tile blocks dealt round robin over the grid) ----

@pytest.mark.parametrize("M,N,K,P,Q,cm,cn,tm,tn,Bo", [
    (1152, 700, 96, 5, 4, 1, 2, 128, 128, 64),
    (130, 900, 64, 4, 6, 2, 2, 128, 128, 64),          # cluster rows wholly outside M
    (9, 10, 5, 4, 4, 2, 4, 128, 128, 16),
    (4000, 4000, 1024, 6, 8, 2, 1, 128, 256, 512),
    (3000, 2000, 640, 12, 5, 1, 1, 128, 128, 128),
])
def test_cyclic_counters_enumeration_equals_closed_form(M, N, K, P, Q, cm, cn, tm, tn, Bo):
    for npairs in (1, 15):
        e = gs.counters_enumerated(M, N, K, P, Q, cm, cn, tm, tn, Bo, npairs, cyclic=True)
        c = gs.counters_closed_form(M, N, K, P, Q, cm, cn, tm, tn, Bo, npairs, cyclic=True)
        assert e == c


def test_cyclic_counts_worked_by_hand():
    # M = 520 rows over P = 4 processor rows, 128-row sub-tiles, one tile column,
    # K = 128, B = 64 (two outer blocks).  Block: Mt = 130, so every processor
    # sweeps two sub-tiles (128 + 2 rows): 8 sub-tiles, each reading the 128 x 256
    # B panel.  Block-cyclic: 5 tile rows (4 full + 8 rows) dealt 2, 1, 1, 1:
    # 5 sub-tiles.  Owners of the two outer blocks: column 0 (Q = 1) for A,
    # rows 0 and 1 for B, so the prefetches are
    # row 0: 2 sub-tiles x (2 + 1), row 1: 1 x (2 + 1), rows 2, 3: 1 x 2 each = 13.
    blk = gs.counters_closed_form(520, 256, 128, 4, 1, 1, 1, 128, 256, 64)
    cyc = gs.counters_closed_form(520, 256, 128, 4, 1, 1, 1, 128, 256, 64, cyclic=True)
    assert blk["b_loaded"] == 8 * 128 * 256 and cyc["b_loaded"] == 5 * 128 * 256
    assert blk["a_loaded"] == cyc["a_loaded"] == 520 * 128
    # block: 2 sub-tile steps x 2 outer blocks x (4 A owners + 1 B owner)
    assert blk["l2_prefetch"] == 2 * 2 * (4 + 1) and cyc["l2_prefetch"] == 13


@pytest.mark.parametrize("P,Q,cm,cn", [(4, 4, 2, 2), (4, 4, 1, 1), (6, 2, 3, 1), (2, 8, 2, 4)])
def test_cyclic_equals_block_with_one_aligned_sub_tile_per_cta(P, Q, cm, cn):
    # M = P tm, N = Q tn: both layouts give every CTA the same single sub-tile
    tm, tn = 128, 256
    for K, Bo in ((512, 64), (640, 128)):
        blk = gs.counters_closed_form(P * tm, Q * tn, K, P, Q, cm, cn, tm, tn, Bo)
        cyc = gs.counters_closed_form(P * tm, Q * tn, K, P, Q, cm, cn, tm, tn, Bo, cyclic=True)
        assert blk == cyc
