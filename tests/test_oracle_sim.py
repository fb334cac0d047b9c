"""Pins of the distributed SUMMA / HSUMMA simulation (no GPU):
  * C equals the triple-loop oracle bit for bit, for every valid G, every tree
    and float inputs (same per-element operation order), and equals the exact
    product on small integers;
  * the counted broadcast volumes reproduce the paper's Tables I and II, typed
    here from the paper (not from the oracle's own closed-form helper);
  * the Section III invariants: n/b steps whatever B, the same total data as
    SUMMA, and SUMMA at G = 1 and G = p."""
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads
from oracle import hsumma_sim as hs
from oracle import native


def divisor_pairs(P, Q):
    return [(I, J) for I in range(1, P + 1) if P % I == 0 for J in range(1, Q + 1) if Q % J == 0]


@pytest.mark.parametrize("tree", hs.TREES)
def test_hsumma_equals_oracle_every_group_shape(tree):
    P, Q = 4, 4
    M = N = K = 32
    A = workloads.matrix(M, K, 101, "uniform")
    B = workloads.matrix(K, N, 102, "wide")
    C0 = native.dgemm(A, B)
    for I, J in divisor_pairs(P, Q):
        res = hs.hsumma(A, B, P, Q, I, J, b=2, Bo=4, tree=tree)
        assert np.array_equal(res.C, C0), (I, J)
    assert np.array_equal(hs.summa(A, B, P, Q, 4, tree).C, C0)


def test_nonsquare_grid_and_integers_exact():
    P, Q = 2, 6
    M, N, K = 12, 18, 24
    A = workloads.matrix(M, K, 103, "smallint")
    B = workloads.matrix(K, N, 104, "smallint")
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    for I, J in divisor_pairs(P, Q):
        res = hs.hsumma(A, B, P, Q, I, J, b=2, Bo=4, tree="binomial")
        assert np.array_equal(res.C, exact)


def table1_binomial(n, p, G, b, B):
    # Table I: latency factors log2(p/G) n/b + log2(G) n/B, bandwidth factors
    # log2(p/G) n^2/sqrt(p) + log2(G) n^2/sqrt(p); SUMMA: log2(p) n/b, log2(p) n^2/sqrt(p)
    sp = math.isqrt(p)
    return dict(lat_in=math.log2(p / G) * n / b, lat_out=math.log2(G) * n / B,
                band_in=math.log2(p / G) * n * n / sp, band_out=math.log2(G) * n * n / sp,
                summa_lat=math.log2(p) * n / b, summa_band=math.log2(p) * n * n / sp)


def table2_vdg(n, p, G, b, B):
    # Table II
    sp, sg = math.isqrt(p), math.isqrt(G)
    return dict(lat_in=(math.log2(p / G) + 2 * (sp / sg - 1)) * n / b,
                lat_out=(math.log2(G) + 2 * (sg - 1)) * n / B,
                band_in=4 * (1 - sg / sp) * n * n / sp,
                band_out=4 * (1 - 1 / sg) * n * n / sp,
                summa_lat=(math.log2(p) + 2 * (sp - 1)) * n / b,
                summa_band=4 * (1 - 1 / sp) * n * n / sp)


def crit(stats, level):
    a, b = stats[level, "A"], stats[level, "B"]
    return a.crit_rounds + b.crit_rounds, a.crit_words + b.crit_words


@pytest.mark.parametrize("p,G", [(16, 1), (16, 4), (16, 16), (64, 4), (64, 16), (64, 64), (64, 1)])
@pytest.mark.parametrize("tree,table", [("binomial", table1_binomial), ("vdg", table2_vdg)])
def test_counters_reproduce_tables(p, G, tree, table):
    n, b, Bo = 64, 4, 8
    sp, sg = math.isqrt(p), math.isqrt(G)
    A = workloads.matrix(n, n, 201, "smallint")
    B = workloads.matrix(n, n, 202, "smallint")
    res = hs.hsumma(A, B, sp, sp, sg, sg, b=b, Bo=Bo, tree=tree)
    t = table(n, p, G, b, Bo)
    lat_in, band_in = crit(res.stats, "inner")
    lat_out, band_out = crit(res.stats, "outer")
    assert lat_in == pytest.approx(t["lat_in"]) and band_in == pytest.approx(t["band_in"])
    assert lat_out == pytest.approx(t["lat_out"]) and band_out == pytest.approx(t["band_out"])
    s = hs.summa(A, B, sp, sp, b, tree)
    lat, band = crit(s.stats, "summa")
    assert lat == pytest.approx(t["summa_lat"]) and band == pytest.approx(t["summa_band"])


def test_table2_sqrtp_row():
    # Table II, last row: G = sqrt(p), b = B: latency (log2 p + 4 (p^(1/4) - 1)) n / b,
    # bandwidth 8 (1 - p^(-1/4)) n^2 / sqrt(p)
    n, p, b = 64, 16, 8
    A = workloads.matrix(n, n, 203, "smallint")
    B = workloads.matrix(n, n, 204, "smallint")
    res = hs.hsumma(A, B, 4, 4, 2, 2, b=b, Bo=b, tree="vdg")
    li, bi = crit(res.stats, "inner")
    lo, bo = crit(res.stats, "outer")
    q4 = p ** 0.25
    assert li + lo == pytest.approx((math.log2(p) + 4 * (q4 - 1)) * n / b)
    assert bi + bo == pytest.approx(8 * (1 - 1 / q4) * n * n / math.sqrt(p))


def test_same_total_data_and_steps_as_summa():
    # Section III: n/B outer steps of B/b inner steps = n/b steps, and the
    # amount of data sent equals SUMMA's (flat trees: every word sent once per
    # receiver)
    n, P, Q, b = 48, 4, 6, 2
    A = workloads.matrix(n, n, 205, "smallint")
    B = workloads.matrix(n, n, 206, "smallint")
    s = hs.summa(A, B, P, Q, b, "flat")
    total = s.stats["summa", "A"].words + s.stats["summa", "B"].words
    for I, J in divisor_pairs(P, Q):
        for Bo in (2, 4):
            r = hs.hsumma(A, B, P, Q, I, J, b=b, Bo=Bo, tree="flat")
            w = sum(r.stats[lv, m].words for lv in ("outer", "inner") for m in "AB")
            assert w == total
            inner_steps = r.stats["inner", "A"].broadcasts // (P * J) if Q // J > 1 else None
            if inner_steps is not None:
                assert inner_steps == n // b


@pytest.mark.parametrize("tree", hs.TREES)
def test_G1_and_Gp_reduce_to_summa(tree):
    n, P, Q, b = 32, 4, 4, 4
    A = workloads.matrix(n, n, 207, "smallint")
    B = workloads.matrix(n, n, 208, "smallint")
    s = hs.summa(A, B, P, Q, b, tree)
    g1 = hs.hsumma(A, B, P, Q, 1, 1, b=b, Bo=2 * b, tree=tree)
    for m in "AB":
        assert vars(g1.stats["inner", m]) == vars(s.stats["summa", m])
        assert g1.stats["outer", m].messages == 0
    sB = hs.summa(A, B, P, Q, 2 * b, tree)
    gp = hs.hsumma(A, B, P, Q, P, Q, b=b, Bo=2 * b, tree=tree)
    for m in "AB":
        assert vars(gp.stats["outer", m]) == vars(sB.stats["summa", m])
        assert gp.stats["inner", m].messages == 0


def test_broadcast_trees_deliver_and_count():
    for q in (1, 2, 3, 5, 8):
        x = np.arange(24.0).reshape(4, 6)
        for tree in hs.TREES:
            for root in range(q):
                got, st = hs.broadcast(tree, x, q, root)
                assert all(np.array_equal(g, x) for g in got)
                if q > 1 and tree != "vdg":
                    assert st.messages == q - 1 and st.words == (q - 1) * x.size
                if tree == "binomial":
                    assert st.crit_rounds == hs.log2c(q)


def test_closed_form_helper_matches_simulation():
    # the oracle's own closed-form helper against its simulation, non-square too
    M, N, K, P, Q, b, Bo = 24, 16, 48, 2, 4, 2, 4
    A = workloads.matrix(M, K, 209, "smallint")
    B = workloads.matrix(K, N, 210, "smallint")
    for tree in ("flat", "binomial"):
        for I, J in divisor_pairs(P, Q):
            r = hs.hsumma(A, B, P, Q, I, J, b=b, Bo=Bo, tree=tree)
            for lv in ("outer", "inner"):
                for m in "AB":
                    cf = hs.closed_form(lv, m, M, N, K, P, Q, I, J, b, Bo, tree)
                    assert vars(cf) == vars(r.stats[lv, m]), (tree, I, J, lv, m)


# ---- block-cyclic distribution (Section VI names it as future work) ----

def test_owned_indices_worked_by_hand():
    # blocks of blk indices dealt round robin: block t to owner t mod owners
    assert hs.owned(5, 2, 2, 0).tolist() == [0, 1, 4]
    assert hs.owned(5, 2, 2, 1).tolist() == [2, 3]
    assert hs.owned(7, 3, 1, 2).tolist() == [2, 5]
    assert hs.owned(3, 4, 1, 3).tolist() == []
    assert hs.owned(12, 3, 4, 1).tolist() == [4, 5, 6, 7]        # one block each
    assert hs.owned(10, 3, 3, 0).tolist() == [0, 1, 2, 9]        # last block clipped


@pytest.mark.parametrize("tree", hs.TREES)
def test_cyclic_equals_oracle_ragged(tree):
    # rows and columns that do not divide into whole blocks per processor
    P, Q, M, N, K = 2, 4, 22, 26, 32
    A = workloads.matrix(M, K, 111, "uniform")
    B = workloads.matrix(K, N, 112, "wide")
    C0 = native.dgemm(A, B)
    for I, J in divisor_pairs(P, Q):
        res = hs.hsumma(A, B, P, Q, I, J, b=2, Bo=4, tree=tree, dist="cyclic", mb=3, nb=2)
        assert np.array_equal(res.C, C0), (I, J)
    assert np.array_equal(hs.summa(A, B, P, Q, 4, tree, dist="cyclic", mb=5, nb=3).C, C0)


def test_cyclic_integers_exact():
    P, Q, M, N, K = 3, 2, 13, 9, 24
    A = workloads.matrix(M, K, 113, "smallint")
    B = workloads.matrix(K, N, 114, "smallint")
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    for I, J in divisor_pairs(P, Q):
        res = hs.hsumma(A, B, P, Q, I, J, b=4, Bo=8, dist="cyclic", mb=2, nb=4)
        assert np.array_equal(res.C, exact)


def test_outer_roots_rotate_under_cyclic():
    # 4 x 4 grid, K = 32, B = 4: eight outer blocks.  Block distribution: A's
    # columns 8c..8c+7 live on processor column c, so the owners run
    # 0 0 1 1 2 2 3 3; block-cyclic: outer block o on column o mod 4.
    A = workloads.matrix(16, 32, 115, "uniform")
    B = workloads.matrix(32, 16, 116, "uniform")
    blk = hs.hsumma(A, B, 4, 4, 2, 2, b=2, Bo=4)
    cyc = hs.hsumma(A, B, 4, 4, 2, 2, b=2, Bo=4, dist="cyclic", mb=2, nb=2)
    assert blk.roots["A"] == [0, 0, 1, 1, 2, 2, 3, 3] == blk.roots["B"]
    assert cyc.roots["A"] == [0, 1, 2, 3, 0, 1, 2, 3] == cyc.roots["B"]
    assert np.array_equal(blk.C, cyc.C)
    # on a 2 x 4 grid the B owners cycle over the two processor rows
    cyc2 = hs.hsumma(A, B, 2, 4, 1, 2, b=2, Bo=4, dist="cyclic", mb=2, nb=2)
    assert cyc2.roots["B"] == [0, 1] * 4 and cyc2.roots["A"] == [0, 1, 2, 3] * 2


@pytest.mark.parametrize("tree", hs.TREES)
def test_cyclic_moves_the_same_data_when_blocks_are_even(tree):
    # P mb | M and Q nb | N: every processor holds M/P rows and N/Q columns, so
    # each broadcast carries as much as under the block distribution; only the
    # roots move.  Counts equal the block distribution's and Tables I / II.
    P = Q = 4
    n = 32
    A = workloads.matrix(n, n, 117, "uniform")
    B = workloads.matrix(n, n, 118, "uniform")
    for I, J in divisor_pairs(P, Q):
        if I != J:
            continue
        blk = hs.hsumma(A, B, P, Q, I, J, b=2, Bo=4, tree=tree)
        cyc = hs.hsumma(A, B, P, Q, I, J, b=2, Bo=4, tree=tree, dist="cyclic", mb=2, nb=4)
        for key in blk.stats:
            assert vars(cyc.stats[key]) == vars(blk.stats[key]), (I, key)
        for lv in ("outer", "inner"):
            for m in ("A", "B"):
                want = hs.closed_form(lv, m, n, n, n, P, Q, I, J, 2, 4, tree)
                assert vars(cyc.stats[lv, m]) == vars(want), (I, lv, m)


def test_cyclic_G1_reduces_to_summa():
    # one group: the outer level is empty and the inner broadcasts are SUMMA's,
    # with the same rotating owners when B = b
    P, Q, M, N, K = 2, 4, 12, 20, 16
    A = workloads.matrix(M, K, 119, "uniform")
    B = workloads.matrix(K, N, 120, "uniform")
    for tree in ("flat", "binomial"):
        s = hs.summa(A, B, P, Q, 2, tree, dist="cyclic", mb=3, nb=2)
        g1 = hs.hsumma(A, B, P, Q, 1, 1, b=2, Bo=2, tree=tree, dist="cyclic", mb=3, nb=2)
        assert vars(g1.stats["inner", "A"]) == vars(s.stats["summa", "A"])
        assert vars(g1.stats["inner", "B"]) == vars(s.stats["summa", "B"])
        assert g1.stats["outer", "A"].broadcasts == 0
        assert g1.roots == s.roots == {"A": [k % Q for k in range(8)],
                                       "B": [k % P for k in range(8)]}
        assert np.array_equal(g1.C, s.C)


def test_cyclic_argument_checks():
    A = np.zeros((8, 12))
    B = np.zeros((12, 8))
    with pytest.raises(ValueError):
        hs.hsumma(A, B, 2, 2, 1, 1, b=2, Bo=8, dist="cyclic", mb=2, nb=2)   # B does not divide K
    with pytest.raises(ValueError):
        hs.hsumma(A, B, 2, 2, 1, 1, b=2, Bo=4, dist="cyclic")               # no block sizes
    with pytest.raises(ValueError):
        hs.hsumma(A, B, 2, 2, 1, 1, b=2, Bo=4, dist="diagonal", mb=2, nb=2)
