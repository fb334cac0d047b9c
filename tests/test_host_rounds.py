"""Row blocks of the host-buffer pipeline for products on persistent CTA pairs
(CPU: host arithmetic of the library): every block after the first spans a
whole number of rounds of the resident clusters, the first takes the
remaining tile rows, at most four blocks, and the processor rows add up."""
import math

import pytest

import paper_1306_4161_gb300 as hs
from paper_1306_4161_gb300 import _build


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def test_bench_grid():
    # 128 x 64 processors, two column blocks of 32, 2 x 1 groups, 76 resident
    # pair clusters: 32 tiles per tile row, 19 tile rows a whole number of
    # rounds (608 tiles = 8 rounds); 64 tile rows = 7 + 3 x 19
    assert hs.host_row_rounds(128, 32, 1, 76) == [14, 38, 38, 38]


def test_more_than_four_steps_merge():
    # 128 tile rows: 14 + 6 x 19 would be seven blocks; steps of 38 tile rows
    assert hs.host_row_rounds(256, 32, 1, 76) == [28, 76, 76, 76]
    assert hs.host_row_rounds(128, 32, 1, 1) == [32, 32, 32, 32]


@pytest.mark.parametrize("P,Qc,cn,res", [(7, 8, 1, 76), (40, 4, 1, 76), (38, 4, 1, 76),
                                         (20, 2, 2, 38), (2, 32, 1, 76)])
def test_no_split_or_small_cases(P, Qc, cn, res):
    got = hs.host_row_rounds(P, Qc, cn, res)
    T, u = P // 2, Qc // cn
    t = res // math.gcd(res, u)
    if P % 2 or t >= T:
        assert got == []
    else:
        assert len(got) >= 2


def test_properties_over_a_grid():
    seen = 0
    for P in range(2, 260, 2):
        for Qc in (1, 2, 3, 4, 8, 12, 16, 19, 32, 38, 64):
            for cn in (1, 2):
                if Qc % cn:
                    continue
                for res in (1, 19, 38, 76, 74):
                    got = hs.host_row_rounds(P, Qc, cn, res)
                    T, u = P // 2, Qc // cn
                    t = res // math.gcd(res, u)
                    if not got:
                        assert t >= T       # no whole-round block below all of P
                        continue
                    seen += 1
                    assert 2 <= len(got) <= 4 and sum(got) == P
                    assert all(p % 2 == 0 and p > 0 for p in got)
                    step = got[-1] // 2
                    assert all(p == 2 * step for p in got[1:-1])
                    assert step % t == 0 and (step * u) % res == 0
                    if got[0] != got[1]:
                        assert got[0] < got[1]          # the remainder comes first
                    else:
                        assert T % step == 0
    assert seen > 500


def test_rejects_bad_arguments():
    with pytest.raises(hs.HsummaError):
        hs.host_row_rounds(0, 4, 1, 76)
    with pytest.raises(hs.HsummaError):
        hs.host_row_rounds(8, 4, 3, 76)
    with pytest.raises(hs.HsummaError):
        hs.host_row_rounds(8, 4, 1, 0)
