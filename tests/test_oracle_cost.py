"""Pins of the cost-model oracle (no GPU): the paper's printed worked checks
(tests/golden/model_validation.txt), finite-difference derivatives, special
cases G = 1 and G = p, and the equivalences between the general model and the
tables."""
import math
import os

import pytest

from oracle import cost_model as cm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_printed_model_validation_checks():
    rows = read_rows("model_validation.txt")
    assert len(rows) == 3
    for name, a, bta, n, p, b, thr, holds in rows:
        a, bta = float(a), float(bta)
        n, p, b = int(n), int(p), int(b)
        assert 2 * n * b / p == int(thr)
        assert cm.sqrtp_is_minimum(n, p, b, a, bta) == bool(int(holds))
    # Grid5000: alpha/beta = 1e5 as printed
    assert 1e-4 / 1e-9 == pytest.approx(1e5)


def test_printed_bgp_speedups():
    for q, s, h, printed in read_rows("bgp_speedups.txt"):
        assert round(float(s) / float(h), 2) == float(printed)


@pytest.mark.parametrize("n,p,b,alpha,beta", [(8192, 128, 64, 1e-4, 1e-9),
                                               (65536, 16384, 256, 3e-6, 1e-9),
                                               (4096, 64, 32, 1e-6, 1e-8)])
def test_eq9_matches_finite_differences(n, p, b, alpha, beta):
    for G in (2.0, 5.5, math.sqrt(p), p / 3):
        h = 1e-4 * G
        fd = (cm.hsumma_vdg(n, p, G + h, b, b, alpha, beta)
              - cm.hsumma_vdg(n, p, G - h, b, b, alpha, beta)) / (2 * h)
        scale = (n * alpha / b + 2 * n * n * beta / p) / (G * math.sqrt(G))
        assert cm.dT_dG_vdg(n, p, G, b, alpha, beta) == pytest.approx(fd, rel=1e-5, abs=1e-6 * scale)


def test_general_model_derivative_matches_eq9():
    # eq. (6)-(8) with the Van de Geijn L(q) = log2 q + q - 1, W(q) = 2 (q-1)/q
    # equal eq. (9)
    dL = lambda q: 1 / (q * math.log(2)) + 1
    dW = lambda q: 2 / q ** 2
    n, p, b, alpha, beta = 4096, 256, 64, 2e-6, 1e-9
    for G in (3.0, 16.0, 40.0):
        g = cm.dT_dG_general(n, p, G, b, alpha, beta, dL, dW)
        assert g == pytest.approx(cm.dT_dG_vdg(n, p, G, b, alpha, beta), rel=1e-12)


def test_general_model_reproduces_tables():
    n, p, b = 8192, 256, 64
    alpha, beta = 1e-5, 1e-9
    for G in (1, 4, 16, 64, 256):
        t = cm.t_hsumma_general(n, p, G, b, alpha, beta, cm.L_binomial, cm.W_binomial)
        assert t == pytest.approx(cm.hsumma_binomial(n, p, G, b, b, alpha, beta))
        t = cm.t_hsumma_general(n, p, G, b, alpha, beta, cm.L_vdg, cm.W_vdg)
        assert t == pytest.approx(cm.hsumma_vdg(n, p, G, b, b, alpha, beta))
    assert cm.t_summa_general(n, p, b, alpha, beta, cm.L_vdg, cm.W_vdg) == pytest.approx(
        cm.summa_vdg(n, p, b, alpha, beta))


@pytest.mark.parametrize("fn,summa", [(cm.hsumma_binomial, cm.summa_binomial),
                                      (cm.hsumma_vdg, cm.summa_vdg)])
def test_G1_and_Gp_equal_summa(fn, summa):
    n, p, b, alpha, beta = 8192, 1024, 128, 3e-6, 1e-9
    assert fn(n, p, 1, b, b, alpha, beta) == pytest.approx(summa(n, p, b, alpha, beta))
    assert fn(n, p, p, b, b, alpha, beta) == pytest.approx(summa(n, p, b, alpha, beta))


def test_minimum_at_sqrtp_iff_ratio_condition():
    n, p, b = 8192, 1024, 64
    Gs = [2 ** (k / 4) for k in range(0, 41)]
    for alpha, beta in ((1e-4, 1e-9), (1e-9, 1e-6)):
        costs = [cm.hsumma_vdg(n, p, G, b, b, alpha, beta) for G in Gs]
        gbest = Gs[min(range(len(Gs)), key=costs.__getitem__)]
        if cm.sqrtp_is_minimum(n, p, b, alpha, beta):
            assert gbest == pytest.approx(math.sqrt(p))
        else:
            assert gbest in (1.0, float(p))


def test_eq12_is_cost_at_sqrtp():
    n, p, b, alpha, beta = 65536, 16384, 256, 3e-6, 1e-9
    assert cm.hsumma_optimal_vdg(n, p, b, alpha, beta) == pytest.approx(
        cm.hsumma_vdg(n, p, math.sqrt(p), b, b, alpha, beta))


def test_exascale_plot_formulas():
    n, p, b, alpha, beta, gamma = 2 ** 22, 2 ** 20, 256, 5e-7, 1e-11, 1e-18
    s = cm.exascale_summa(n, p, b, alpha, beta, gamma)
    assert cm.exascale_hsumma(1, n, p, b, alpha, beta, gamma) == pytest.approx(s)
    assert cm.exascale_hsumma(p, n, p, b, alpha, beta, gamma) == pytest.approx(s)
    best = min(cm.exascale_hsumma(2 ** k, n, p, b, alpha, beta, gamma) for k in range(21))
    assert best == pytest.approx(cm.exascale_hsumma(2 ** 10, n, p, b, alpha, beta, gamma))
    assert best < s
    # the plot is the Van de Geijn cost plus computation
    assert cm.exascale_hsumma(64, n, p, b, alpha, beta, gamma) == pytest.approx(
        cm.summa_comp(n, p) * gamma + cm.hsumma_vdg(n, p, 64, b, b, alpha, beta))


def test_table_sums_match_functions():
    n, p, G, b, B = 4096, 256, 16, 32, 64
    t1 = cm.table1(n, p, G, b, B)["hsumma"]
    alpha, beta = 1.0, 0.0
    assert t1["lat_in"] + t1["lat_out"] == pytest.approx(cm.hsumma_binomial(n, p, G, b, B, alpha, beta))
    assert t1["band_in"] + t1["band_out"] == pytest.approx(cm.hsumma_binomial(n, p, G, b, B, 0.0, 1.0))
    t2 = cm.table2(n, p, G, b, B)["hsumma"]
    assert t2["lat_in"] + t2["lat_out"] == pytest.approx(cm.hsumma_vdg(n, p, G, b, B, 1.0, 0.0))
    assert t2["band_in"] + t2["band_out"] == pytest.approx(cm.hsumma_vdg(n, p, G, b, B, 0.0, 1.0))


def test_paper_rule_groups():
    assert cm.paper_rule_groups(256, [1, 4, 16, 64, 256]) == 16
    assert cm.paper_rule_groups(192, [1, 3, 4, 12, 16, 48]) in (12, 16)
