"""The paper's communication-cost model (Section IV), as plain functions.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Hockney model: one message of m words costs alpha + m beta; gamma is the time of
one combined multiply-add.  Square n x n matrices on a sqrt(p) x sqrt(p) grid,
G groups as a sqrt(G) x sqrt(G) grid, inner block b, outer block B.
"""
from __future__ import annotations

import math


def log2(x):
    return math.log2(x)


# Section IV, broadcast costs among p processors for a message of m words
def bcast_binomial(m, p, alpha, beta):
    return log2(p) * (alpha + m * beta)


def bcast_vdg(m, p, alpha, beta):
    return (log2(p) + p - 1) * alpha + 2 * (p - 1) / p * m * beta


# Section IV-A, SUMMA
def summa_comp(n, p):
    return 2 * n ** 3 / p


def summa_binomial(n, p, b, alpha, beta):
    return log2(p) * (alpha * n / b + beta * n ** 2 / math.sqrt(p))


def summa_vdg(n, p, b, alpha, beta):
    sp = math.sqrt(p)
    return ((log2(p) + 2 * (sp - 1)) * alpha * n / b
            + 4 * (1 - 1 / sp) * n ** 2 / sp * beta)


# Section IV-B, HSUMMA inner (inside groups) and outer (between groups) costs
def hsumma_inner_binomial(n, p, G, b, alpha, beta):
    return log2(p / G) * (alpha * n / b + beta * n ** 2 / math.sqrt(p))


def hsumma_inner_vdg(n, p, G, b, alpha, beta):
    sp, sg = math.sqrt(p), math.sqrt(G)
    return ((log2(p / G) + 2 * (sp / sg - 1)) * alpha * n / b
            + 4 * (1 - sg / sp) * n ** 2 / sp * beta)


def hsumma_outer_binomial(n, p, G, B, alpha, beta):
    return log2(G) * (alpha * n / B + beta * n ** 2 / math.sqrt(p))


def hsumma_outer_vdg(n, p, G, B, alpha, beta):
    sp, sg = math.sqrt(p), math.sqrt(G)
    return ((log2(G) + 2 * (sg - 1)) * alpha * n / B
            + 4 * (1 - 1 / sg) * n ** 2 / sp * beta)


def hsumma_binomial(n, p, G, b, B, alpha, beta):
    return (hsumma_inner_binomial(n, p, G, b, alpha, beta)
            + hsumma_outer_binomial(n, p, G, B, alpha, beta))


def hsumma_vdg(n, p, G, b, B, alpha, beta):
    return (hsumma_inner_vdg(n, p, G, b, alpha, beta)
            + hsumma_outer_vdg(n, p, G, B, alpha, beta))


# Tables I and II: latency factors (multiply alpha) and bandwidth factors
# (multiply beta), split into inside / between groups
def table1(n, p, G, b, B):
    sp = math.sqrt(p)
    return {
        "summa": dict(comp=2 * n ** 3 / p, lat=log2(p) * n / b,
                      band=n ** 2 * log2(p) / sp),
        "hsumma": dict(comp=2 * n ** 3 / p, lat_in=log2(p / G) * n / b,
                       lat_out=log2(G) * n / B, band_in=log2(p / G) * n ** 2 / sp,
                       band_out=log2(G) * n ** 2 / sp),
    }


def table2(n, p, G, b, B):
    sp, sg = math.sqrt(p), math.sqrt(G)
    q4 = p ** 0.25
    return {
        "summa": dict(comp=2 * n ** 3 / p, lat=(log2(p) + 2 * (sp - 1)) * n / b,
                      band=4 * (1 - 1 / sp) * n ** 2 / sp),
        "hsumma": dict(comp=2 * n ** 3 / p,
                       lat_in=(log2(p / G) + 2 * (sp / sg - 1)) * n / b,
                       lat_out=(log2(G) + 2 * (sg - 1)) * n / B,
                       band_in=4 * (1 - sg / sp) * n ** 2 / sp,
                       band_out=4 * (1 - 1 / sg) * n ** 2 / sp),
        "hsumma_sqrtp_b_eq_B": dict(comp=2 * n ** 3 / p,
                                    lat=(log2(p) + 4 * (q4 - 1)) * n / b,
                                    band=8 * (1 - 1 / q4) * n ** 2 / sp),
    }


# Section IV-C, general broadcast model T = L(p) alpha + m W(p) beta, eq. (1)
def t_summa_general(n, p, b, alpha, beta, L, W):
    """Eq. (2)."""
    sp = math.sqrt(p)
    return 2 * (n / b * L(sp) * alpha + n ** 2 / sp * W(sp) * beta)


def t_hsumma_latency(n, p, G, b, alpha, L):
    """Eq. (4), b = B."""
    return 2 * n / b * (L(math.sqrt(G)) + L(math.sqrt(p) / math.sqrt(G))) * alpha


def t_hsumma_bandwidth(n, p, G, beta, W):
    """Eq. (5)."""
    sp = math.sqrt(p)
    return 2 * n ** 2 / sp * (W(math.sqrt(G)) + W(sp / math.sqrt(G))) * beta


def t_hsumma_general(n, p, G, b, alpha, beta, L, W):
    """Eq. (3) = (4) + (5)."""
    return t_hsumma_latency(n, p, G, b, alpha, L) + t_hsumma_bandwidth(n, p, G, beta, W)


def L_binomial(q):
    return log2(q)


def W_binomial(q):
    return log2(q)


def L_vdg(q):
    return log2(q) + q - 1


def W_vdg(q):
    return 2 * (q - 1) / q


def dL1(p, G, dL):
    """Eq. (7): L_1(p, G) from the derivative dL of L."""
    sg, sp = math.sqrt(G), math.sqrt(p)
    return dL(sg) / sg - dL(sp / sg) * sp / (G * sg)


def dT_dG_general(n, p, G, b, alpha, beta, dL, dW):
    """Eq. (6) with (7) and (8)."""
    return n / b * dL1(p, G, dL) * alpha + n ** 2 / math.sqrt(p) * dL1(p, G, dW) * beta


def dT_dG_vdg(n, p, G, b, alpha, beta):
    """Eq. (9): derivative of the Van de Geijn HSUMMA cost in G (b = B)."""
    return (G - math.sqrt(p)) / (G * math.sqrt(G)) * (n * alpha / b - 2 * n ** 2 / p * beta)


def sqrtp_is_minimum(n, p, b, alpha, beta) -> bool:
    """Eq. (10): G = sqrt(p) minimises the cost iff alpha/beta > 2 n b / p."""
    return alpha / beta > 2 * n * b / p


def hsumma_optimal_vdg(n, p, b, alpha, beta):
    """Eq. (12): cost at G = sqrt(p), b = B."""
    q4 = p ** 0.25
    return ((log2(p) + 4 * (q4 - 1)) * n / b * alpha
            + 8 * (1 - 1 / q4) * n ** 2 / math.sqrt(p) * beta)


# Section V-C, the exascale prediction plot (Figure 9): total time including
# the computation 2 n^3 gamma / p
def exascale_hsumma(G, n, p, b, alpha, beta, gamma):
    sp, sg = math.sqrt(p), math.sqrt(G)
    return (2 * n ** 3 * gamma / p + n / b * (log2(p) + 2 * (sp / sg + sg - 2)) * alpha
            + 4 * (n * n / sp) * (2 - sg / sp - 1 / sg) * beta)


def exascale_summa(n, p, b, alpha, beta, gamma):
    sp = math.sqrt(p)
    return (2 * n ** 3 * gamma / p + n / b * (log2(p) + 2 * (sp - 1)) * alpha
            + 4 * (n * n / sp) * (1 - 1 / sp) * beta)


def paper_rule_groups(p: int, valid) -> int:
    """The paper's choice of G (Section IV-C): the valid group count nearest to
    sqrt(p) on a log scale (ties: the smaller)."""
    target = 0.5 * math.log2(p)
    return min(valid, key=lambda g: (abs(math.log2(g) - target), g))
