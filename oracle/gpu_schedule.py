"""Oracle for the host-side group resolution and the GPU panel-load counters.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

On one GPU the virtual P x Q processor grid of Section III becomes a grid of
P x Q thread blocks (CTAs), one per virtual processor, each owning the C block
of rows [r*Mt, (r+1)*Mt) and columns [c*Nt, (c+1)*Nt), Mt = ceil(M/P),
Nt = ceil(N/Q), which it sweeps in tm x tn sub-tiles in a fixed order.
  * group (Section III, Figure 2): I x J groups of (P/I) x (Q/J) CTAs;
  * inner, in-group broadcast (Figure 4): when a whole group fits in one thread
    block cluster, the group is that cluster, and every b-wide panel of A is
    loaded once per cluster row and multicast to the Q/J CTAs of the row (B: once
    per cluster column, to the P/I CTAs of the column);  a group that does not
    fit (a "software group"), and a group of one processor, loads flat: each CTA
    fetches its own panels;
  * outer, between-group broadcast (Figure 3): at each outer step the group that
    owns the outer block (Algorithm 1's Pivot_group_col / Pivot_group_row)
    prefetches the next outer panels into L2, from where every group reads them.

Block-cyclic layout (Section VI's future-work distribution, here with the
sub-tile as the distribution block): CTA (r, c) sweeps the sub-tiles of tile
rows r, r + P, r + 2P, ... and tile columns c, c + Q, ...; every CTA sweeps the
nominal ceil(ceil(M/tm)/P) x ceil(ceil(N/tn)/Q) sub-tiles in lockstep with its
cluster, and skips a sub-tile when its whole cluster lies outside the matrix
(the cluster's first tile row at or past M, or its first tile column at or
past N).  The owner of outer block o is processor column o mod Q (A) and
processor row o mod P (B).
"""
from __future__ import annotations

import math


def group_shape(P: int, Q: int, G: int):
    """Factor G = I * J with I | P and J | Q (Section III leaves the choice
    open; Section IV-B uses sqrt(G) x sqrt(G)).  Reading: the most square
    in-group grid, i.e. minimal |log((P/I) / (Q/J))|; ties go to the smaller I.
    Returns (I, J) or None when no factorisation exists."""
    best = None
    for I in range(1, G + 1):
        if G % I:
            continue
        J = G // I
        if P % I or Q % J:
            continue
        key = (abs(math.log((P / I) / (Q / J))), I)
        if best is None or key < best[0]:
            best = (key, (I, J))
    return None if best is None else best[1]


def cluster_shape(P: int, Q: int, I: int, J: int, limit: int = 16):
    """Realised cluster (rows, cols) of CTAs: the whole group when it has at
    least two CTAs and at most `limit`, otherwise 1 x 1 (flat)."""
    pi, qj = P // I, Q // J
    if pi * qj <= limit and pi * qj > 1:
        return pi, qj
    return 1, 1


def ceil_div(a, b):
    return -(-a // b)


def _active_steps(T, P, cm, r):
    """Sub-steps i of processor row r (block-cyclic layout) whose cluster,
    with first row r - r % cm, holds a tile row r - r % cm + i P < T."""
    r0 = r - r % cm
    return ceil_div(T - r0, P) if r0 < T else 0


def _owned_outer(nout, q, who):
    """Outer blocks o < nout with o mod q == who."""
    return ceil_div(nout - who, q) if who < nout else 0


def counters_closed_form_cyclic(M, N, K, P, Q, cm, cn, tm, tn, Bo, npairs=1):
    """Panel-load counters of one launch in the block-cyclic layout.

    With Tm = ceil(M/tm), Tn = ceil(N/tn) tiles and act_m(r), act_n(c) the
    sub-steps a CTA row / column does not skip, every tile row is swept once
    per active column step, so
      a_delivered = npairs * M * K * sum_c act_n(c),  a_loaded = a_delivered / cn
      b_delivered = npairs * K * N * sum_r act_m(r),  b_loaded = b_delivered / cm
      l2_prefetch = npairs * sum_{r,c} act_m(r) act_n(c) (own_Q(c) + own_P(r))
    with own_Q(c) the outer blocks o with o mod Q = c."""
    Tm, Tn = ceil_div(M, tm), ceil_div(N, tn)
    nout = ceil_div(K, Bo) if K else 0
    am = [_active_steps(Tm, P, cm, r) for r in range(P)]
    an = [_active_steps(Tn, Q, cn, c) for c in range(Q)]
    sm, sn = sum(am), sum(an)
    assert sm % cm == 0 and sn % cn == 0
    pf = (sm * sum(an[c] * _owned_outer(nout, Q, c) for c in range(Q))
          + sn * sum(am[r] * _owned_outer(nout, P, r) for r in range(P)))
    return dict(a_loaded=npairs * M * K * sn // cn, a_delivered=npairs * M * K * sn,
                b_loaded=npairs * K * N * sm // cm, b_delivered=npairs * K * N * sm,
                l2_prefetch=npairs * pf)


def counters_closed_form(M, N, K, P, Q, cm, cn, tm, tn, Bo, npairs=1, cyclic=False):
    """Panel-load counters of one launch, in elements.

    a_loaded    = npairs * (Q / cn) * nsub_n * M * K   (one load per cluster row)
    a_delivered = npairs *  Q       * nsub_n * M * K   (every CTA receives it)
    b_loaded    = npairs * (P / cm) * nsub_m * K * N
    b_delivered = npairs *  P       * nsub_m * K * N
    l2_prefetch = npairs * nsub_m * nsub_n * ceil(K / Bo) * (P + Q)
    with nsub_m = ceil(ceil(M/P) / tm), nsub_n = ceil(ceil(N/Q) / tn) sub-tiles
    per CTA (every CTA sweeps the nominal count so that a cluster runs in
    lockstep; rows and columns outside its block are not counted).
    cyclic=True: the block-cyclic layout (counters_closed_form_cyclic)."""
    if cyclic:
        return counters_closed_form_cyclic(M, N, K, P, Q, cm, cn, tm, tn, Bo, npairs)
    Mt, Nt = ceil_div(M, P), ceil_div(N, Q)
    nsm, nsn = ceil_div(Mt, tm), ceil_div(Nt, tn)
    nout = ceil_div(K, Bo) if K else 0
    return dict(
        a_loaded=npairs * (Q // cn) * nsn * M * K,
        a_delivered=npairs * Q * nsn * M * K,
        b_loaded=npairs * (P // cm) * nsm * K * N,
        b_delivered=npairs * P * nsm * K * N,
        l2_prefetch=npairs * nsm * nsn * nout * (P + Q),
    )


def counters_enumerated(M, N, K, P, Q, cm, cn, tm, tn, Bo, npairs=1, cyclic=False):
    """The same counters by walking every CTA and sub-tile: the CTA at cluster
    column rank x issues the rows [x*tm/cn, (x+1)*tm/cn) of each A sub-tile panel
    (multicast to its cluster row); the CTA at cluster row rank y issues the
    columns [y*tn/cm, (y+1)*tn/cm) of each B sub-tile panel; only elements
    inside the CTA's block and the matrix count.  cyclic=True walks the
    block-cyclic layout, sub-tile by sub-tile and outer block by outer block."""
    if cyclic:
        return _counters_enumerated_cyclic(M, N, K, P, Q, cm, cn, tm, tn, Bo, npairs)
    Mt, Nt = ceil_div(M, P), ceil_div(N, Q)
    nsm, nsn = ceil_div(Mt, tm), ceil_div(Nt, tn)
    out = dict(a_loaded=0, a_delivered=0, b_loaded=0, b_delivered=0, l2_prefetch=0)
    nout = ceil_div(K, Bo) if K else 0
    for r in range(P):
        rlo, rhi = r * Mt, min(M, (r + 1) * Mt)
        for c in range(Q):
            clo, chi = c * Nt, min(N, (c + 1) * Nt)
            x, y = c % cn, r % cm
            for mi in range(nsm):
                for ni in range(nsn):
                    m0 = rlo + mi * tm
                    a0, a1 = m0 + x * tm // cn, m0 + (x + 1) * tm // cn
                    arows = max(0, min(a1, rhi) - max(a0, rlo))
                    out["a_loaded"] += npairs * arows * K
                    out["a_delivered"] += npairs * cn * arows * K
                    n0 = clo + ni * tn
                    b0, b1 = n0 + y * tn // cm, n0 + (y + 1) * tn // cm
                    bcols = max(0, min(b1, chi) - max(b0, clo))
                    out["b_loaded"] += npairs * bcols * K
                    out["b_delivered"] += npairs * cm * bcols * K
    # outer step: one A panel prefetch per processor row and one B panel
    # prefetch per processor column, per sub-tile and outer step
    out["l2_prefetch"] = npairs * nsm * nsn * nout * (P + Q)
    return out


def _counters_enumerated_cyclic(M, N, K, P, Q, cm, cn, tm, tn, Bo, npairs):
    Tm, Tn = ceil_div(M, tm), ceil_div(N, tn)
    nsm, nsn = ceil_div(Tm, P), ceil_div(Tn, Q)
    nout = ceil_div(K, Bo) if K else 0
    out = dict(a_loaded=0, a_delivered=0, b_loaded=0, b_delivered=0, l2_prefetch=0)
    for r in range(P):
        for c in range(Q):
            x, y = c % cn, r % cm
            r0, c0 = r - y, c - x                 # the cluster's first row and column
            for mi in range(nsm):
                if (r0 + mi * P) * tm >= M:       # no row of the cluster in the matrix
                    continue
                m0 = (r + mi * P) * tm
                rlo, rhi = m0, min(M, m0 + tm)
                for ni in range(nsn):
                    if (c0 + ni * Q) * tn >= N:
                        continue
                    n0 = (c + ni * Q) * tn
                    clo, chi = n0, min(N, n0 + tn)
                    a0, a1 = m0 + x * tm // cn, m0 + (x + 1) * tm // cn
                    arows = max(0, min(a1, rhi) - max(a0, rlo))
                    out["a_loaded"] += npairs * arows * K
                    out["a_delivered"] += npairs * cn * arows * K
                    b0, b1 = n0 + y * tn // cm, n0 + (y + 1) * tn // cm
                    bcols = max(0, min(b1, chi) - max(b0, clo))
                    out["b_loaded"] += npairs * bcols * K
                    out["b_delivered"] += npairs * cm * bcols * K
                    for o in range(nout):         # the owners of outer block o prefetch
                        out["l2_prefetch"] += npairs * ((o % Q == c) + (o % P == r))
    return out


def paper_volumes(M, N, K, P, Q, I, J):
    """Flat-tree word counts of the paper's broadcasts (A and B), for the
    identity with the GPU counters at one sub-tile per CTA:
    outer (J-1) M K, inner (Q-J) M K; B: (I-1) K N and (P-I) K N."""
    return dict(a_outer=(J - 1) * M * K, a_inner=(Q - J) * M * K,
                b_outer=(I - 1) * K * N, b_inner=(P - I) * K * N)
