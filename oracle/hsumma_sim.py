"""CPU simulation of SUMMA and HSUMMA on a virtual P x Q processor grid.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Every virtual processor holds its own blocks (numpy arrays); broadcasts are
executed as explicit point-to-point messages along a chosen tree, so that the
data each processor multiplies has really travelled through the tree, and every
message is counted.

Data distribution (Algorithm 1, block-checkerboard): processor (r, c) holds
  A[r*Mt:(r+1)*Mt, c*Kq:(c+1)*Kq]   with Mt = M/P, Kq = K/Q
  B[r*Kp:(r+1)*Kp, c*Nt:(c+1)*Nt]   with Kp = K/P, Nt = N/Q
  C[r*Mt:(r+1)*Mt, c*Nt:(c+1)*Nt].

SUMMA (Section II-A): K/b steps; in step k the owners of the pivot column of A
broadcast it along their processor row, the owners of the pivot row of B along
their processor column, and every processor adds the rank-b product.

HSUMMA (Section III, Figures 2-4, Algorithm 1): the grid is split into I x J
groups of (P/I) x (Q/J) processors; processor P_(x,y)(i,j) is processor (i, j)
of group (x, y), i.e. grid position (x*(P/I) + i, y*(Q/J) + j).  Outer step
(K/B of them): the owner of the outer A block sends it to the processors with the
same (x, i, j) in the other group columns (group_row_comm); the owner of the
outer B block to those with the same (y, i, j) in the other group rows
(group_col_comm).  Inner steps (B/b per outer step): inside every group, the
holder of the outer A block sends its b-wide slice along the in-group row
(row_comm), the holder of the outer B block along the in-group column (col_comm);
then the local update.

Block-cyclic distribution (the extension the paper's conclusion names as
future work, Section VI): the rows of A and C are cut into blocks of mb rows
dealt round robin to the P processor rows (row block t to processor row
t mod P), the columns of B and C into blocks of nb dealt to the Q processor
columns, and the k index into blocks of B (= Bouter) dealt to the processor
columns (A) and rows (B), so that every outer block has one owner: outer block o
of A is held by processor column o mod Q, of B by processor row o mod P.  The
block-checkerboard distribution above is the special case mb = M/P, nb = N/Q
and k blocks K/Q (A) and K/P (B): one block per processor.  The broadcasts and
the local update are the same; only the owners (the roots of the outer
broadcasts) and the rows and columns a processor holds change.

Readings of garbled indices: the outer A broadcast runs
over the J group columns (the text's range 1..I is read as 1..J) and the inner
one over the Q/J in-group columns; B swaps the roles; Algorithm 1's tests on
i/x for the A pivot are read as tests on j/y (the A pivot is a column index).

Local update order: C_local is updated one rank-1 term at a time in ascending
global k, c <- c + a*b with a rounded product and a rounded sum, the same
per-element operation sequence as the oracle triple loop; so for any input the
simulated C equals oracle_dgemm bit for bit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TREES = ("flat", "binomial", "vdg")


@dataclass
class BcastStats:
    """Counts for one kind of broadcast (one level, one matrix)."""
    broadcasts: int = 0        # broadcast operations with >= 2 members
    messages: int = 0          # point-to-point messages
    words: int = 0             # elements moved by all messages
    crit_rounds: int = 0       # message latencies on the critical path
    crit_words: int = 0        # elements on the critical path

    def add(self, other: "BcastStats"):
        for k in ("broadcasts", "messages", "words", "crit_rounds", "crit_words"):
            setattr(self, k, getattr(self, k) + getattr(other, k))


@dataclass
class SimResult:
    C: np.ndarray
    stats: dict = field(default_factory=dict)   # (level, matrix) -> BcastStats
    # roots of the outer broadcasts (SUMMA: of every step): "A" -> processor
    # column of each step's A owner, "B" -> processor row of each B owner
    roots: dict = field(default_factory=dict)


DISTS = ("block", "cyclic")


@dataclass(frozen=True)
class Layout:
    """Distribution blocks: rows of A and C (mb), columns of B and C (nb), the
    k index of A (ka, dealt over the Q processor columns) and of B (kb, dealt
    over the P processor rows)."""
    mb: int
    nb: int
    ka: int
    kb: int


def owned(n: int, owners: int, blk: int, who: int) -> np.ndarray:
    """The indices in [0, n) that owner `who` of `owners` holds when blocks of
    `blk` consecutive indices are dealt round robin (block t to owner
    t mod owners; the last block is clipped at n), ascending."""
    nblk = -(-n // blk) if n else 0
    parts = [np.arange(t * blk, min(n, (t + 1) * blk)) for t in range(who, nblk, owners)]
    return np.concatenate(parts) if parts else np.zeros(0, dtype=np.int64)


def make_layout(dist, M, N, K, P, Q, kblk, mb=None, nb=None) -> Layout:
    """"block": one block per processor (Algorithm 1's block-checkerboard
    distribution; needs P | M, Q | N, P | K, Q | K).  "cyclic": blocks of mb
    rows and nb columns, k blocks of `kblk` (the outer width B) for A and B."""
    if dist == "block":
        _check_shapes(M, N, K, P, Q)
        return Layout(M // P, N // Q, K // Q, K // P)
    if dist == "cyclic":
        if not (mb and nb and mb > 0 and nb > 0):
            raise ValueError("the block-cyclic distribution needs block sizes mb, nb >= 1")
        if K % kblk:
            raise ValueError("the block-cyclic distribution needs whole k blocks: B | K")
        return Layout(mb, nb, kblk, kblk)
    raise ValueError(f"unknown distribution {dist!r}")


def _rounds_flat(q, root):
    # the root sends to every other member in turn: q-1 sequential rounds
    return [[(root, (root + k) % q, None)] for k in range(1, q)]


def _rounds_binomial(q, root):
    # relative-rank binomial tree rooted at the owner: in round k every member
    # with relative rank < 2^k sends to relative rank + 2^k
    rounds = []
    k = 1
    while k < q:
        rnd = []
        for rel in range(k):
            if rel + k < q:
                rnd.append(((rel + root) % q, (rel + k + root) % q, None))
        rounds.append(rnd)
        k *= 2
    return rounds


def broadcast(tree: str, payload: np.ndarray, q: int, root: int):
    """Execute one broadcast among q members (member indices 0..q-1) from
    `root`.  Returns (list of the q received arrays, BcastStats)."""
    st = BcastStats()
    if q == 1:
        return [payload.copy()], st
    st.broadcasts = 1
    m = payload.size
    if tree in ("flat", "binomial"):
        have = [None] * q
        have[root] = payload.copy()
        rounds = _rounds_flat(q, root) if tree == "flat" else _rounds_binomial(q, root)
        for rnd in rounds:
            sent = [(src, dst, have[src]) for (src, dst, _) in rnd]
            for src, dst, data in sent:
                assert data is not None, "sender does not hold the data"
                have[dst] = data.copy()
                st.messages += 1
                st.words += data.size
            st.crit_rounds += 1
            st.crit_words += max(d.size for _, _, d in sent)
        assert all(h is not None for h in have)
        return have, st
    if tree == "vdg":
        # Van de Geijn: binomial scatter of q pieces, then ring allgather
        flat = payload.reshape(-1)
        pieces = np.array_split(flat, q)          # piece i ends at relative rank i
        held = [dict() for _ in range(q)]          # relative rank -> {piece: array}
        held[0] = {i: pieces[i].copy() for i in range(q)}
        mask = 1
        while mask < q:
            mask *= 2
        mask //= 2
        while mask >= 1:
            sizes = []
            for rel in range(0, q, 2 * mask):
                dst = rel + mask
                if dst < q:
                    part = {i: held[rel].pop(i) for i in range(dst, min(q, dst + mask))}
                    held[dst].update(part)
                    n = sum(p.size for p in part.values())
                    st.messages += 1
                    st.words += n
                    sizes.append(n)
            if sizes:
                st.crit_rounds += 1
                st.crit_words += max(sizes)
            mask //= 2
        for rel in range(q):
            assert set(held[rel]) == {rel}
        for k in range(q - 1):
            moves = []
            for rel in range(q):
                piece = (rel - k) % q
                moves.append((rel, (rel + 1) % q, piece, held[rel][piece]))
            sizes = []
            for src, dst, piece, data in moves:
                held[dst][piece] = data.copy()
                st.messages += 1
                st.words += data.size
                sizes.append(data.size)
            st.crit_rounds += 1
            st.crit_words += max(sizes)
        out = [None] * q
        for rel in range(q):
            assert set(held[rel]) == set(range(q))
            vec = np.concatenate([held[rel][i] for i in range(q)])
            out[(rel + root) % q] = vec.reshape(payload.shape)
        return out, st
    raise ValueError(f"unknown tree {tree!r}")


def _check_shapes(M, N, K, P, Q):
    if M % P or N % Q or K % P or K % Q:
        raise ValueError("block distribution needs P | M, Q | N, P | K, Q | K")


class Distributed:
    """Every processor's own blocks of A, B and C under a Layout: processor
    (r, c) holds A[rows[r]][:, acols[c]], B[brows[r]][:, cols[c]] and
    C[rows[r]][:, cols[c]]."""

    def __init__(self, A, B, P, Q, L: Layout):
        M, K = A.shape
        N = B.shape[1]
        self.P, self.Q, self.L, self.M, self.N = P, Q, L, M, N
        self.rows = [owned(M, P, L.mb, r) for r in range(P)]
        self.cols = [owned(N, Q, L.nb, c) for c in range(Q)]
        self.acols = [owned(K, Q, L.ka, c) for c in range(Q)]
        self.brows = [owned(K, P, L.kb, r) for r in range(P)]
        self.Al = [[A[np.ix_(self.rows[r], self.acols[c])] for c in range(Q)] for r in range(P)]
        self.Bl = [[B[np.ix_(self.brows[r], self.cols[c])] for c in range(Q)] for r in range(P)]
        self.Cl = [[np.zeros((len(self.rows[r]), len(self.cols[c]))) for c in range(Q)]
                   for r in range(P)]

    def owner_a(self, k0):
        """(processor column, local column offset) of the A column k0."""
        t = k0 // self.L.ka
        return t % self.Q, (t // self.Q) * self.L.ka + k0 % self.L.ka

    def owner_b(self, k0):
        """(processor row, local row offset) of the B row k0."""
        t = k0 // self.L.kb
        return t % self.P, (t // self.P) * self.L.kb + k0 % self.L.kb

    def gather(self):
        C = np.zeros((self.M, self.N))
        for r in range(self.P):
            for c in range(self.Q):
                C[np.ix_(self.rows[r], self.cols[c])] = self.Cl[r][c]
        return C


def _local_update(Cl, a, b):
    # rank-1 updates in ascending k: c <- c + a*b, rounded product then rounded sum
    for k in range(a.shape[1]):
        Cl += np.multiply.outer(a[:, k], b[k, :])


def summa(A, B, P, Q, b, tree="binomial", dist="block", mb=None, nb=None) -> SimResult:
    """SUMMA (Section II-A) with block width b; under the block-cyclic
    distribution the k blocks are b wide (one pivot block per step)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[1]
    L = make_layout(dist, M, N, K, P, Q, b, mb, nb)
    if L.ka % b or L.kb % b:
        raise ValueError("each pivot block must have one owner: b | K/Q and b | K/P")
    D = Distributed(A, B, P, Q, L)
    sA, sB = BcastStats(), BcastStats()
    roots = {"A": [], "B": []}
    for step in range(K // b):
        k0 = step * b
        c0, off_a = D.owner_a(k0)
        r0, off_b = D.owner_b(k0)
        roots["A"].append(c0)
        roots["B"].append(r0)
        recvA, recvB = {}, {}
        crit_r, crit_w = 0, 0
        per_step = BcastStats()
        for r in range(P):      # row broadcasts of the A pivot column, in parallel
            got, st = broadcast(tree, D.Al[r][c0][:, off_a:off_a + b], Q, c0)
            for c in range(Q):
                recvA[r, c] = got[c]
            per_step.add(st)
            crit_r, crit_w = max(crit_r, st.crit_rounds), max(crit_w, st.crit_words)
        sA.broadcasts += per_step.broadcasts
        sA.messages += per_step.messages
        sA.words += per_step.words
        sA.crit_rounds += crit_r
        sA.crit_words += crit_w
        crit_r, crit_w = 0, 0
        per_step = BcastStats()
        for c in range(Q):      # column broadcasts of the B pivot row
            got, st = broadcast(tree, D.Bl[r0][c][off_b:off_b + b, :], P, r0)
            for r in range(P):
                recvB[r, c] = got[r]
            per_step.add(st)
            crit_r, crit_w = max(crit_r, st.crit_rounds), max(crit_w, st.crit_words)
        sB.broadcasts += per_step.broadcasts
        sB.messages += per_step.messages
        sB.words += per_step.words
        sB.crit_rounds += crit_r
        sB.crit_words += crit_w
        for r in range(P):
            for c in range(Q):
                _local_update(D.Cl[r][c], recvA[r, c], recvB[r, c])
    return SimResult(D.gather(), {("summa", "A"): sA, ("summa", "B"): sB}, roots)


def _acc(dst: BcastStats, parallel: list):
    """Add a set of broadcasts that run at the same time: totals add up, the
    critical path takes the longest one."""
    for st in parallel:
        dst.broadcasts += st.broadcasts
        dst.messages += st.messages
        dst.words += st.words
    if parallel:
        dst.crit_rounds += max(st.crit_rounds for st in parallel)
        dst.crit_words += max(st.crit_words for st in parallel)


def hsumma(A, B, P, Q, I, J, b, Bo, tree="binomial", outer_tree=None, dist="block",
           mb=None, nb=None) -> SimResult:
    """HSUMMA (Section III, Algorithm 1) with I x J groups, inner width b and
    outer width Bo (b <= Bo, b | Bo), under the block-checkerboard ("block")
    or the block-cyclic ("cyclic", blocks mb x nb, k blocks Bo) distribution."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    outer_tree = outer_tree or tree
    M, K = A.shape
    N = B.shape[1]
    if P % I or Q % J:
        raise ValueError("groups must tile the grid: I | P and J | Q")
    if b > Bo or Bo % b:
        raise ValueError("inner block b must divide the outer block B (b <= B)")
    L = make_layout(dist, M, N, K, P, Q, Bo, mb, nb)
    if L.ka % Bo or L.kb % Bo:
        raise ValueError("each outer block must have one owner: B | K/Q and B | K/P")
    pi, qj = P // I, Q // J        # in-group grid (s/I) x (t/J)
    D = Distributed(A, B, P, Q, L)
    stats = {(lv, m): BcastStats() for lv in ("outer", "inner") for m in ("A", "B")}
    roots = {"A": [], "B": []}
    for ko in range(K // Bo):
        k0 = ko * Bo
        c0, off_a = D.owner_a(k0)      # owner processor column of the outer A block
        y0, j0 = divmod(c0, qj)        # its group column and in-group column
        r0, off_b = D.owner_b(k0)      # owner processor row of the outer B block
        x0, i0 = divmod(r0, pi)
        roots["A"].append(c0)
        roots["B"].append(r0)
        # outer A: for every processor row r, among the J processors
        # P_(x, y)(i, j0), y = 0..J-1 (group_row_comm), root y0
        outerA, par = {}, []
        for r in range(P):
            got, st = broadcast(outer_tree, D.Al[r][c0][:, off_a:off_a + Bo], J, y0)
            for y in range(J):
                outerA[r, y * qj + j0] = got[y]
            par.append(st)
        _acc(stats["outer", "A"], par)
        # outer B: for every processor column c, among the I processors
        # P_(x, y)(i0, j), x = 0..I-1 (group_col_comm), root x0
        outerB, par = {}, []
        for c in range(Q):
            got, st = broadcast(outer_tree, D.Bl[r0][c][off_b:off_b + Bo, :], I, x0)
            for x in range(I):
                outerB[x * pi + i0, c] = got[x]
            par.append(st)
        _acc(stats["outer", "B"], par)
        for ki in range(Bo // b):
            sl = slice(ki * b, (ki + 1) * b)
            recvA, par = {}, []
            for r in range(P):             # inner A: row_comm inside group (x, y)
                for y in range(J):
                    holder = y * qj + j0
                    got, st = broadcast(tree, outerA[r, holder][:, sl], qj, j0)
                    for j in range(qj):
                        recvA[r, y * qj + j] = got[j]
                    par.append(st)
            _acc(stats["inner", "A"], par)
            recvB, par = {}, []
            for c in range(Q):             # inner B: col_comm inside group (x, y)
                for x in range(I):
                    holder = x * pi + i0
                    got, st = broadcast(tree, outerB[holder, c][sl, :], pi, i0)
                    for i in range(pi):
                        recvB[x * pi + i, c] = got[i]
                    par.append(st)
            _acc(stats["inner", "B"], par)
            for r in range(P):
                for c in range(Q):
                    _local_update(D.Cl[r][c], recvA[r, c], recvB[r, c])
    return SimResult(D.gather(), stats, roots)


def log2c(q: int) -> int:
    """ceil(log2 q) for q >= 1."""
    return (q - 1).bit_length()


def closed_form(level: str, matrix: str, M, N, K, P, Q, I, J, b, Bo, tree):
    """Closed-form counts for one (level, matrix), written from the cost
    analysis of Section IV (binomial: log2(q)(alpha + m beta); Van de Geijn:
    (log2 q + q - 1) alpha + 2 (q-1)/q m beta; message size m of one
    broadcast), for comparison with the simulated counters."""
    if matrix == "B":      # B swaps the roles of (M, P, I) and (N, Q, J)
        M, N, P, Q, I, J = N, M, Q, P, J, I
    if level == "summa":
        q, nb, m = Q, K // b, (M // P) * b
    elif level == "outer":
        q, nb, m = J, K // Bo, (M // P) * Bo
    else:
        q, nb, m = Q // J, K // b, (M // P) * b
    nrow = P if level != "inner" else P * J     # broadcasts running in parallel
    st = BcastStats()
    if q == 1:
        return st
    st.broadcasts = nrow * nb
    st.messages = nrow * nb * (q - 1)
    st.words = nrow * nb * (q - 1) * m
    if tree == "flat":
        st.crit_rounds, st.crit_words = nb * (q - 1), nb * (q - 1) * m
    elif tree == "binomial":
        st.crit_rounds, st.crit_words = nb * log2c(q), nb * log2c(q) * m
    elif tree == "vdg":
        assert q & (q - 1) == 0 and m % q == 0, "closed form for powers of two"
        lg = int(math.log2(q))
        # scatter: q-1 messages, piece i makes popcount(i) hops (sum = q lg / 2
        # pieces of m/q); ring allgather: q (q-1) messages of m/q
        st.messages = nrow * nb * (q - 1 + q * (q - 1))
        st.words = nrow * nb * (lg * m // 2 + (q - 1) * m)
        st.crit_rounds = nb * (lg + q - 1)
        st.crit_words = nb * (2 * (q - 1) * m // q)
    return st
