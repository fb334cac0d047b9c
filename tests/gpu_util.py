"""Helpers shared by the GPU tests: seeded inputs on the device and the library
initialised once."""
import numpy as np
import pytest

import workloads


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def lib_ready():
    import paper_1306_4161_gb300 as hs
    from paper_1306_4161_gb300 import _build
    _build.build()
    hs.init(0)
    return hs


def pair(M, N, K, seed, dist="uniform", dist_b=None):
    """Seeded host matrices A (M x K) and B (K x N) and their device copies."""
    torch = torch_cuda()
    A = workloads.matrix(M, K, seed, dist)
    B = workloads.matrix(K, N, seed + 1, dist_b or dist)
    return A, B, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()


def sample_entries(M, N, n, seed):
    """n seeded (row, col) entries plus every corner and tile border."""
    x = workloads.splitmix64(seed, 0, 2 * n)
    rows = (x[0::2] % np.uint64(max(M, 1))).astype(np.int64)
    cols = (x[1::2] % np.uint64(max(N, 1))).astype(np.int64)
    extra_r = [0, M - 1, 0, M - 1] + [min(M - 1, r) for r in (127, 128, 255, 256)]
    extra_c = [0, 0, N - 1, N - 1] + [min(N - 1, c) for c in (255, 256, 127, 128)]
    return np.concatenate([rows, extra_r]), np.concatenate([cols, extra_c])


def border_grid(M, N, tm, tn, n_rows, n_cols, seed):
    """Row and column sets of a sampled accuracy check: every tile-border row
    (the first and last row of each tm-row block) and column (of each tn-column
    block), plus n_rows / n_cols seeded ones; the entries are their cross
    product, column by column (so the reference reads each column of B once)."""
    x = workloads.splitmix64(seed, 0, n_rows + n_cols)
    rows = set((x[:n_rows] % np.uint64(max(M, 1))).astype(np.int64).tolist())
    cols = set((x[n_rows:] % np.uint64(max(N, 1))).astype(np.int64).tolist())
    for b in range(0, M, tm):
        rows.update((b, min(M, b + tm) - 1))
    for b in range(0, N, tn):
        cols.update((b, min(N, b + tn) - 1))
    rows = np.array(sorted(rows), dtype=np.int64)
    cols = np.array(sorted(cols), dtype=np.int64)
    ri = np.tile(np.arange(rows.size, dtype=np.int64), cols.size)   # index into rows
    cj = np.repeat(cols, rows.size)
    return rows, cols, ri, cj
