"""A seeded sweep over shapes, kinds, slice counts, configurations and grid
layouts (GPU): every product equals the oracle's bit for bit -- binary64 on
small integers (every order of summation is exact there), the split kinds on
wide-range inputs against the oracle's split_gemm.  The configuration of each
case is one of the library's own candidates for that product (any grid, group
count, cluster shape and panel width the automatic choice may run)."""
import numpy as np
import pytest

import workloads
from oracle import split
from tests.gpu_util import lib_ready, torch_cuda

pytestmark = pytest.mark.gpu


def sweep_cases(n, seed):
    x = workloads.splitmix64(seed, 0, 8 * n)
    out = []
    for i in range(n):
        r = [int(v) for v in x[8 * i:8 * (i + 1)]]
        kind = ("fp64", "bf16", "int8")[r[0] % 3]
        M, N, K = 1 + r[1] % 700, 1 + r[2] % 700, 1 + r[3] % 900
        S = {"fp64": 0, "bf16": 1 + r[4] % 6, "int8": 1 + r[4] % 8}[kind]
        layout = "cyclic" if r[5] % 3 == 0 else "block"
        out.append((kind, M, N, K, S, layout, r[6] % 1000, r[7] % 100000))
    return out


@pytest.mark.parametrize("case", sweep_cases(60, 7001), ids=lambda c: "-".join(map(str, c[:6])))
def test_sweep_matches_oracle(case):
    kind, M, N, K, S, layout, pick, seed = case
    hs = lib_ready()
    torch = torch_cuda()
    cands = hs.candidates(M, N, K, kind, S)
    P, Q, G, b, Bo = cands[pick % len(cands)]
    dist = "smallint" if kind == "fp64" else "wide"
    A = workloads.matrix(M, K, seed, dist)
    B = workloads.matrix(K, N, seed + 1, dist)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = hs.gemm(dA, dB, P=P, Q=Q, G=G, b=b, Bouter=Bo, kind=kind, slices=S, layout=layout)
    hs.sync()
    if kind == "fp64":
        want = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    else:
        want = split.split_gemm(A, B, S, kind)
    assert np.array_equal(C.cpu().numpy(), want), (P, Q, G, b, Bo, hs.group_shape(P, Q, G))
