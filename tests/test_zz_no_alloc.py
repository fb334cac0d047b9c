"""The allocation-free backward pass of the cost model (GPU): through the C ABI
it gives the gradient and loss of hsumma_mlp_backward on two calls in a row
that share its fixed scratch, and rejects a batch beyond its maximum."""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import mlp
from tests.gpu_util import lib_ready, torch_cuda

pytestmark = pytest.mark.gpu


def _inputs(torch, batch, seed):
    th = 0.3 * workloads.matrix(1, mlp.N_PARAMS, seed, "uniform")[0]
    X = workloads.matrix(batch, 10, seed + 1, "uniform")
    y = workloads.matrix(1, batch, seed + 2, "uniform")[0]
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    return f32(th), f32(X), f32(y)


def _backward(hs, torch, name, batch, th, X, y):
    g = torch.full((mlp.N_PARAMS,), float("nan"), dtype=torch.float32, device="cuda")
    loss = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
    fn = getattr(hs.lib(), name)
    hs._check(fn(batch, th.data_ptr(), X.data_ptr(), y.data_ptr(), g.data_ptr(),
                 loss.data_ptr(), None))
    hs.sync(None)
    return g.cpu().numpy().astype(np.float64), float(loss.item())


def test_no_alloc_backward_matches_backward_twice():
    torch = torch_cuda()
    hs = lib_ready()
    # the largest batch first, then a smaller one that reads fewer block slots
    # of the scratch the first call left behind
    for batch, seed in [(4096, 31), (777, 47)]:
        th, X, y = _inputs(torch, batch, seed)
        want_g, want_l = _backward(hs, torch, "hsumma_mlp_backward", batch, th, X, y)
        got_g, got_l = _backward(hs, torch, "hsumma_mlp_backward_noalloc", batch, th, X, y)
        assert np.all(np.isfinite(got_g))
        assert got_l == pytest.approx(want_l, rel=1e-4)
        assert np.max(np.abs(got_g - want_g)) <= 1e-4 * np.abs(want_g).max()


def test_no_alloc_backward_rejects_large_batch():
    torch = torch_cuda()
    hs = lib_ready()
    batch = 4097
    th, X, y = _inputs(torch, batch, 5)  # sized for the batch, so nothing could read past it
    g = torch.empty(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    rc = hs.lib().hsumma_mlp_backward_noalloc(batch, th.data_ptr(), X.data_ptr(), y.data_ptr(),
                                               g.data_ptr(), ctypes.c_void_p(0), None)
    assert rc == -1
    assert b"HSUMMA_MLP_NOALLOC_MAX_BATCH" in hs.lib().hsumma_last_error()
