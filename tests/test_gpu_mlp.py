"""The learned cost model's device kernels against the float64 MLP oracle
(GPU): forward, backpropagated gradient, Adam step, bf16 scoring and argmin."""
import numpy as np
import pytest

import workloads
from oracle import mlp
from tests.gpu_util import lib_ready, torch_cuda

pytestmark = pytest.mark.gpu


def setup(batch=200, seed=5):
    torch = torch_cuda()
    hs = lib_ready()
    th = 0.3 * workloads.matrix(1, mlp.N_PARAMS, seed, "uniform")[0]
    X = workloads.matrix(batch, 10, seed + 1, "uniform")
    y = workloads.matrix(1, batch, seed + 2, "uniform")[0]
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    return hs, torch, th, X, y, f32


def test_forward_matches_oracle():
    hs, torch, th, X, y, f32 = setup()
    dth, dX = f32(th), f32(X)
    out = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    cache = torch.empty((X.shape[0], 192), dtype=torch.float32, device="cuda")
    hs._check(hs.lib().hsumma_mlp_forward(X.shape[0], dth.data_ptr(), dX.data_ptr(),
                                           out.data_ptr(), cache.data_ptr(), None))
    hs.sync(None)
    th32 = th.astype(np.float32).astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    want, oc = mlp.forward(th32, X32)
    assert np.allclose(out.cpu().numpy(), want, rtol=1e-4, atol=1e-5)
    z1 = oc[0][1]
    assert np.allclose(cache.cpu().numpy()[:, :64], z1, rtol=1e-4, atol=1e-5)


def test_backward_matches_oracle_gradient():
    hs, torch, th, X, y, f32 = setup()
    dth, dX, dy = f32(th), f32(X), f32(y)
    g = torch.empty(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    hs._check(hs.lib().hsumma_mlp_backward(X.shape[0], dth.data_ptr(), dX.data_ptr(),
                                            dy.data_ptr(), g.data_ptr(), loss.data_ptr(), None))
    hs.sync(None)
    th32 = th.astype(np.float32).astype(np.float64)
    L, G = mlp.loss_and_grad(th32, X.astype(np.float32).astype(np.float64),
                             y.astype(np.float32).astype(np.float64))
    got = g.cpu().numpy().astype(np.float64)
    assert loss.item() == pytest.approx(L, rel=1e-4)
    scale = np.abs(G).max()
    assert np.max(np.abs(got - G)) <= 1e-4 * scale


def test_adam_matches_oracle():
    hs, torch, th, X, y, f32 = setup()
    gr = workloads.matrix(1, mlp.N_PARAMS, 9, "uniform")[0]
    m0 = 0.1 * workloads.matrix(1, mlp.N_PARAMS, 10, "uniform")[0]
    v0 = np.abs(0.1 * workloads.matrix(1, mlp.N_PARAMS, 11, "uniform")[0])
    dth, dg, dm, dv = f32(th), f32(gr), f32(m0), f32(v0)
    hs._check(hs.lib().hsumma_mlp_adam(mlp.N_PARAMS, dth.data_ptr(), dg.data_ptr(), dm.data_ptr(),
                                        dv.data_ptr(), 3, 1e-3, 0.9, 0.999, 1e-8, None))
    hs.sync(None)
    f = lambda a: np.asarray(a).astype(np.float32).astype(np.float64)
    # the kernel trains in fp32: its hyperparameters are the fp32 roundings
    # (0.999 is not exact in fp32, so 1 - beta2 differs by ~1e-5 relative)
    hp = {k: float(f(v)) for k, v in dict(lr=1e-3, b1=0.9, b2=0.999, eps=1e-8).items()}
    t1, m1, v1 = mlp.adam_step(f(th), f(gr), f(m0), f(v0), 3, **hp)
    assert np.allclose(dth.cpu().numpy(), t1, rtol=1e-5, atol=1e-7)
    assert np.allclose(dm.cpu().numpy(), m1, rtol=1e-5, atol=1e-7)
    assert np.allclose(dv.cpu().numpy(), v1, rtol=1e-5, atol=1e-9)


def test_bf16_pick_and_argmin():
    hs, torch, th, X, y, f32 = setup(batch=777)
    dth, dX = f32(th), f32(X)
    pred = torch.empty(777, dtype=torch.float32, device="cuda")
    best = torch.empty(1, dtype=torch.int32, device="cuda")
    hs._check(hs.lib().hsumma_mlp_pick(777, dth.data_ptr(), dX.data_ptr(), pred.data_ptr(),
                                        best.data_ptr(), None))
    hs.sync(None)
    p = pred.cpu().numpy()
    want, _ = mlp.forward(th, X)
    # bf16 weights and activations: about 3 significant digits
    assert np.max(np.abs(p - want)) <= 0.05 * (np.abs(want).max() + 1)
    assert int(best.item()) == int(np.argmin(p))


def test_training_reduces_loss_on_device():
    hs, torch, th, X, y, f32 = setup(batch=256)
    target = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]
    dth, dX, dy = f32(0.5 * th), f32(X), f32(target)
    g = torch.empty(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(g)
    v = torch.zeros_like(g)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    lib = hs.lib()
    first = None
    for t in range(1, 301):
        hs._check(lib.hsumma_mlp_backward(256, dth.data_ptr(), dX.data_ptr(), dy.data_ptr(),
                                          g.data_ptr(), loss.data_ptr(), None))
        if first is None:
            first = loss.item()
        hs._check(lib.hsumma_mlp_adam(mlp.N_PARAMS, dth.data_ptr(), g.data_ptr(), m.data_ptr(),
                                      v.data_ptr(), t, 3e-3, 0.9, 0.999, 1e-8, None))
    hs.sync(None)
    assert loss.item() < 0.05 * first
