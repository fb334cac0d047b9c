"""The automatic configuration on the GPU: every cluster shape its candidate
sets realise runs each kernel to the oracle's result; training by the library's
kernels follows the float64 oracle's Adam trajectory; hsumma_gemm with
P = Q = G = b = Bouter = 0 picks by the model, by timing, or from its cache and
computes the right product; and the committed model's picks (bf16 on the
device) stay within 10% of the exhaustive best on the held-out products and
beat the paper's standard setting."""
import math
import os

import numpy as np
import pytest

import workloads
from oracle import gpu_schedule as gsched
from oracle import mlp, split
from tests.gpu_util import lib_ready, torch_cuda

pytestmark = pytest.mark.gpu

TILES = {"fp64": (128, 128, 32, 448), "int8": (128, 128, 128, 640), "bf16": (128, 256, 64, 448)}
CLUSTERS = [(1, 2), (1, 4), (1, 8), (1, 16), (2, 1), (2, 2), (2, 4), (2, 8), (4, 1), (4, 2),
            (4, 3), (4, 4), (5, 2), (5, 3), (6, 2), (7, 2), (8, 1), (8, 2), (16, 1)]


def realise(cm, cn):
    """The smallest grid (P, Q, G) whose groups the oracle's rule realises as
    cm x cn clusters."""
    best = None
    for P in range(1, 17):
        for Q in range(1, 17):
            if best and P * Q >= best[0] * best[1]:
                continue
            for G in range(1, P * Q + 1):
                if (P * Q) % G:
                    continue
                ij = gsched.group_shape(P, Q, G)
                if ij and gsched.cluster_shape(P, Q, ij[0], ij[1], limit=16) == (cm, cn):
                    best = (P, Q, G)
                    break
    return best


@pytest.mark.parametrize("kind", ["fp64", "int8", "bf16"])
@pytest.mark.parametrize("cm,cn", CLUSTERS)
def test_every_cluster_shape_matches_oracle(kind, cm, cn):
    hs = lib_ready()
    torch = torch_cuda()
    P, Q, G = realise(cm, cn)
    assert hs.group_shape(P, Q, G)[2:] == (cm, cn)
    tm, tn, b, K = TILES[kind]
    M, N = P * tm - 29, Q * tn - 13          # short last blocks
    seed = 700 + 10 * cm + cn
    if kind == "fp64":
        A = workloads.matrix(M, K, seed, "smallint")
        B = workloads.matrix(K, N, seed + 1, "smallint")
        want = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
        S = 0
    else:
        A = workloads.matrix(M, K, seed, "uniform")
        B = workloads.matrix(K, N, seed + 1, "wide")
        S = 3
        want = split.split_gemm(A, B, S, kind)
    C = hs.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), P=P, Q=Q, G=G, b=b,
                Bouter=4 * b, kind=kind, slices=S)
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), want)


def test_training_follows_oracle_adam():
    hs = lib_ready()
    torch_cuda()
    from paper_1306_4161_gb300 import autotune
    n, steps, lr = 300, 25, 1e-3
    X = workloads.matrix(n, 10, 61, "uniform") * 3.0 + 1.0
    y = workloads.matrix(1, n, 62, "uniform")[0] * 2.0
    model = autotune.train(X.astype(np.float32), y, steps=steps, lr=lr, seed=63,
                           log=lambda *_: None)
    # the oracle's run: same standardisation and schedule, float64 arithmetic
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    mu, sd = X32.mean(axis=0), X32.std(axis=0)
    assert np.allclose(model["mean"], mu, rtol=1e-5, atol=1e-6)
    assert np.allclose(model["std"], sd, rtol=1e-5)
    Xn = f32((X32 - f32(model["mean"])) / f32(model["std"]))
    yn = f32((y - y.mean()) / y.std())
    th0 = f32(autotune.init_params(63))
    th, m, v = th0.copy(), np.zeros_like(th0), np.zeros_like(th0)
    hp = dict(b1=float(f32(0.9)), b2=float(f32(0.999)), eps=float(f32(1e-8)))
    losses = {}
    for t in range(1, steps + 1):
        lr_t = float(f32(lr * 0.5 * (1.0 + math.cos(math.pi * (t - 1) / steps))))
        losses[t], g = mlp.loss_and_grad(th, Xn, yn)   # loss before step t's update
        th, m, v = mlp.adam_step(th, g, m, v, t, lr=lr_t, **hp)
    moved = np.linalg.norm(th - th0)
    assert moved > 0
    assert np.linalg.norm(model["theta"].astype(np.float64) - th) <= 2e-2 * moved
    for t, L in model["history"]:
        assert L == pytest.approx(losses[int(t)], rel=2e-3), t
    assert losses[steps] < losses[1]


def _exact_pair(torch, M, N, K, seed):
    A = workloads.matrix(M, K, seed, "smallint")
    B = workloads.matrix(K, N, seed + 1, "smallint")
    want = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    return torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), want


def test_automatic_choice_by_model_then_cached():
    hs = lib_ready()
    torch = torch_cuda()
    from paper_1306_4161_gb300 import autotune
    theta = autotune.init_params(71)            # any network gives a valid pick
    hs.load_model(theta, np.zeros(10), np.ones(10))
    try:
        M, N, K = 1000, 1200, 512
        dA, dB, want = _exact_pair(torch, M, N, K, 72)
        cfg, how = hs.choose(dA, dB, kind="fp64")
        assert how == "model"
        assert cfg in hs.candidates(M, N, K, "fp64")
        X = (hs.features(M, N, K, hs.candidates(M, N, K, "fp64"), "fp64") - 0.0) / 1.0
        pred, _ = mlp.forward(theta.astype(np.float64), X.astype(np.float64))
        j = hs.candidates(M, N, K, "fp64").index(cfg)
        assert pred[j] <= pred.min() + 0.02 * (abs(pred.min()) + 1.0)   # bf16 scoring
        C = hs.gemm(dA, dB)                     # P = Q = G = b = Bouter = 0
        hs.sync()
        assert np.array_equal(C.cpu().numpy(), want)
        assert hs.choose(dA, dB, kind="fp64") == (cfg, "cached")
    finally:
        autotune.load_into_library()


def test_automatic_choice_by_timing_without_model():
    hs = lib_ready()
    torch = torch_cuda()
    hs.load_model(None, None, None)
    with pytest.raises(hs.HsummaError) as ei:
        hs.choose(*_exact_pair(torch, 64, 64, 64, 80)[:2], kind="fp64", policy="model")
    assert ei.value.status == -2
    M, N, K = 700, 900, 384
    dA, dB, want = _exact_pair(torch, M, N, K, 81)
    cfg, how = hs.choose(dA, dB, kind="fp64")
    assert how == "timed" and cfg in hs.candidates(M, N, K, "fp64")
    C = hs.gemm(dA, dB)
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), want)
    # the split path chooses the same way and stays bit-exact with the oracle
    A = workloads.matrix(300, 200, 82, "uniform")
    B = workloads.matrix(200, 520, 83, "wide")
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = hs.gemm(dA, dB, kind="bf16", slices=4)
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), split.split_gemm(A, B, 4, "bf16"))
    assert hs.choose(dA, dB, kind="bf16", slices=4)[1] == "cached"
    from paper_1306_4161_gb300 import autotune
    autotune.load_into_library()
    # loading drops the cache; 300 x 520 x 200 lies below the model's trained
    # sizes, so the automatic choice verifies the model's pick by timing
    assert hs.choose(dA, dB, kind="bf16", slices=4)[1] == "verified"
    hs.load_model_range(None, None)
    assert hs.choose(dA, dB, kind="bf16", slices=4)[1] == "model"
    autotune.load_into_library()


def test_automatic_choice_verifies_outside_the_trained_range():
    """S = 7 was never trained on (bf16 samples hold S = 3..6): the automatic
    choice times the model's four best-predicted candidates there, and the
    best-predicted of every cluster shape they leave out, and caches that
    pick; inside the range (S = 5, same sizes) it takes the model's."""
    hs = lib_ready()
    torch = torch_cuda()
    from paper_1306_4161_gb300 import autotune
    if not os.path.exists(autotune.MODEL_PATH):
        pytest.skip("no committed model")
    autotune.load_into_library()
    n = 1536
    A = workloads.matrix(n, n, 94, "uniform")
    B = workloads.matrix(n, n, 95, "uniform")
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    cfg, how = hs.choose(dA, dB, kind="bf16", slices=7)
    cands = hs.candidates(n, n, n, "bf16", 7)
    order = autotune.ranked(autotune.read_model(), n, n, n, "bf16", 7, cands)
    timed, shapes = [], set()
    for r, i in enumerate(order):
        sh = hs.group_shape(*cands[i][:3])[2:]
        if r < autotune.VERIFIED_CANDIDATES or sh not in shapes:
            timed.append(cands[i])
        shapes.add(sh)
    assert how == "verified" and cfg in timed
    assert hs.choose(dA, dB, kind="bf16", slices=7) == (cfg, "cached")
    cfg5, how5 = hs.choose(dA, dB, kind="bf16", slices=5)
    assert how5 == "model"
    # whatever the configuration, the split product is the same bits
    C = hs.gemm(dA, dB, kind="bf16", slices=7)
    C1 = hs.gemm(dA, dB, kind="bf16", slices=7, P=12, Q=6, G=36, b=64, Bouter=256)
    hs.sync()
    assert torch.equal(C, C1)


def test_library_loads_the_shipped_model():
    hs = lib_ready()
    torch = torch_cuda()
    from paper_1306_4161_gb300 import autotune
    if not os.path.exists(autotune.MODEL_PATH):
        pytest.skip("no committed model")
    autotune.load_into_library()
    A = workloads.matrix(2048, 1536, 90, "uniform")
    B = workloads.matrix(1536, 3072, 91, "uniform")
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    cfg, how = hs.choose(dA, dB, kind="bf16", slices=5)
    assert how == "model" and cfg in hs.candidates(2048, 3072, 1536, "bf16", 5)
    C = hs.gemm(dA, dB, kind="bf16", slices=5)
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), split.split_gemm(A, B, 5, "bf16"))


def test_committed_model_beats_paper_setting_on_held_out_products():
    hs = lib_ready()
    torch_cuda()
    from paper_1306_4161_gb300 import autotune
    path = os.path.join(autotune.TUNING_DIR, "heldout.npz")
    if not (os.path.exists(path) and os.path.exists(autotune.MODEL_PATH)):
        pytest.skip("no committed tuning data")
    rep = autotune.evaluate(autotune.read_model(), autotune.load_heldout(path))
    print("HELDOUT", rep["model"], rep["paper_rule"])
    assert rep["model"]["n"] == 200
    assert rep["model"]["geomean"] <= 1.10
    assert rep["model"]["geomean"] < rep["paper_rule"]["geomean"]
    # the large products (M, N, K in [8192, 32768], bf16 and int8, and the
    # benchmark's product), which the model reaches by extrapolation in log2
    large = os.path.join(autotune.TUNING_DIR, "heldout_large.npz")
    if os.path.exists(large):
        rep = autotune.evaluate(autotune.read_model(), autotune.load_heldout(large))
        print("HELDOUT LARGE", rep["model"], rep["paper_rule"])
        assert rep["model"]["n"] >= 31
        assert rep["model"]["geomean"] <= 1.10
        assert rep["model"]["geomean"] < rep["paper_rule"]["geomean"]


def test_model_pick_holds_when_retimed():
    # the model's pick is re-timed, not read from the committed table: for ten
    # held-out products -- the smallest of each kind, three more of the
    # standard range, and the three smallest of the large extension (bf16 and
    # int8 with M, N, K in [8192, 32768]) -- the picked configuration and the
    # stored exhaustive best are timed afresh, back to back
    hs = lib_ready()
    torch_cuda()
    from paper_1306_4161_gb300 import autotune
    path = os.path.join(autotune.TUNING_DIR, "heldout.npz")
    large = os.path.join(autotune.TUNING_DIR, "heldout_large.npz")
    if not (os.path.exists(path) and os.path.exists(autotune.MODEL_PATH)):
        pytest.skip("no committed tuning data")
    model = autotune.read_model()
    size = lambda h: h["M"] * h["N"] * h["K"] * max(h["S"], 1) ** 2
    held = sorted(autotune.load_heldout(path), key=size)
    chosen = [next(h for h in held if h["kind"] == k) for k in ("fp64", "int8", "bf16")]
    chosen += [h for h in held if h not in chosen][:4]
    if os.path.exists(large):
        chosen += sorted(autotune.load_heldout(large), key=size)[:3]
    assert len(chosen) >= 10
    timer = autotune.Timer()
    ratios = []
    for i, h in enumerate(chosen):
        cfgs = [tuple(int(v) for v in c) for c in h["cfg"]]
        j = autotune.pick(model, h["M"], h["N"], h["K"], h["kind"], h["S"], cfgs)
        best = cfgs[int(np.argmin(h["ms"]))]
        A, B, C = autotune.operands(h["M"], h["N"], h["K"], 900 + i)
        autotune.time_config(timer, A, B, C, best, h["kind"], h["S"], reps=1)
        t_pick = autotune.time_config(timer, A, B, C, cfgs[j], h["kind"], h["S"], reps=3)
        t_best = autotune.time_config(timer, A, B, C, best, h["kind"], h["S"], reps=3)
        ratios.append(t_pick / t_best)
        del A, B, C
    print("RETIMED", [round(r, 3) for r in ratios])
    # the stored ratios of these picks reach 1.10, and a large bf16 product's
    # time varies by several per cent from run to run (a pick stored at 1.05
    # has re-timed at 1.25)
    assert max(ratios) <= 1.35
    assert math.exp(np.mean(np.log(ratios))) <= 1.10


def test_analytic_policy_picks_and_computes():
    hs = lib_ready()
    torch = torch_cuda()
    from paper_1306_4161_gb300 import autotune
    m = autotune.read_model()
    if "analytic" not in m:
        pytest.skip("no committed analytic coefficients")
    hs.load_analytic(m["analytic"])
    M, N, K = 1200, 900, 640
    dA, dB, want = _exact_pair(torch, M, N, K, 95)
    cfg, how = hs.choose(dA, dB, kind="fp64", policy="analytic")
    assert how == "analytic" and cfg in hs.candidates(M, N, K, "fp64")
    T = hs.analytic_terms(M, N, K, hs.candidates(M, N, K, "fp64"), "fp64")
    assert hs.candidates(M, N, K, "fp64").index(cfg) == int(np.argmin(T @ m["analytic"][0]))
    C = hs.gemm(dA, dB, P=cfg[0], Q=cfg[1], G=cfg[2], b=cfg[3], Bouter=cfg[4])
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), want)
    hs.load_analytic(None)
    with pytest.raises(hs.HsummaError):
        hs.choose(dA, dB, kind="fp64", policy="analytic")
    autotune.load_into_library()


def test_verified_policy_times_the_models_four_best():
    # the verified policy: the loaded model's four best-predicted candidates,
    # each timed once on the operands; the pick is one of them, it computes the
    # product exactly, and it is cached for the automatic choice
    hs = lib_ready()
    torch = torch_cuda()
    from paper_1306_4161_gb300 import autotune
    if not os.path.exists(autotune.MODEL_PATH):
        pytest.skip("no committed model")
    model = autotune.load_into_library()
    M, N, K = 1536, 2304, 1280
    dA, dB, want = _exact_pair(torch, M, N, K, 97)
    cands = hs.candidates(M, N, K, "bf16", 4)
    top = [cands[i] for i in
           autotune.ranked(model, M, N, K, "bf16", 4, cands)[:autotune.VERIFIED_CANDIDATES]]
    cfg, how = hs.choose(dA, dB, kind="bf16", slices=4, policy="verified")
    assert how == "verified" and cfg in top
    C = hs.gemm(dA, dB, P=cfg[0], Q=cfg[1], G=cfg[2], b=cfg[3], Bouter=cfg[4], kind="bf16",
                slices=4)
    hs.sync()
    assert np.array_equal(C.cpu().numpy(), want)    # small integers: exact for any S
    assert hs.choose(dA, dB, kind="bf16", slices=4) == (cfg, "cached")
    autotune.load_into_library()                   # drops the cache again
