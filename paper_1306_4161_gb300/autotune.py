"""Autotuner and learned cost model of the automatic configuration.

The paper picks the number of groups by timing a few runs (Section V-A-1,
Section VI) and otherwise runs HSUMMA with G = sqrt(p) and b = B (Section IV);
it leaves the grid and the panel sizes to the user.  This module

  - times the library's candidate configurations (hsumma_candidates) of seeded
    products on the GPU (each run after an L2 flush, CUDA events, best of two);
  - trains the 10 -> 64 -> 64 -> 64 -> 1 GELU network on those timings on the
    GPU with the library's kernels (hsumma_mlp_backward, hsumma_mlp_adam:
    fp32, full batch, Adam with cosine-decayed step size, MSE on standardised
    ln t);
  - evaluates its picks (hsumma_mlp_pick: bf16 scoring + argmin on the device)
    on held-out products by the pick's time over the exhaustive best, beside the
    paper's standard setting (G = sqrt(p), b = B, one sub-tile per block);
  - loads a trained model into the library (hsumma_mlp_load) so that hsumma_gemm
    with P = Q = G = b = Bouter = 0 uses it.

    python -m paper_1306_4161_gb300.autotune collect --out DIR
    python -m paper_1306_4161_gb300.autotune collect-large --out DIR
    python -m paper_1306_4161_gb300.autotune train --data DIR --out DIR/cost_model.npz
    python -m paper_1306_4161_gb300.autotune range --data DIR --model DIR/cost_model.npz
    python -m paper_1306_4161_gb300.autotune evaluate --data DIR --model DIR/cost_model.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

import paper_1306_4161_gb300 as hs

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING_DIR = os.path.join(HERE, "tuning")
MODEL_PATH = os.path.join(TUNING_DIR, "cost_model.npz")
# candidates the library's verified policy times (the model's best-predicted)
VERIFIED_CANDIDATES = 4
KIND_CODE = {"fp64": 0, "int8": 1, "bf16": 2}
KIND_NAME = {v: k for k, v in KIND_CODE.items()}
LAYERS = ((10, 64), (64, 64), (64, 64), (64, 1))   # (fan_in, fan_out), row-major W[out][in]


def _workloads():
    root = os.path.dirname(HERE)
    if root not in sys.path:
        sys.path.insert(0, root)
    import workloads
    return workloads


# ---------------------------------------------------------------- the baseline
def _divisors(n: int) -> list[int]:
    small = [d for d in range(1, int(math.isqrt(n)) + 1) if n % d == 0]
    return sorted(set(small + [n // d for d in small]))


def paper_rule(M, N, K, kind, S):
    """HSUMMA's standard setting (Section IV: G = sqrt(p), b = B) on the grid of
    one kernel sub-tile per block: the valid group count nearest sqrt(p) on a
    log scale (ties: the smaller), b the stage width and B = b."""
    P, Q, _, b, _ = hs.candidates(M, N, K, kind, S)[0]
    p = P * Q
    valid = []
    for G in _divisors(p):
        try:
            hs.group_shape(P, Q, G)
            valid.append(G)
        except hs.HsummaError:
            pass
    half = 0.5 * math.log2(p)
    G = min(valid, key=lambda g: (abs(math.log2(g) - half), g))
    return (P, Q, G, b, b)


# ---------------------------------------------------------------- timing
class Timer:
    """Device time of one call on torch's current stream, after writing a
    buffer larger than the L2 (so every run starts with a cold L2)."""

    def __init__(self, flush_bytes: int = 256 << 20):
        import torch
        self.torch = torch
        self.flush = torch.empty(flush_bytes, dtype=torch.uint8, device="cuda")
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)

    def time(self, fn, reps: int = 2) -> float:
        best = math.inf
        for _ in range(reps):
            self.flush.zero_()
            self.e0.record()
            fn()
            self.e1.record()
            self.e1.synchronize()
            best = min(best, self.e0.elapsed_time(self.e1))
        return best


def operands(M, N, K, seed):
    """Seeded uniform[-1, 1) operands on the device and an output buffer (the
    values do not change any timing)."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    A = torch.rand((M, K), generator=g, dtype=torch.float64, device="cuda") * 2 - 1
    B = torch.rand((K, N), generator=g, dtype=torch.float64, device="cuda") * 2 - 1
    C = torch.empty((M, N), dtype=torch.float64, device="cuda")
    return A, B, C


def time_config(timer, A, B, C, cfg, kind, S, reps=2) -> float:
    P, Q, G, b, Bo = cfg
    try:
        return timer.time(lambda: hs.gemm(A, B, P=P, Q=Q, G=G, b=b, Bouter=Bo, kind=kind,
                                          slices=S, out=C), reps)
    except hs.HsummaError:
        return math.inf


# ---------------------------------------------------------------- collection
def collect(out_dir, n_samples=2000, per_shape=20, n_heldout=200, seed=4000, reps=2,
            log=print):
    """Training samples: per_shape seeded candidates of each of a seeded
    sequence of products, timed, until n_samples are taken.  Held-out set:
    every candidate plus the paper's setting of each of n_heldout other
    products.  Writes samples.npz (rows M, N, K, kind, S, P, Q, G, b, B, ms;
    column 11 numbers the product) and heldout.npz under out_dir."""
    import torch
    wl = _workloads()
    os.makedirs(out_dir, exist_ok=True)
    hs.init(0)
    timer = Timer()
    t0 = time.time()
    train_shapes = wl.tuning_shapes(4 * n_samples // per_shape + 8, seed + 1)
    held_shapes = wl.tuning_shapes(n_heldout, seed + 2)

    rows = []
    for i, (M, N, K, kind, S) in enumerate(train_shapes):
        if len(rows) >= n_samples:
            break
        A, B, C = operands(M, N, K, seed + 10 + i)
        cands = hs.candidates(M, N, K, kind, S)
        order = np.argsort(wl.splitmix64(seed + 100000 + i, 0, len(cands)), kind="stable")
        chosen = sorted(order[:min(per_shape, n_samples - len(rows))].tolist())
        time_config(timer, A, B, C, cands[0], kind, S, reps=1)     # grows the workspace
        for j in chosen:
            ms = time_config(timer, A, B, C, cands[j], kind, S, reps)
            rows.append((M, N, K, KIND_CODE[kind], S, *cands[j], ms, i))
        hs.sync()
        del A, B, C
        if (i + 1) % 10 == 0:
            log(f"train {i + 1} shapes, {len(rows)} samples, {time.time() - t0:.0f}s")
    if n_samples > 0:
        rows = np.array(rows, dtype=np.float64)
        np.savez_compressed(os.path.join(out_dir, "samples.npz"), rows=rows)

    shape_rows, offs, cfgs, mss, base_cfg, base_ms = [], [0], [], [], [], []
    for i, (M, N, K, kind, S) in enumerate(held_shapes):
        A, B, C = operands(M, N, K, seed + 20000 + i)
        cands = hs.candidates(M, N, K, kind, S)
        time_config(timer, A, B, C, cands[0], kind, S, reps=1)
        ms = [time_config(timer, A, B, C, c, kind, S, reps) for c in cands]
        base = paper_rule(M, N, K, kind, S)
        bms = time_config(timer, A, B, C, base, kind, S, reps)
        hs.sync()
        shape_rows.append((M, N, K, KIND_CODE[kind], S))
        cfgs.extend(cands)
        mss.extend(ms)
        offs.append(len(cfgs))
        base_cfg.append(base)
        base_ms.append(bms)
        del A, B, C
        if (i + 1) % 10 == 0:
            log(f"held-out {i + 1}/{n_heldout} shapes, {time.time() - t0:.0f}s")
            _save_heldout(out_dir, shape_rows, offs, cfgs, mss, base_cfg, base_ms)
    _save_heldout(out_dir, shape_rows, offs, cfgs, mss, base_cfg, base_ms)
    torch.cuda.synchronize()
    log(f"collected in {time.time() - t0:.0f}s")


BENCH_PRODUCT = (16384, 16384, 16384, "bf16", 5)   # the benchmark's split product


def collect_large(out_dir, n_train=40, per_shape=10, n_heldout=30, seed=4000, reps=1,
                  log=print, samples_name="samples_large.npz"):
    """The large-product extension (M, N, K in [8192, 32768], bf16 and int8;
    workloads.tuning_shapes_large): training samples, per_shape seeded
    candidates of each of n_train products (samples_large.npz, product ids from
    100000), and a held-out set, every candidate of each of n_heldout other
    products and of the benchmark's product (heldout_large.npz).  One timed run
    per configuration (these products run 0.1 to several seconds)."""
    import torch
    wl = _workloads()
    os.makedirs(out_dir, exist_ok=True)
    hs.init(0)
    timer = Timer()
    t0 = time.time()
    rows = []
    for i, (M, N, K, kind, S) in enumerate(wl.tuning_shapes_large(n_train, seed + 5)):
        A, B, C = operands(M, N, K, seed + 30000 + i)
        cands = hs.candidates(M, N, K, kind, S)
        order = np.argsort(wl.splitmix64(seed + 200000 + i, 0, len(cands)), kind="stable")
        time_config(timer, A, B, C, cands[0], kind, S, reps=1)     # grows the workspace
        for j in sorted(order[:per_shape].tolist()):
            ms = time_config(timer, A, B, C, cands[j], kind, S, reps)
            rows.append((M, N, K, KIND_CODE[kind], S, *cands[j], ms, 100000 + i))
        hs.sync()
        del A, B, C
        torch.cuda.empty_cache()
        log(f"large train {i + 1}/{n_train} shapes, {time.time() - t0:.0f}s")
    if rows:
        np.savez_compressed(os.path.join(out_dir, samples_name),
                            rows=np.array(rows, dtype=np.float64))
    if n_heldout <= 0:
        return
    shapes = wl.tuning_shapes_large(n_heldout, seed + 6) + [BENCH_PRODUCT]
    shape_rows, offs, cfgs, mss, base_cfg, base_ms = [], [0], [], [], [], []
    for i, (M, N, K, kind, S) in enumerate(shapes):
        A, B, C = operands(M, N, K, seed + 40000 + i)
        cands = hs.candidates(M, N, K, kind, S)
        time_config(timer, A, B, C, cands[0], kind, S, reps=1)
        ms = [time_config(timer, A, B, C, c, kind, S, reps) for c in cands]
        base = paper_rule(M, N, K, kind, S)
        bms = time_config(timer, A, B, C, base, kind, S, reps)
        hs.sync()
        shape_rows.append((M, N, K, KIND_CODE[kind], S))
        cfgs.extend(cands)
        mss.extend(ms)
        offs.append(len(cfgs))
        base_cfg.append(base)
        base_ms.append(bms)
        del A, B, C
        torch.cuda.empty_cache()
        log(f"large held-out {i + 1}/{len(shapes)} shapes, {time.time() - t0:.0f}s")
        _save_heldout(out_dir, shape_rows, offs, cfgs, mss, base_cfg, base_ms,
                      name="heldout_large.npz")
    log(f"collected the large products in {time.time() - t0:.0f}s")


def _save_heldout(out_dir, shape_rows, offs, cfgs, mss, base_cfg, base_ms,
                  name="heldout.npz"):
    np.savez_compressed(os.path.join(out_dir, name),
                        shapes=np.array(shape_rows, dtype=np.int64),
                        offsets=np.array(offs, dtype=np.int64),
                        cfg=np.array(cfgs, dtype=np.int64).reshape(-1, 5),
                        ms=np.array(mss, dtype=np.float64),
                        base_cfg=np.array(base_cfg, dtype=np.int64).reshape(-1, 5),
                        base_ms=np.array(base_ms, dtype=np.float64))


def load_heldout(path):
    d = np.load(path)
    n = len(d["shapes"])
    out = []
    for i in range(n):
        a, b = int(d["offsets"][i]), int(d["offsets"][i + 1])
        M, N, K, kc, S = (int(v) for v in d["shapes"][i])
        out.append(dict(M=M, N=N, K=K, kind=KIND_NAME[kc], S=S, cfg=d["cfg"][a:b],
                        ms=d["ms"][a:b], base_cfg=tuple(int(v) for v in d["base_cfg"][i]),
                        base_ms=float(d["base_ms"][i])))
    return out


def load_samples(data_dir):
    """Training rows: samples.npz and every samples_large*.npz present
    (untimed configurations, which failed to launch, left out)."""
    parts = [np.load(os.path.join(data_dir, "samples.npz"))["rows"]]
    for name in sorted(os.listdir(data_dir)):
        if name.startswith("samples_large") and name.endswith(".npz"):
            parts.append(np.load(os.path.join(data_dir, name))["rows"])
    rows = np.concatenate(parts)
    return rows[np.isfinite(rows[:, 10])]


def split_by_product(rows, frac=0.1):
    """Training and validation rows: the last frac of the products (column 11)
    are the validation set."""
    ids = np.unique(rows[:, 11])
    cut = ids[int(round(len(ids) * (1 - frac)))] if len(ids) > 1 else ids[-1] + 1
    return rows[rows[:, 11] < cut], rows[rows[:, 11] >= cut]


def sample_features(rows):
    """Raw features (n x 10) and ln t of training rows (M, N, K, kind, S, cfg, ms)."""
    X = np.empty((len(rows), 10), dtype=np.float32)
    for i, r in enumerate(rows):
        M, N, K, kc, S = (int(v) for v in r[:5])
        X[i] = hs.features(M, N, K, [tuple(int(v) for v in r[5:10])], KIND_NAME[kc], S)[0]
    return X, np.log(rows[:, 10])


# ---------------------------------------------------------------- training
def init_params(seed: int) -> np.ndarray:
    """Glorot-uniform weights from the seeded uniform stream, zero biases."""
    wl = _workloads()
    u = wl.matrix(1, hs.N_MLP_PARAMS, seed, "uniform")[0]
    theta = np.zeros(hs.N_MLP_PARAMS, dtype=np.float64)
    off = 0
    for fi, fo in LAYERS:
        lim = math.sqrt(6.0 / (fi + fo))
        theta[off:off + fi * fo] = lim * u[off:off + fi * fo]
        off += fi * fo + fo
    assert off == hs.N_MLP_PARAMS
    return theta.astype(np.float32)


def train(X, y, steps=6000, lr=1e-3, seed=4003, log=print, X_val=None, y_val=None,
          check_every=250, val_products=None):
    """Fit the network to ln t on the GPU: full-batch Adam (beta = 0.9, 0.999;
    eps = 1e-8) with the step size decayed on a cosine from lr to 0.  Features
    and targets are standardised with the training set's statistics.  Every
    check_every steps a checkpoint is scored and the best one kept: by the
    geometric mean of pick time over best time on val_products (products with
    every candidate timed, as load_heldout returns them) when given, else by
    the mean squared error on (X_val, y_val).  Returns the model dict."""
    import torch
    hs.init(0)
    lib = hs.lib()
    mean = X.mean(axis=0).astype(np.float32)
    std = X.std(axis=0).astype(np.float32)
    std[std == 0] = 1.0
    ym, ys = float(y.mean()), float(y.std()) or 1.0
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    dX, dy = dev((X - mean) / std), dev((y - ym) / ys)
    theta = dev(init_params(seed))
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    grad = torch.empty_like(theta)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    n = X.shape[0]
    stream = hs._stream_ptr()
    hist = []
    best = (math.inf, 0, None)
    if X_val is not None:
        dXv, yv = dev((X_val - mean) / std), (np.asarray(y_val) - ym) / ys
        pv = torch.empty(len(yv), dtype=torch.float32, device="cuda")
    if val_products:
        Xp = np.concatenate([hs.features(h["M"], h["N"], h["K"],
                                         [tuple(int(v) for v in c) for c in h["cfg"]],
                                         h["kind"], h["S"]) for h in val_products])
        dXp = dev((Xp - mean) / std)
        pp = torch.empty(Xp.shape[0], dtype=torch.float32, device="cuda")
        bounds = np.cumsum([0] + [len(h["ms"]) for h in val_products])
    for t in range(1, steps + 1):
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * (t - 1) / steps))
        hs._check(lib.hsumma_mlp_backward(n, theta.data_ptr(), dX.data_ptr(), dy.data_ptr(),
                                          grad.data_ptr(), loss.data_ptr(), stream))
        hs._check(lib.hsumma_mlp_adam(hs.N_MLP_PARAMS, theta.data_ptr(), grad.data_ptr(),
                                      m.data_ptr(), v.data_ptr(), t, lr_t, 0.9, 0.999, 1e-8,
                                      stream))
        if t == 1 or t % 500 == 0 or t == steps:
            hist.append((t, float(loss.item())))
            log(f"step {t}: mse {hist[-1][1]:.5f}")
        if (val_products or X_val is not None) and (t % check_every == 0 or t == steps):
            if val_products:
                hs._check(lib.hsumma_mlp_forward(Xp.shape[0], theta.data_ptr(), dXp.data_ptr(),
                                                 pp.data_ptr(), None, stream))
                pred = pp.cpu().numpy()
                r = [h["ms"][int(np.argmin(pred[a:b]))] / np.min(h["ms"])
                     for h, a, b in zip(val_products, bounds[:-1], bounds[1:])]
                err = float(np.exp(np.mean(np.log(r))))
            else:
                hs._check(lib.hsumma_mlp_forward(len(yv), theta.data_ptr(), dXv.data_ptr(),
                                                 pv.data_ptr(), None, stream))
                err = float(np.mean((pv.cpu().numpy().astype(np.float64) - yv) ** 2))
            if err < best[0]:
                best = (err, t, theta.cpu().numpy().copy())
    hs.sync()
    out = dict(theta=theta.cpu().numpy(), mean=mean, std=std, y_mean=np.float64(ym),
               y_std=np.float64(ys), history=np.array(hist))
    if best[2] is not None:
        what = "pick/best geomean" if val_products else "mse"
        log(f"kept step {best[1]}: validation {what} {best[0]:.5f}")
        out.update(theta=best[2], val_score=np.float64(best[0]), val_step=np.int64(best[1]),
                   lr=np.float64(lr), steps=np.int64(steps))
    return out


def save_model(model, path):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    np.savez(path, **model)


def read_model(path=MODEL_PATH):
    d = np.load(path)
    return {k: d[k] for k in d.files}


def load_into_library(path=MODEL_PATH):
    """Load the trained model at path into the library (hsumma_gemm's automatic
    choice then uses it), with the analytic model's coefficients when present."""
    m = read_model(path)
    hs.load_model(m["theta"], m["mean"], m["std"])
    if "analytic" in m:
        hs.load_analytic(m["analytic"])
    if "range_lo" in m:
        hs.load_model_range(m["range_lo"], m["range_hi"])
    return m


def trained_range(X):
    """Per mode kind (feature 8), the smallest and largest value of each
    feature over the training rows X (lo > hi for a kind without rows)."""
    lo = np.full((3, X.shape[1]), np.inf, dtype=np.float32)
    hi = np.full((3, X.shape[1]), -np.inf, dtype=np.float32)
    for k in range(3):
        sel = X[np.round(X[:, 8]).astype(int) == k]
        if len(sel):
            lo[k], hi[k] = sel.min(axis=0), sel.max(axis=0)
    return lo, hi


# ---------------------------------------------------------------- analytic model
def fit_analytic(rows):
    """Coefficients (3 kinds x 5 terms) of Section IV's model, read for this GPU
    (hsumma_analytic_terms), fitted per kind by non-negative least squares on
    the relative error sum_i ((model_i - t_i) / t_i)^2 of the training rows."""
    from scipy.optimize import nnls
    coef = np.zeros((3, 5))
    for kc in range(3):
        sel = rows[rows[:, 3] == kc]
        if len(sel) == 0:
            continue
        T = np.stack([hs.analytic_terms(int(r[0]), int(r[1]), int(r[2]),
                                        [tuple(int(v) for v in r[5:10])], KIND_NAME[kc],
                                        int(r[4]))[0] for r in sel])
        t = sel[:, 10] * 1e-3                      # seconds
        A = T / t[:, None]
        scale = np.maximum(np.abs(A).max(axis=0), 1e-300)   # column scaling for NNLS
        x, _ = nnls(A / scale, np.ones(len(t)))
        coef[kc] = x / scale
    return coef


def analytic_pick(coef, h) -> int:
    """Index of the candidate with the smallest analytic time."""
    cfgs = [tuple(int(v) for v in c) for c in h["cfg"]]
    T = hs.analytic_terms(h["M"], h["N"], h["K"], cfgs, h["kind"], h["S"])
    return int(np.argmin(T @ coef[KIND_CODE[h["kind"]]]))


def sampled_pick(h) -> int:
    """The paper's own tuning (Section V-A-1, Section VI): run a few group counts
    and keep the fastest -- here every candidate group count of the grid of one
    sub-tile per block, with b = B; index of the fastest by the timed table."""
    cfgs = [tuple(int(v) for v in c) for c in h["cfg"]]
    P0, Q0 = cfgs[0][:2]
    idx = [i for i, c in enumerate(cfgs) if c[:2] == (P0, Q0) and c[3] == c[4]]
    return min(idx, key=lambda i: h["ms"][i])


# ---------------------------------------------------------------- evaluation
def pick(model, M, N, K, kind, S, cfgs) -> int:
    """Index of the configuration the model picks: bf16 scoring and argmin on
    the device (hsumma_mlp_pick), as in the library's automatic choice."""
    import torch
    X = hs.features(M, N, K, cfgs, kind, S)
    Xn = (X - model["mean"]) / model["std"]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    dth, dX = dev(model["theta"]), dev(Xn)
    pred = torch.empty(len(cfgs), dtype=torch.float32, device="cuda")
    best = torch.empty(1, dtype=torch.int32, device="cuda")
    hs._check(hs.lib().hsumma_mlp_pick(len(cfgs), dth.data_ptr(), dX.data_ptr(),
                                       pred.data_ptr(), best.data_ptr(), hs._stream_ptr()))
    return int(best.item())


def ranked(model, M, N, K, kind, S, cfgs):
    """Candidate indices in order of the model's predicted time, scored as the
    library scores them (bf16 on the device, hsumma_mlp_pick's predictions)."""
    import torch
    X = hs.features(M, N, K, cfgs, kind, S)
    Xn = (X - model["mean"]) / model["std"]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    dth, dX = dev(model["theta"]), dev(Xn)
    pred = torch.empty(len(cfgs), dtype=torch.float32, device="cuda")
    best = torch.empty(1, dtype=torch.int32, device="cuda")
    hs._check(hs.lib().hsumma_mlp_pick(len(cfgs), dth.data_ptr(), dX.data_ptr(),
                                       pred.data_ptr(), best.data_ptr(), hs._stream_ptr()))
    return np.argsort(pred.cpu().numpy(), kind="stable")


def _stats(r):
    r = np.asarray(r, dtype=np.float64)
    return dict(geomean=float(np.exp(np.mean(np.log(r)))), mean=float(r.mean()),
                median=float(np.median(r)), p90=float(np.quantile(r, 0.9)), max=float(r.max()),
                within_10pct=float(np.mean(r <= 1.10)), n=int(r.size))


def evaluate(model, heldout, picker=None, ranker=None):
    """Ratios to the exhaustive best (the fastest candidate), over the held-out
    products, overall and per kind, of: the model's pick ("model"), the fastest
    of its VERIFIED_CANDIDATES best-predicted candidates by the timed table (the
    verified policy, "verified"), the paper's static setting G = sqrt(p), b = B
    ("paper_rule"), the paper's tuning by a few runs ("sampled") and, when the
    model carries its coefficients, the fitted analytic model ("analytic")."""
    cfgs_of = lambda h: [tuple(int(v) for v in c) for c in h["cfg"]]
    if picker is None:
        picker = lambda h: pick(model, h["M"], h["N"], h["K"], h["kind"], h["S"], cfgs_of(h))
        if ranker is None:
            ranker = lambda h: ranked(model, h["M"], h["N"], h["K"], h["kind"], h["S"],
                                      cfgs_of(h))
    coef = model.get("analytic") if isinstance(model, dict) else None
    rows = []
    for h in heldout:
        ms = h["ms"]
        best = float(np.min(ms))
        r = {"kind": h["kind"], "model": ms[picker(h)] / best, "paper_rule": h["base_ms"] / best,
             "sampled": ms[sampled_pick(h)] / best}
        if ranker is not None:
            r["verified"] = float(min(ms[i] for i in ranker(h)[:VERIFIED_CANDIDATES])) / best
        if coef is not None:
            r["analytic"] = ms[analytic_pick(coef, h)] / best
        rows.append(r)
    keys = [k for k in ("model", "verified", "analytic", "sampled", "paper_rule")
            if k in rows[0]]
    out = {k: _stats([r[k] for r in rows]) for k in keys}
    for kind in KIND_CODE:
        sel = [r for r in rows if r["kind"] == kind]
        if sel:
            out[kind] = {k: _stats([r[k] for r in sel]) for k in keys}
    return out


# ---------------------------------------------------------------- CLI
def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1306_4161_gb300.autotune")
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--out", default=TUNING_DIR)
    c.add_argument("--samples", type=int, default=2000)
    c.add_argument("--per-shape", type=int, default=20)
    c.add_argument("--heldout", type=int, default=200)
    c.add_argument("--seed", type=int, default=4000)
    t = sub.add_parser("train")
    t.add_argument("--data", default=TUNING_DIR)
    t.add_argument("--out", default=MODEL_PATH)
    t.add_argument("--steps", type=int, default=6000)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--seed", type=int, default=4003)
    t.add_argument("--seeds", type=int, default=1,
                   help="train from this many initialisations (seed, seed + 10, ...) and keep "
                        "the one that scores best on the validation products")
    t.add_argument("--val", default=os.path.join(TUNING_DIR, "validation.npz"),
                   help="products with every candidate timed (heldout.npz format) that select "
                        "the checkpoint; '' uses the training products' last 10 %% instead")
    cl = sub.add_parser("collect-large")
    cl.add_argument("--out", default=TUNING_DIR)
    cl.add_argument("--products", type=int, default=40)
    cl.add_argument("--per-shape", type=int, default=10)
    cl.add_argument("--heldout", type=int, default=30)
    cl.add_argument("--seed", type=int, default=4000)
    cl.add_argument("--samples-name", default="samples_large.npz",
                    help="file of the training samples (every samples_large*.npz trains)")
    r = sub.add_parser("range", help="record the training samples' feature range in a "
                                     "trained model (the automatic choice verifies by timing "
                                     "outside it)")
    r.add_argument("--data", default=TUNING_DIR)
    r.add_argument("--model", default=MODEL_PATH)
    e = sub.add_parser("evaluate")
    e.add_argument("--data", default=TUNING_DIR)
    e.add_argument("--model", default=MODEL_PATH)
    e.add_argument("--report", default=None)
    a = ap.parse_args(argv)
    if a.cmd == "collect":
        collect(a.out, a.samples, a.per_shape, a.heldout, a.seed)
    elif a.cmd == "train":
        rows = load_samples(a.data)
        if a.val:
            X, y = sample_features(rows)
            val = load_heldout(a.val)
            model = None
            for i in range(max(1, a.seeds)):
                m = train(X, y, a.steps, a.lr, a.seed + 10 * i, val_products=val)
                m["seed"] = np.int64(a.seed + 10 * i)
                if model is None or m["val_score"] < model["val_score"]:
                    model = m
            print(f"kept seed {int(model['seed'])}: validation {float(model['val_score']):.5f}")
        else:
            tr, va = split_by_product(rows)
            X, y = sample_features(tr)
            Xv, yv = sample_features(va)
            model = train(X, y, a.steps, a.lr, a.seed, X_val=Xv, y_val=yv)
        model["analytic"] = fit_analytic(rows)
        model["range_lo"], model["range_hi"] = trained_range(sample_features(rows)[0])
        save_model(model, a.out)
    elif a.cmd == "range":
        model = read_model(a.model)
        model["range_lo"], model["range_hi"] = trained_range(
            sample_features(load_samples(a.data))[0])
        save_model(model, a.model)
    elif a.cmd == "collect-large":
        collect_large(a.out, a.products, a.per_shape, a.heldout, a.seed,
                      samples_name=a.samples_name)
    else:
        hs.init(0)
        model = read_model(a.model)
        rep = evaluate(model, load_heldout(os.path.join(a.data, "heldout.npz")))
        large = os.path.join(a.data, "heldout_large.npz")
        if os.path.exists(large):
            held = load_heldout(large)
            rep["large"] = evaluate(model, held)
            bench = [h for h in held if (h["M"], h["N"], h["K"], h["kind"], h["S"]) ==
                     BENCH_PRODUCT]
            if bench:
                rep["large"]["bench_product"] = evaluate(model, bench)
        text = json.dumps(rep, indent=1)
        print(text)
        if a.report:
            with open(a.report, "w") as f:
                f.write(text + "\n")


if __name__ == "__main__":
    main()
