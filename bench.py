"""Benchmark: FP64-accurate TFLOP/s of C = A x B at M = N = K = 16384 on one
GB300, split-precision (bf16 slices, tcgen05) against native binary64 (DMMA),
each as a fraction of its roofline.

One step = one hsumma_gemm call on the split path: exponent scan, slicing,
the HSUMMA diagonal products on the tensor cores, exact recombination, on
seeded uniform[-1, 1] inputs already resident in HBM (each 2 GiB, larger than
L2, so no flush is needed between steps).  The library records CUDA events
around each stage of the timed steps (hsumma_stage_timing), which give the
dominant kernel's duration for the roofline.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (the plain binary64 triple loop) on a
bounded sample of the same product (a band of rows of C) on the host cores.

The library is single-GPU: its cluster kernels deliver panels by TMA multicast
inside a thread-block cluster, and no run of it spans two or more GPUs.  Under
torchrun with WORLD_SIZE > 1 the native arm therefore launches nothing: rank 0
prints one line with an "unavailable" reason and every rank exits 0.  The
reference arm (CPU only) runs on rank 0 alone; the other ranks exit 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIZE = 16384
METRIC = "FP64-accurate TFLOP/s at n=16384, split-precision vs native FP64, % of roofline"
SPLIT = dict(P=128, Q=64, G=4096, b=64, Bouter=512, kind="bf16", slices=4)
NATIVE = dict(P=128, Q=128, G=8192, b=32, Bouter=128)
WORKLOAD = ("split_vs_fp64_16384: M=N=K=16384, A,B uniform[-1,1] (SplitMix64 seeds 1002/2002), "
            "bf16 slices S=4 of 9-bit digits (10 pair products), virtual grid 128x64 of 128x256 blocks, "
            "G=4096 groups of 2x1 (each group one CTA pair: the in-group B broadcast is the "
            "two-SM MMA; persistent clusters, one launch per diagonal), b=64, B=512 "
            "(owner L2 prefetch); "
            "native fp64 beside it on a 128x128 grid, G=8192 groups of 2x1 (2-CTA clusters), "
            "b=32, B=128")


def configure(n):
    """Grids for an n x n x n product: 128 x 256 blocks (split) and 128 x 128
    blocks (binary64), groups of 2 x 1 processors."""
    global N_SIZE, SPLIT, NATIVE, WORKLOAD
    if n % 256:
        raise SystemExit("--size must be a multiple of 256")
    N_SIZE = n
    SPLIT = dict(SPLIT, P=n // 128, Q=n // 256, G=max(1, (n // 128) * (n // 256) // 2))
    NATIVE = dict(NATIVE, P=n // 128, Q=n // 128, G=max(1, (n // 128) ** 2 // 2))
    if n != 16384:
        WORKLOAD = (f"split_vs_fp64_{n}: M=N=K={n}, bf16 S={SPLIT['slices']}, grid {n // 128}x{n // 256} of "
                    f"128x256 blocks, G={SPLIT['G']} (2x1 groups, CTA pairs), b=64, "
                    f"B={SPLIT['Bouter']}; native fp64 grid {n // 128}x{n // 128}, "
                    f"G={NATIVE['G']}")


def flops(n=None):
    n = N_SIZE if n is None else n
    return 2.0 * n ** 3


def traffic_record(kernel="bf16_pair_kernel"):
    """(DRAM bytes per product stage from the committed ncu record, whether
    the kernel's sources -- its file and the device headers it includes -- are
    still the ones the counters were taken on); (None, False) without one."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return rec["dram_bytes_read"] + rec["dram_bytes_write"], \
            h.hexdigest()[:16] == rec["sha256_prefix"]
    except Exception:
        return None, False


def measured_traffic(kernel="bf16_pair_kernel"):
    """The record's bytes, only while the kernel is unchanged since (else None)."""
    value, current = traffic_record(kernel)
    return value if current else None


MULTI_GPU_UNAVAILABLE = ("single-GPU library: its cluster kernels deliver panels by TMA "
                         "multicast, so no run of it spans two or more GPUs")


def multi_gpu_line(world: int):
    """The native arm's line under torchrun with world > 1: nothing runs."""
    return {"metric": METRIC, "impl": "native", "n_gpus": world,
            "unavailable": MULTI_GPU_UNAVAILABLE}


def timeline_summary(tl, n):
    """One host-buffer call's pipeline, from its timed phases: the device time
    of the block products (each from the arrival of its column block of B, so
    the first includes the wait for A's first row block), when the first one
    started (the exposed copy-in), the time after the last one (the exposed
    copy-out), the products' waits for data in between, and the host-link
    rates the copies ran at."""
    prod = sorted((a, b) for nm, r, c, a, b in tl if nm == "product")
    cin = [(a, b) for nm, r, c, a, b in tl if nm in ("B in", "A in")]
    cout = [(a, b) for nm, r, c, a, b in tl if nm == "C out"]
    if not prod:
        return {}
    waits = sum(max(0.0, prod[i][0] - prod[i - 1][1]) for i in range(1, len(prod)))
    busy_in = sum(b - a for a, b in cin)
    busy_out = sum(b - a for a, b in cout)
    return {"products_ms": round(sum(b - a for a, b in prod), 2),
            "first_block_at_ms": round(prod[0][0], 2),
            "waits_between_ms": round(waits, 2),
            "after_last_product_ms": round(max(b for a, b in cout) - prod[-1][1], 2),
            "h2d_gbps": round(2 * 8 * n * n / busy_in / 1e6, 1) if busy_in > 0 else None,
            "d2h_gbps": round(8 * n * n / busy_out / 1e6, 1) if busy_out > 0 else None}


def read_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(A, B, target_s=15.0):
    """The oracle triple loop on a band of rows of C, sized to about target_s
    seconds on all host cores; returns (TFLOP/s, rows, cores, seconds)."""
    from oracle import native
    cores = native.default_threads()
    n = A.shape[1]
    rows = 8
    while True:
        t0 = time.perf_counter()
        native.dgemm(A[:rows], B, nthreads=cores)
        dt = time.perf_counter() - t0
        if dt > target_s / 4 or rows >= A.shape[0]:
            break
        rows = min(A.shape[0], max(rows * 2, int(rows * target_s / max(dt, 1e-3) / 2)))
    return 2.0 * rows * n * B.shape[1] / dt / 1e12, rows, cores, dt


def cpu_leg(A_band, A_rows, B, ri, cj, sampled):
    """The bench's CPU leg (with the reference arm, the only code here that runs
    the oracle): the plain binary64 triple loop timed on a band of rows of C
    (cpu_baseline), and the compensated (Dot2) reference of the sampled
    entries, against which the GPU results' errors max |C - C^| / (|A||B|)
    are reported."""
    from oracle import native, split
    rate, rws, cores, dt = cpu_oracle_rate(A_band, B, target_s=12.0)
    cpu = {"value": rate, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
           "sample": f"{rws} rows of C at n={B.shape[0]} by the plain binary64 triple loop "
                     f"({dt:.1f} s)"}
    import numpy as np
    ref, absab = native.dot2_entries(A_rows, B, ri, cj)
    acc = {f"{k}_max_rel_err": split.max_rel_error(v, ref, absab) for k, v in sampled.items()}
    acc["tolerance_2Ku"] = split.tolerance(B.shape[0])
    acc["reference"] = (f"Dot2 on {len(cj)} entries: every 128-tile border row and column "
                        f"and seeded ones")
    return cpu, acc


def run_reference(args, rank, world):
    import numpy as np
    import workloads
    out = {"impl": "reference"}
    if rank != 0:
        return None
    n = N_SIZE
    # bounded sample: a band of rows of A (whole) times B; B is the full matrix
    B = workloads.matrix(n, n, 2002, "uniform")
    A = workloads.matrix(256, n, 1002, "uniform")
    rate, rows, cores, dt = cpu_oracle_rate(A, B, target_s=float(os.environ.get("HS_REF_S", 12)))
    times = []
    for _ in range(args.warmup):
        from oracle import native
        native.dgemm(A[:rows], B, nthreads=cores)
    from oracle import native
    for _ in range(args.steps):
        t0 = time.perf_counter()
        native.dgemm(A[:rows], B, nthreads=cores)
        times.append(time.perf_counter() - t0)
    t = max(times) if times else dt
    value = 2.0 * rows * n * n / t / 1e12
    sample = f"{rows} rows of C = A x B at n=16384 (plain binary64 triple loop), per step"
    out.update({
        "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "inputs larger than L2 (2 GiB each)",
                   "parallelism": "single GPU"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    })
    return out


def run_table(sections):
    """Throughput of the five workloads' configurations (one JSON line each,
    "table" rows; no oracle: the accuracy of these launches is checked by the
    GPU tests).  Times are CUDA events on the launching stream, best of the
    runs, each run after an L2 flush."""
    import numpy as np
    import torch
    import paper_1306_4161_gb300 as hs
    import workloads
    hs.init(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dmma = hs.peak("dmma", 4000) / 1e12
    imma = hs.peak("imma", 4000) / 1e12
    bf16 = read_peaks().get("bf16_tflops_sustained") or 1700.0

    def timed(fn, reps=1, warm=True):
        if warm:               # also grows the split path's workspace
            fn()
            hs.sync()
        best, stages = float("inf"), None
        for _ in range(reps):
            flush.zero_()
            hs.stage_timing(True)
            e0.record()
            fn()
            e1.record()
            hs.stage_timing(False)
            e1.synchronize()
            t = e0.elapsed_time(e1)
            if t < best:
                best, stages = t, hs.stage_times()[0]
        hs.sync()
        return best, stages

    def emit(**kw):
        print(json.dumps({"table": True, **kw}), flush=True)

    def product(M, N, K, distA, distB, seedA, seedB):
        return (workloads.matrix_torch(M, K, seedA, distA, device="cuda"),
                workloads.matrix_torch(K, N, seedB, distB, device="cuda"),
                torch.empty((M, N), dtype=torch.float64, device="cuda"))

    if 0 in sections:
        A, B, C = product(512, 512, 512, "uniform", "uniform", 1000, 2000)
        ms, _ = timed(lambda: hs.gemm(A, B, out=C, P=4, Q=4, G=4, b=32, Bouter=64), reps=20)
        tf = 2 * 512 ** 3 / ms / 1e9
        emit(workload="hsumma_fp64_512", path="fp64", cfg="4x4 G=4 b=32 B=64", ms=ms,
             tflops=tf, frac_of_dmma=tf / dmma)
    if 1 in sections:
        n = 8192
        A, B, C = product(n, n, n, "uniform", "uniform", 1001, 2001)
        for G in (1, 4, 16, 64, 256):
            for b in (32, 64, 128):
                for Bo in (b, 2 * b, 4 * b):
                    ms, _ = timed(lambda: hs.gemm(A, B, out=C, P=16, Q=16, G=G, b=b, Bouter=Bo),
                                  warm=False)
                    tf = 2 * n ** 3 / ms / 1e9
                    emit(workload="hsumma_fp64_8192_gsweep", path="fp64",
                         cfg=f"16x16 G={G} b={b} B={Bo}", cluster=hs.group_shape(16, 16, G)[2:],
                         ms=ms, tflops=tf, frac_of_dmma=tf / dmma, counters=hs.counters())
        del A, B, C
    if 2 in sections:
        n = 16384
        A, B, C = product(n, n, n, "uniform", "uniform", 1002, 2002)
        ms, _ = timed(lambda: hs.gemm(A, B, out=C, **NATIVE), warm=False)
        tf = 2 * n ** 3 / ms / 1e9
        emit(workload="split_vs_fp64_16384", path="fp64",
             cfg=" ".join(f"{k}={v}" for k, v in NATIVE.items()), ms=ms, tflops=tf,
             frac_of_dmma=tf / dmma)
        split_cfg = {k: v for k, v in SPLIT.items() if k not in ("kind", "slices")}
        for kind, slices, cfg, peak in (
                ("bf16", range(3, 7), split_cfg, bf16),
                ("int8", range(3, 9), dict(P=128, Q=128, G=1, b=128, Bouter=2048), imma)):
            for S in slices:
                ms, st = timed(lambda: hs.gemm(A, B, out=C, kind=kind, slices=S, **cfg))
                npairs = S * (S + 1) // 2
                unit = npairs * 2 * n ** 3 / st[2] / 1e9
                emit(workload="split_vs_fp64_16384", path=kind, slices=S,
                     cfg=" ".join(f"{k}={v}" for k, v in cfg.items()), ms=ms,
                     tflops=2 * n ** 3 / ms / 1e9, stage_ms=st,
                     product_kernel={"achieved": unit, "peak": peak, "frac": unit / peak})
        del A, B, C
    if 3 in sections:
        M, N, K = 24576, 16384, 32768
        A, B, C = product(M, N, K, "normal_spiked", "normal", 1003, 2003)
        for G in (1, 3, 4, 12, 16, 48):
            ms, _ = timed(lambda: hs.gemm(A, B, out=C, P=12, Q=16, G=G, b=32, Bouter=128),
                          warm=False)
            tf = 2 * M * N * K / ms / 1e9
            emit(workload="rect_24576x16384x32768", path="fp64", cfg=f"12x16 G={G} b=32 B=128",
                 cluster=hs.group_shape(12, 16, G)[2:], ms=ms, tflops=tf,
                 frac_of_dmma=tf / dmma)
        # S = 5: the fewest 9-bit slices within 2 K u on these spiked columns.
        # The automatic choice first: an explicit policy's pick is cached for
        # the automatic choice of the same product.
        for policy in ("auto", "model", "timed"):
            cfg, how = hs.choose(A, B, C, kind="bf16", slices=5, policy=policy)
            ms, st = timed(lambda: hs.gemm(A, B, out=C, kind="bf16", slices=5, P=cfg[0],
                                           Q=cfg[1], G=cfg[2], b=cfg[3], Bouter=cfg[4]))
            emit(workload="rect_24576x16384x32768", path="bf16", slices=5, policy=policy,
                 chosen_by=how,
                 cfg=cfg, ms=ms, tflops=2 * M * N * K / ms / 1e9, stage_ms=st)
    if 4 in sections:
        # the two layouts of the grid at the same P x Q: block-checkerboard
        # (Algorithm 1) and block-cyclic (sub-tiles dealt round robin); aligned
        # grids do the same work in both, ragged ones sweep partial sub-tiles
        # in every block of the former and only at the matrix edge in the latter
        n = 16384
        A, B, C = product(n, n, n, "uniform", "uniform", 1002, 2002)
        for P, Q, G, note in ((128, 64, 4096, "aligned"), (120, 60, 3600, "ragged, many waves"),
                              (12, 12, 72, "ragged, one wave")):
            for layout in ("block", "cyclic"):
                cfg = dict(P=P, Q=Q, G=G, b=64, Bouter=512, kind="bf16", slices=SPLIT["slices"],
                           layout=layout)
                ms, st = timed(lambda: hs.gemm(A, B, out=C, **cfg), reps=2)
                npairs = SPLIT["slices"] * (SPLIT["slices"] + 1) // 2
                unit = npairs * 2 * n ** 3 / st[2] / 1e9
                emit(workload="layout_bf16_16384", layout=layout, grid=f"{P}x{Q}", G=G, note=note,
                     cluster=hs.group_shape(P, Q, G)[2:], ms=ms, tflops=2 * n ** 3 / ms / 1e9,
                     stage_ms=st, counters=hs.counters(),
                     product_kernel={"achieved": unit, "peak": bf16, "frac": unit / bf16})
        del A, B, C
        n = 8192
        A, B, C = product(n, n, n, "uniform", "uniform", 1001, 2001)
        for P, Q, G, note in ((16, 16, 16, "aligned"), (24, 24, 144, "ragged"),
                              (20, 20, 400, "ragged, flat")):
            for layout in ("block", "cyclic"):
                ms, _ = timed(lambda: hs.gemm(A, B, out=C, P=P, Q=Q, G=G, b=32, Bouter=128,
                                              layout=layout), warm=False)
                tf = 2 * n ** 3 / ms / 1e9
                emit(workload="layout_fp64_8192", layout=layout, grid=f"{P}x{Q}", G=G, note=note,
                     cluster=hs.group_shape(P, Q, G)[2:], ms=ms, tflops=tf,
                     frac_of_dmma=tf / dmma, counters=hs.counters())
        del A, B, C


# Small cases for profiler captures: (n, configuration).  Each run makes one
# warm-up product and then the product to capture (ncu -s 1 -c 1).
PROFILE_CASES = {
    # bf16 S = 4 on CTA pairs (2 x 1 groups): one persistent launch at this size
    "pair6144": (6144, dict(P=48, Q=24, G=576, b=64, Bouter=512, kind="bf16", slices=4)),
    # the same with the benchmark's launch policy at n = 16384: one persistent
    # launch per diagonal (four launches a product)
    "pair6144_diag": (6144, dict(P=48, Q=24, G=576, b=64, Bouter=512, kind="bf16", slices=4,
                                 launch=("per_diagonal", True))),
    # bf16 S = 4 on single CTAs, flat (64-processor software groups)
    "diag6144": (6144, dict(P=48, Q=24, G=18, b=64, Bouter=1024, kind="bf16", slices=4)),
    # int8 S = 5, flat
    "int8_4096": (4096, dict(P=32, Q=32, G=1, b=128, Bouter=2048, kind="int8", slices=5)),
    # binary64 with 2 x 2 clusters (inner level by multicast), and flat
    "fp64_2048_cluster": (2048, dict(P=16, Q=16, G=64, b=32, Bouter=128)),
    "fp64_2048_flat": (2048, dict(P=16, Q=16, G=256, b=32, Bouter=128)),
}


def run_mlp_profile():
    """The cost model's kernels on the committed training set, for a profiler:
    two training steps (backward, block reduction, Adam; a forward pass over
    256 samples after each), then the bf16 pick among the benchmark product's
    candidates (scoring and argmin)."""
    import paper_1306_4161_gb300 as hs
    from paper_1306_4161_gb300 import autotune
    hs.init(0)
    rows = autotune.load_samples(autotune.TUNING_DIR)
    X, y = autotune.sample_features(rows)
    autotune.train(X, y, steps=2, log=lambda *_: None, X_val=X[:256], y_val=y[:256],
                   check_every=1)
    model = autotune.read_model()
    M, N, K, kind, S = autotune.BENCH_PRODUCT
    cfgs = hs.candidates(M, N, K, kind, S)
    j = autotune.pick(model, M, N, K, kind, S, cfgs)
    print(json.dumps({"case": "mlp", "samples": int(X.shape[0]), "candidates": len(cfgs),
                      "pick": list(cfgs[j])}), flush=True)


def run_profile_case(name):
    """Two products of a small case (seeded uniform inputs), for a profiler
    to capture the second; prints the group shape and the counters."""
    if name == "mlp":
        run_mlp_profile()
        return
    import torch
    import paper_1306_4161_gb300 as hs
    import workloads
    n, cfg = PROFILE_CASES[name]
    cfg = dict(cfg)
    hs.init(0)
    if "launch" in cfg:
        hs.pair_launch(*cfg.pop("launch"))
    A = workloads.matrix_torch(n, n, 1002, "uniform", device="cuda")
    B = workloads.matrix_torch(n, n, 2002, "uniform", device="cuda")
    C = torch.empty((n, n), dtype=torch.float64, device="cuda")
    for _ in range(2):
        hs.gemm(A, B, out=C, **cfg)
        hs.sync()
    print(json.dumps({"case": name, "n": n, "group_shape": hs.group_shape(cfg["P"], cfg["Q"],
                                                                          cfg["G"]),
                      "counters": hs.counters()}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--native-steps", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end (host buffers) measurement")
    ap.add_argument("--e2e-calls", type=int, default=9,
                    help="timed host-buffer calls (the e2e value is their median)")
    ap.add_argument("--size", type=int, default=N_SIZE,
                    help="n of the n x n x n product (multiple of 256; default 16384)")
    ap.add_argument("--table", default=None,
                    help="comma-separated workload numbers 0..3 (4: block against "
                         "block-cyclic layout): print throughput rows of their "
                         "configurations instead of the benchmark line")
    ap.add_argument("--profile-case", default=None, choices=sorted(PROFILE_CASES) + ["mlp"],
                    help="run one small case twice (for a profiler) instead of the benchmark")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    configure(args.size)
    if args.table is not None:
        run_table({int(x) for x in args.table.split(",") if x.strip()})
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        # no kernel of this library runs on two or more GPUs (module docstring)
        if rank == 0:
            print(json.dumps(multi_gpu_line(world)), flush=True)
        return

    import numpy as np
    import torch
    import paper_1306_4161_gb300 as hs
    import workloads

    torch.cuda.set_device(local)
    hs.init(local)
    n = N_SIZE
    dA = workloads.matrix_torch(n, n, 1002, "uniform", device="cuda")
    dB = workloads.matrix_torch(n, n, 2002, "uniform", device="cuda")
    dC = torch.empty((n, n), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()

    def step():
        hs.gemm(dA, dB, out=dC, **SPLIT)

    for _ in range(args.warmup):
        step()
    hs.sync()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hs.stage_timing(True)
    launches0 = hs.launches()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    launches = hs.launches() - launches0
    hs.stage_timing(False)
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    hs.sync()
    value = flops() / (ms * 1e-3) / 1e12

    # per-stage device time of the timed steps (events the library recorded
    # around each kernel on the launching stream while the steps ran)
    stage_ms, ncalls = hs.stage_times()
    dur = np.array(stage_ms) / max(ncalls, 1)
    counters = hs.counters()
    S = SPLIT["slices"]
    npairs = S * (S + 1) // 2
    peaks = read_peaks()
    bf16_peak = peaks.get("bf16_tflops_sustained") or 1700.0
    gemm_tflops = npairs * flops() / (dur[2] * 1e-3) / 1e12
    burst = peaks.get("bf16_tflops") or 1900.0
    # the tensor pipe's own rate at the clock sampled during the timed steps:
    # 8192 bf16 flops per cycle and SM (hsumma_peak(TC05_*) measures it)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    pipe = 8192.0 * sms * clk["sm_mhz"] * 1e6 / 1e12 if clk.get("sm_mhz") else None
    roofline = {"bound": "tensor", "kernel": "bf16_pair_kernel",
                "achieved": gemm_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                "frac": gemm_tflops / bf16_peak,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (measured)",
                "frac_of_burst": gemm_tflops / burst,
                "frac_of_tensor_pipe_at_clock": gemm_tflops / pipe if pipe else None,
                "algorithmic": f"{npairs} bf16 products x 2 n^3 per product stage "
                               f"({S} launches of the kernel, one per diagonal)",
                "duration_ms": dur[2], "timed_stages": ncalls,
                "traffic": measured_traffic() if N_SIZE == 16384 else None,
                "traffic_unit": "bytes per product stage (ncu dram read + write), scaled from "
                                "a capture at n = 6144 (profiles/traffic.json)"}
    if N_SIZE == 16384 and roofline["traffic"] is None:
        # the last capture, taken on an earlier build of the kernel (the same
        # copy schedule, or not: see the record's note)
        roofline["traffic_previous_capture"] = traffic_record()[0]
    breakdown_ms = {"exponent_scan": dur[0], "slicing": dur[1], "diagonal_products": dur[2],
                    "recombination": dur[3]}

    # end to end through the C ABI with host buffers (pinned), copies inside
    e2e = None
    if not args.no_e2e:
        hA = dA.cpu().pin_memory()
        hB = dB.cpu().pin_memory()
        hC = torch.empty((n, n), dtype=torch.float64).pin_memory()
        hs.gemm_host(hA, hB, hC, **SPLIT)
        # every call with its pipeline phases timed (CUDA events on the streams
        # that ran them): where the time above the device time goes, call by call
        calls, lines = [], []
        hs.stage_timing(True)
        for _ in range(args.e2e_calls):
            t0 = time.perf_counter()
            hs.gemm_host(hA, hB, hC, **SPLIT)
            calls.append(time.perf_counter() - t0)
            lines.append(hs.host_timeline())
        hs.stage_timing(False)
        te = float(np.median(calls))
        med = int(np.argsort(calls)[len(calls) // 2])
        e2e = {"value": flops() / te / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": 2 * 8 * n * n, "d2h_bytes_per_step": 8 * n * n,
               "ms_per_step": te * 1e3, "of": f"median of {len(calls)} calls",
               "calls": [dict(call_ms=round(c * 1e3, 1), **timeline_summary(tl, n))
                         for c, tl in zip(calls, lines)],
               "median_call_phases_ms": [[nm, r, c, round(a, 2), round(b, 2)]
                                         for nm, r, c, a, b in lines[med]]}
        # this box's pinned host-link rates (outside the timed region): the
        # copies alone need max(H2D bytes / H2D rate, D2H bytes / D2H rate)
        scratch = torch.empty_like(dA)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        rates = {}
        for name, dst, src in (("h2d", scratch, hA), ("d2h", hA, scratch)):
            best = float("inf")
            for _ in range(3):
                c0.record(stream)
                dst.copy_(src, non_blocking=True)
                c1.record(stream)
                c1.synchronize()
                best = min(best, c0.elapsed_time(c1))
            rates[name] = src.numel() * 8 / best / 1e6
        e2e["link_gbps"] = {k: round(v, 1) for k, v in rates.items()}
        e2e["copy_floor_ms"] = max(2 * 8 * n * n / rates["h2d"], 8 * n * n / rates["d2h"]) / 1e6
        del hA, hB, hC, scratch

    # sampled entries of the split result (accuracy is computed in the CPU leg):
    # every tile-border row and column (128 x 128 tiles) and seeded ones, their
    # cross product column by column
    x = workloads.splitmix64(77, 0, 192)
    rows = set((x[:64] % np.uint64(n)).astype(np.int64).tolist())
    cols = set((x[64:] % np.uint64(n)).astype(np.int64).tolist())
    for b0 in range(0, n, 128):
        rows.update((b0, min(n, b0 + 128) - 1))
        cols.update((b0, min(n, b0 + 128) - 1))
    rows = np.array(sorted(rows), dtype=np.int64)
    cols = np.array(sorted(cols), dtype=np.int64)
    ri = np.tile(np.arange(rows.size, dtype=np.int64), cols.size)
    cj = np.repeat(cols, rows.size)
    ir, ic = torch.as_tensor(rows, device="cuda"), torch.as_tensor(cols, device="cuda")
    sampled = {"split": dC[ir][:, ic].cpu().numpy().T.ravel()}

    # native binary64 path on the same inputs
    native_out = None
    if args.native_steps > 0:
        dC2 = torch.empty_like(dC)
        hs.gemm(dA, dB, out=dC2, **NATIVE)
        hs.sync()
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.native_steps):
            hs.gemm(dA, dB, out=dC2, **NATIVE)
        f1.record(stream)
        barrier()
        hs.sync()
        nms = f0.elapsed_time(f1) / args.native_steps
        ntf = flops() / (nms * 1e-3) / 1e12
        dmma_peak = hs.peak("dmma", 4000) / 1e12
        native_out = {"tflops": ntf, "ms_per_step": nms,
                      "roofline": {"bound": "fp64 tensor (DMMA)", "achieved": ntf,
                                   "peak": dmma_peak, "unit": "TFLOP/s",
                                   "frac": ntf / dmma_peak,
                                   "peak_source": "measured by hsumma_peak(DMMA) in this run"}}
        sampled["native"] = dC2[ir][:, ic].cpu().numpy().T.ravel()
        del dC2

    cpu, acc = None, {}
    if not args.no_cpu:
        cpu, acc = cpu_leg(dA[:256].cpu().numpy(), dA[ir].cpu().numpy(), dB.cpu().numpy(),
                           ri, cj, sampled)

    out = {
        "metric": METRIC,
        "value": value, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "inputs larger than L2 (2 GiB each)",
                   "parallelism": "single GPU"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clk,
        "breakdown_ms": breakdown_ms, "native_fp64": native_out, "accuracy": acc,
        "counters": counters,
    }
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
