"""Python binding of libhsumma (single-GPU Hierarchical SUMMA for sm_103a).

Argument marshalling only: every step of C = A x B runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  The library must have
been built (paper_1306_4161_gb300._build.build(), or __graft_entry__.build());
importing works without it, but every call raises if it is missing.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "_build", "libhsumma.so")
HEADER = os.path.join(ROOT, "include", "hsumma.h")

FP64, INT8_SLICES, BF16_SLICES = 0, 1, 2
KINDS = {"fp64": FP64, "int8": INT8_SLICES, "bf16": BF16_SLICES}
LAYOUT_CYCLIC = 0x10000          # mode bit: block-cyclic layout of the virtual grid
LAYOUTS = {"block": 0, "cyclic": LAYOUT_CYCLIC}
PEAKS = {"dfma": 0, "dmma": 1, "imma": 2, "hmma_bf16": 3, "tc05_bf16": 4, "copy": 5,
         "tc05_bf16_pair": 6}
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_UNSUPPORTED", -3: "ERR_CUDA", -4: "ERR_TIMEOUT",
          -5: "ERR_NOT_INIT", -6: "ERR_NONFINITE"}
N_MLP_PARAMS = 9089


class HsummaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Counters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("a_loaded", "a_delivered", "b_loaded", "b_delivered", "l2_prefetch",
                 "tma_loads")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_lock = threading.Lock()
_lib = None
_i64, _i32, _vp, _dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p

_SIGS = {
    "hsumma_init": ([_i32], _i32),
    "hsumma_finalize": ([], None),
    "hsumma_group_shape": ([_i32, _i32, _i32] + [ctypes.POINTER(ctypes.c_int)] * 4, _i32),
    "hsumma_workspace_size": ([_i64, _i64, _i64, _i32, ctypes.POINTER(ctypes.c_size_t)], _i32),
    "hsumma_gemm": ([_i64, _i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64] + [_i32] * 6 + [_vp],
                    _i32),
    "hsumma_gemm_host": ([_i64, _i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64] + [_i32] * 6
                         + [_vp], _i32),
    "hsumma_get_counters": ([ctypes.POINTER(Counters)], _i32),
    "hsumma_launches": ([], ctypes.c_uint64),
    "hsumma_sync": ([_vp], _i32),
    "hsumma_last_error": ([], ctypes.c_char_p),
    "hsumma_split_exponents": ([_i64, _i64, _i64, _dp, _i64, _dp, _i64, _vp, _vp, _vp], _i32),
    "hsumma_split_slices": ([_i64, _i64, _i64, _dp, _i64, _dp, _i64, _vp, _vp, _i32, _i32,
                             _vp, _vp, _vp], _i32),
    "hsumma_split_planes": ([_i64, _i32, _i32], _i32),
    "hsumma_split_diagonals": ([_i64, _i64, _i64, _i32, _i32, _vp, _vp, _vp] + [_i32] * 5
                               + [_vp], _i32),
    "hsumma_split_recombine": ([_i64, _i64, _i64, _i32, _i32, _vp, _vp, _vp, _vp, _i64, _vp],
                               _i32),
    "hsumma_mlp_forward": ([_i32, _vp, _vp, _vp, _vp, _vp], _i32),
    "hsumma_mlp_backward": ([_i32, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "hsumma_mlp_backward_noalloc": ([_i32, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "hsumma_mlp_adam": ([_i32, _vp, _vp, _vp, _vp, _i32, ctypes.c_float, ctypes.c_float,
                         ctypes.c_float, ctypes.c_float, _vp], _i32),
    "hsumma_mlp_pick": ([_i32, _vp, _vp, _vp, _vp, _vp], _i32),
    "hsumma_mlp_load": ([_vp, _vp, _vp], _i32),
    "hsumma_mlp_range": ([_vp, _vp], _i32),
    "hsumma_mlp_in_range": ([_i64, _i64, _i64, _i32, _vp], _i32),
    "hsumma_pair_kernel": ([_i32], _i32),
    "hsumma_pair_launch": ([_i32], _i32),
    "hsumma_selftest_timeout": ([ctypes.c_longlong, _vp], _i32),
    "hsumma_stage_timing": ([_i32], _i32),
    "hsumma_stage_times": ([_vp, ctypes.POINTER(ctypes.c_int)], _i32),
    "hsumma_host_timeline": ([_vp, _i32, ctypes.POINTER(ctypes.c_int)], _i32),
    "hsumma_host_timeline_blocks": ([ctypes.POINTER(ctypes.c_int)] * 2, _i32),
    "hsumma_host_row_blocks": ([_vp, _i32, ctypes.POINTER(ctypes.c_int)], _i32),
    "hsumma_host_row_rounds": ([_i32, _i32, _i32, _i32, _vp, _i32, ctypes.POINTER(ctypes.c_int)],
                               _i32),
    "hsumma_candidates": ([_i64, _i64, _i64, _i32, _vp, _i32, ctypes.POINTER(ctypes.c_int)],
                          _i32),
    "hsumma_features": ([_i64, _i64, _i64, _i32, _vp, _i32, _vp], _i32),
    "hsumma_analytic_terms": ([_i64, _i64, _i64, _i32, _vp, _i32, _vp], _i32),
    "hsumma_analytic_load": ([_vp], _i32),
    "hsumma_choose": ([_i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _i32, _i32, _vp,
                       ctypes.POINTER(ctypes.c_int), _vp], _i32),
    "hsumma_peak": ([_i32, _i64, ctypes.POINTER(ctypes.c_double)], _i32),
}


def declared_functions() -> list[str]:
    """Names of the functions include/hsumma.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hsumma_\w+)\s*\(", text)))


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libhsumma is not built ({LIB_PATH} missing); run "
                                   "paper_1306_4161_gb300._build.build()")
            l = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                fn = getattr(l, name)
                fn.argtypes = args
                fn.restype = res
            _lib = l
    return _lib


def last_error() -> str:
    return lib().hsumma_last_error().decode()


def _check(status: int):
    if status != 0:
        raise HsummaError(status, last_error())


_DEFAULT = object()


def _stream_ptr(stream=_DEFAULT):
    """cudaStream_t of a torch stream; torch's current stream by default; None
    is the legacy default stream."""
    if stream is None:
        return ctypes.c_void_p(0)
    import torch
    s = stream if stream is not _DEFAULT else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


_inited = None


def init(device: int = 0, cost_model: bool = True):
    """Initialise the library on a device; with cost_model, load the trained
    model shipped in tuning/cost_model.npz for the automatic configuration
    (when the file is present)."""
    global _inited
    _check(lib().hsumma_init(device))
    if cost_model and _inited != device:
        from . import autotune
        if os.path.exists(autotune.MODEL_PATH):
            autotune.load_into_library(autotune.MODEL_PATH)
    _inited = device


def _ensure_init(t=None):
    if _inited is None:
        dev = t.device.index if (t is not None and t.device.index is not None) else 0
        init(dev)


def finalize():
    global _inited
    lib().hsumma_finalize()
    _inited = None


def mode_code(kind: str | int, slices: int = 0, layout: str = "block") -> int:
    """The mode argument: kind in bits 0..7, slices in 8..15, the layout bit."""
    if layout not in LAYOUTS:
        raise ValueError(f"layout must be one of {sorted(LAYOUTS)} (got {layout!r})")
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    return k | (int(slices) << 8) | LAYOUTS[layout]


def group_shape(P: int, Q: int, G: int):
    """(I, J, cluster_m, cluster_n) for a P x Q grid with G groups."""
    out = [ctypes.c_int() for _ in range(4)]
    _check(lib().hsumma_group_shape(P, Q, G, *[ctypes.byref(o) for o in out]))
    return tuple(o.value for o in out)


def workspace_size(M, N, K, kind="fp64", slices=0) -> int:
    b = ctypes.c_size_t()
    _check(lib().hsumma_workspace_size(M, N, K, mode_code(kind, slices), ctypes.byref(b)))
    return b.value


def _check_f64(t, name):
    import torch
    if t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be 2-D with unit column stride")


def gemm(A, B, *, P=0, Q=0, G=0, b=0, Bouter=0, kind="fp64", slices=0, out=None,
         layout="block", stream=_DEFAULT):
    """C = A x B by HSUMMA on a virtual P x Q grid with G groups (torch tensors on
    the GPU, float64, row-major).  P = Q = G = b = Bouter = 0 (the default) lets
    the library choose them (see choose()).  layout: "block" (block-checkerboard,
    Algorithm 1) or "cyclic" (sub-tiles dealt round robin over the grid)."""
    import torch
    _check_f64(A, "A")
    _check_f64(B, "B")
    M, K = A.shape
    K2, N = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    _ensure_init(A)
    C = out if out is not None else torch.empty((M, N), dtype=torch.float64, device=A.device)
    _check_f64(C, "C")
    lda = A.stride(0) if (M and K) else max(K, 1)
    ldb = B.stride(0) if (K and N) else max(N, 1)
    ldc = C.stride(0) if (M and N) else max(N, 1)
    _check(lib().hsumma_gemm(M, N, K, A.data_ptr(), lda, B.data_ptr(), ldb, C.data_ptr(), ldc,
                             P, Q, G, b, Bouter, mode_code(kind, slices, layout),
                             _stream_ptr(stream)))
    return C


def gemm_host(A, B, C, *, P, Q, G, b, Bouter, kind="fp64", slices=0, layout="block",
              stream=_DEFAULT):
    """The same product from host memory (numpy or CPU torch float64 arrays,
    row-major); C is written in place."""
    def ptr_ld(x):
        if hasattr(x, "data_ptr"):
            return x.data_ptr(), x.stride(0)
        return x.ctypes.data, x.strides[0] // 8
    (pa, la), (pb, lb), (pc, lc) = ptr_ld(A), ptr_ld(B), ptr_ld(C)
    M, K = A.shape
    N = B.shape[1]
    _ensure_init()
    _check(lib().hsumma_gemm_host(M, N, K, pa, la, pb, lb, pc, lc, P, Q, G, b, Bouter,
                                  mode_code(kind, slices, layout), _stream_ptr(stream)))
    return C


def sync(stream=_DEFAULT):
    _check(lib().hsumma_sync(_stream_ptr(stream)))


def launches() -> int:
    """Kernel launches the library has issued for products since it was loaded."""
    return int(lib().hsumma_launches())


def counters() -> dict:
    c = Counters()
    _check(lib().hsumma_get_counters(ctypes.byref(c)))
    return c.as_dict()


# ---- split path, step by step ----
def split_exponents(A, B, stream=_DEFAULT):
    import torch
    _check_f64(A, "A")
    _check_f64(B, "B")
    _ensure_init(A)
    M, K = A.shape
    N = B.shape[1]
    e = torch.empty(M, dtype=torch.int32, device=A.device)
    f = torch.empty(N, dtype=torch.int32, device=A.device)
    _check(lib().hsumma_split_exponents(M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(),
                                        B.stride(0), e.data_ptr(), f.data_ptr(),
                                        _stream_ptr(stream)))
    return e, f


def split_slices(A, B, e, f, kind, S, stream=_DEFAULT):
    import torch
    _ensure_init(A)
    M, K = A.shape
    N = B.shape[1]
    Kp = (K + 63) // 64 * 64
    dt = torch.int8 if kind == "int8" else torch.bfloat16
    As = torch.empty((S, M, Kp), dtype=dt, device=A.device)
    Bs = torch.empty((S, N, Kp), dtype=dt, device=A.device)
    _check(lib().hsumma_split_slices(M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(),
                                     B.stride(0), e.data_ptr(), f.data_ptr(), KINDS[kind], S,
                                     As.data_ptr(), Bs.data_ptr(), _stream_ptr(stream)))
    return As, Bs


def split_planes(K, kind, S) -> int:
    n = lib().hsumma_split_planes(K, KINDS[kind], S)
    if n < 0:
        _check(n)
    return n


def split_diagonals(As, Bs, M, N, K, kind, S, *, P, Q, G, b, Bouter, stream=_DEFAULT):
    import torch
    _ensure_init(As)
    g = split_planes(K, kind, S)
    D = torch.empty((S, g, M, N), dtype=torch.int32, device=As.device)
    _check(lib().hsumma_split_diagonals(M, N, K, KINDS[kind], S, As.data_ptr(), Bs.data_ptr(),
                                        D.data_ptr(), P, Q, G, b, Bouter,
                                        _stream_ptr(stream)))
    return D


def split_recombine(D, e, f, M, N, K, kind, S, stream=_DEFAULT):
    import torch
    _ensure_init(D)
    C = torch.empty((M, N), dtype=torch.float64, device=D.device)
    _check(lib().hsumma_split_recombine(M, N, K, KINDS[kind], S, D.data_ptr(), e.data_ptr(),
                                        f.data_ptr(), C.data_ptr(), max(N, 1),
                                        _stream_ptr(stream)))
    return C


def peak(kind: str, work: int) -> float:
    _ensure_init()
    r = ctypes.c_double()
    _check(lib().hsumma_peak(PEAKS[kind], work, ctypes.byref(r)))
    return r.value


# ---- automatic configuration ----
CHOOSE = {"auto": 0, "model": 1, "timed": 2, "analytic": 3, "verified": 4}
CHOSEN = {0: "cached", 1: "model", 2: "timed", 3: "analytic", 4: "verified"}


def candidates(M, N, K, kind="fp64", slices=0) -> list[tuple[int, int, int, int, int]]:
    """The (P, Q, G, b, Bouter) configurations the automatic choice considers."""
    n = ctypes.c_int()
    _check(lib().hsumma_candidates(M, N, K, mode_code(kind, slices), None, 0, ctypes.byref(n)))
    buf = (ctypes.c_int * (5 * max(n.value, 1)))()
    _check(lib().hsumma_candidates(M, N, K, mode_code(kind, slices), buf, n.value,
                                   ctypes.byref(n)))
    return [tuple(buf[5 * i:5 * i + 5]) for i in range(n.value)]


def features(M, N, K, cfgs, kind="fp64", slices=0):
    """The cost model's raw input features (n x 10 float32) of configurations."""
    import numpy as np
    cfg = np.ascontiguousarray(np.asarray(cfgs, dtype=np.int32).reshape(-1, 5))
    X = np.empty((cfg.shape[0], 10), dtype=np.float32)
    _check(lib().hsumma_features(M, N, K, mode_code(kind, slices), cfg.ctypes.data,
                                 cfg.shape[0], X.ctypes.data))
    return X


def choose(A, B, C=None, *, kind="fp64", slices=0, policy="auto", stream=_DEFAULT):
    """(P, Q, G, b, Bouter) that gemm(A, B) runs with when asked to choose, and
    how it was chosen ("cached", "model", "timed", "analytic" or "verified": the
    model's four best-predicted candidates timed, and outside the model's
    trained range the best of every other cluster shape too).  Timing
    overwrites C."""
    import torch
    _check_f64(A, "A")
    _check_f64(B, "B")
    M, K = A.shape
    N = B.shape[1]
    _ensure_init(A)
    if C is None:
        C = torch.empty((M, N), dtype=torch.float64, device=A.device)
    cfg = (ctypes.c_int * 5)()
    how = ctypes.c_int()
    _check(lib().hsumma_choose(M, N, K, A.data_ptr(), A.stride(0) if (M and K) else max(K, 1),
                               B.data_ptr(), B.stride(0) if (K and N) else max(N, 1),
                               C.data_ptr(), C.stride(0) if (M and N) else max(N, 1),
                               mode_code(kind, slices), CHOOSE[policy], cfg, ctypes.byref(how),
                               _stream_ptr(stream)))
    return tuple(cfg), CHOSEN[how.value]


def load_model(theta, mean, std):
    """Load a trained cost model (9089 parameters, 10 feature means and
    deviations) into the library; theta=None unloads it."""
    import numpy as np
    if theta is None:
        _check(lib().hsumma_mlp_load(None, None, None))
        return
    th = np.ascontiguousarray(theta, dtype=np.float32)
    mu = np.ascontiguousarray(mean, dtype=np.float32)
    sd = np.ascontiguousarray(std, dtype=np.float32)
    if th.size != N_MLP_PARAMS or mu.size != 10 or sd.size != 10:
        raise ValueError("a cost model has 9089 parameters and 10 means and deviations")
    _check(lib().hsumma_mlp_load(th.ctypes.data, mu.ctypes.data, sd.ctypes.data))


def load_model_range(lo, hi):
    """The product features (3 kinds x 10, as features() gives them) the
    loaded model was trained on; outside them the automatic choice is verified
    by timing.  lo=None clears it."""
    import numpy as np
    if lo is None:
        _check(lib().hsumma_mlp_range(None, None))
        return
    a = np.ascontiguousarray(lo, dtype=np.float32)
    b = np.ascontiguousarray(hi, dtype=np.float32)
    if a.shape != (3, 10) or b.shape != (3, 10):
        raise ValueError("a trained range is 3 kinds x 10 features, low and high")
    _check(lib().hsumma_mlp_range(a.ctypes.data, b.ctypes.data))


def in_trained_range(M, N, K, kind="fp64", slices=0) -> bool:
    """Whether the product lies inside the loaded model's trained range (the
    automatic choice takes the model's pick there, else verifies it by timing);
    True when no range is loaded."""
    inside = ctypes.c_int()
    _check(lib().hsumma_mlp_in_range(M, N, K, mode_code(kind, slices), ctypes.byref(inside)))
    return bool(inside.value)


def stage_timing(enable: bool):
    """Start (clearing the record) or stop recording per-stage events in
    hsumma_gemm."""
    _ensure_init()
    _check(lib().hsumma_stage_timing(1 if enable else 0))


def stage_times():
    """(summed ms of the four stages over the recorded calls, number of calls)."""
    ms = (ctypes.c_double * 4)()
    n = ctypes.c_int()
    _check(lib().hsumma_stage_times(ms, ctypes.byref(n)))
    return list(ms), n.value


def host_row_blocks() -> list[int]:
    """First row of each row block of the last gemm_host call ([] if it was
    not pipelined)."""
    r0 = (ctypes.c_int64 * 8)()
    n = ctypes.c_int()
    _check(lib().hsumma_host_row_blocks(r0, 8, ctypes.byref(n)))
    return [int(r0[i]) for i in range(min(n.value, 8))]


def host_row_rounds(P: int, Qc: int, cn: int, resident: int) -> list[int]:
    """Processor rows of the round-aligned row blocks the host pipeline uses
    for products on persistent CTA pairs ([] when no such split exists)."""
    pr = (ctypes.c_int * 8)()
    n = ctypes.c_int()
    _check(lib().hsumma_host_row_rounds(P, Qc, cn, resident, pr, 8, ctypes.byref(n)))
    return [int(pr[i]) for i in range(min(n.value, 8))]


def host_timeline():
    """Phases of the last gemm_host call made with stage timing on, when it was
    pipelined: a list of (name, row block, column block, start ms, end ms)
    relative to the call's first event, name one of "B in", "A in", "product",
    "C out" (block -1 where a phase has no such index); [] otherwise."""
    ms = (ctypes.c_double * 64)()
    n, R, Cb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().hsumma_host_timeline(ms, 64, ctypes.byref(n)))
    _check(lib().hsumma_host_timeline_blocks(ctypes.byref(R), ctypes.byref(Cb)))
    R, Cb = R.value, Cb.value
    names = [("B in", -1, c) for c in range(Cb)] + [("A in", r, -1) for r in range(R)]
    names += [("product", r, c) for r in range(R) for c in range(Cb)]
    names += [("C out", r, c) for r in range(R) for c in range(Cb)]
    return [(nm, r, c, ms[2 * i], ms[2 * i + 1]) for i, (nm, r, c) in enumerate(names[:n.value])]


PAIR_LAUNCH = {"auto": 0, "one": 1, "per_diagonal": 2}
PAIR_PERSISTENT = 0x10


def pair_launch(split=None, persistent=False):
    """Launch policy of the CTA-pair kernel: split in {"auto", "one",
    "per_diagonal"} (None only queries), persistent clusters or not.  Returns
    the previous policy as (split, persistent)."""
    _ensure_init()
    code = -1 if split is None else PAIR_LAUNCH[split] | (PAIR_PERSISTENT if persistent else 0)
    r = lib().hsumma_pair_launch(code)
    if r < 0:
        _check(r)
    names = {v: k for k, v in PAIR_LAUNCH.items()}
    return names[r & 0xf], bool(r & PAIR_PERSISTENT)


def pair_kernel(enable=None) -> bool:
    """Whether bf16 products of groups realised as 2 x 1 clusters run on CTA
    pairs; with enable given, set it.  Returns the previous setting."""
    _ensure_init()
    r = lib().hsumma_pair_kernel(-1 if enable is None else int(bool(enable)))
    if r < 0:
        _check(r)
    return bool(r)


def analytic_terms(M, N, K, cfgs, kind="fp64", slices=0):
    """The analytic model's 5 terms (n x 5 float64) of configurations."""
    import numpy as np
    cfg = np.ascontiguousarray(np.asarray(cfgs, dtype=np.int32).reshape(-1, 5))
    T = np.empty((cfg.shape[0], 5), dtype=np.float64)
    _check(lib().hsumma_analytic_terms(M, N, K, mode_code(kind, slices), cfg.ctypes.data,
                                       cfg.shape[0], T.ctypes.data))
    return T


def load_analytic(coef):
    """Load the analytic model's coefficients (3 kinds x 5 terms); None unloads."""
    import numpy as np
    if coef is None:
        _check(lib().hsumma_analytic_load(None))
        return
    c = np.ascontiguousarray(coef, dtype=np.float64).reshape(3, 5)
    _check(lib().hsumma_analytic_load(c.ctypes.data))
