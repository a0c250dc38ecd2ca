"""Thin Python binding of ``libknn_gb300.so`` (C ABI in include/knn_gb300.h).

Argument marshalling only: tensors are checked for device, dtype and layout,
outputs are allocated with torch on the inputs' device, and the library's
entry points are called with raw device pointers on the current torch
stream. Every step of the computation runs in the library's CUDA kernels.
There is no CPU fallback: without the built library every call raises.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libknn_gb300.so")
_lock = threading.Lock()
_lib = None

BOUNDS = {"footnote": 0, "lemma": 1, "exp": 2}
STORAGE = {"f32": 0, "bf16": 1, "fp8": 2}
COPY_SCREEN = 1 << 3
COPY_SCREENS = {"screen": 1 << 3, "screen_f16": 1 << 4, "screen_bf16": 1 << 5}
SCREENS = {"f32": 0, "bf16x3": 1, "f16": 2, "bf16": 3}
ACTIVE, ELIMINATED, ACCEPTED = 0, 1, 2
MAX_KH = 1024  # largest k + h (candidate set size) the library accepts
FULL_MASK = (1 << 64) - 1


class KnnError(RuntimeError):
    pass


class Opts(C.Structure):
    _fields_ = [("h", C.c_int32), ("bound", C.c_int32), ("c_alpha", C.c_double), ("B0", C.c_int32),
                ("B", C.c_int32), ("grow", C.c_int32), ("qid_base", C.c_uint64), ("mask_p", C.c_uint64),
                ("mask_q", C.c_uint64), ("threads", C.c_int32), ("max_ctas", C.c_int32), ("block", C.c_int32),
                ("metric", C.c_int32), ("sampling", C.c_int32), ("r0_tensor", C.c_int32),
                ("query_order", C.c_int32), ("row_pass", C.c_int32)]


_P = C.c_void_p
_SIGS = {
    "knn_opts_default": (None, [C.POINTER(Opts)]),
    "knn_adaptive_workspace_size": (C.c_size_t, [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.POINTER(Opts)]),
    "knn_adaptive": (C.c_int, [_P, C.c_int64, C.c_int32, _P, C.c_int32, C.c_int32, C.c_double, C.c_uint64,
                               C.POINTER(Opts), _P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "knn_rerank": (C.c_int, [_P, C.c_int64, C.c_int32, _P, C.c_int32, _P, C.c_int32, C.c_int32, _P, _P, _P]),
    "knn_rerank_metric": (C.c_int, [_P, C.c_int64, C.c_int32, _P, C.c_int32, _P, C.c_int32, C.c_int32, C.c_int32,
                                    _P, _P, _P]),
    "knn_exact_l1": (C.c_int, [_P, C.c_int64, C.c_int32, _P, C.c_int32, C.c_int32, _P, _P, _P, C.c_size_t, _P]),
    "knn_exact_workspace_size": (C.c_size_t, [C.c_int64, C.c_int32, C.c_int32, C.c_int32]),
    "knn_exact": (C.c_int, [_P, C.c_int64, C.c_int32, _P, C.c_int32, C.c_int32, _P, _P, _P, C.c_size_t, _P]),
    "knn_dataset_create": (C.c_int, [_P, C.c_int64, C.c_int32, C.c_int32, _P, C.POINTER(C.c_void_p)]),
    "knn_dataset_destroy": (C.c_int, [_P]),
    "knn_dataset_error": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_float)]),
    "knn_adaptive_ds": (C.c_int, [_P, C.c_int32, _P, C.c_int32, C.c_int32, C.c_double, C.c_uint64,
                                  C.POINTER(Opts), _P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "knn_exact_ds_workspace_size": (C.c_size_t, [_P, C.c_int32, C.c_int32]),
    "knn_exact_ds": (C.c_int, [_P, C.c_int32, _P, C.c_int32, C.c_int32, _P, _P, _P, C.c_size_t, _P]),
    "knn_device_status": (C.c_int, [C.POINTER(C.c_int32)]),
    "knn_debug_wait_limit": (C.c_int, [C.c_int64]),
    "knn_kernel_timing": (C.c_int, [C.c_int32]),
    "knn_kernel_times": (C.c_int, [C.POINTER(C.c_double), C.c_int32]),
    "knn_phase_clocks": (C.c_int, [C.POINTER(C.c_uint64), C.c_int32]),
    "knn_adaptive_ds_multi_workspace_size": (C.c_size_t, [_P, C.c_int32, C.c_int32, C.POINTER(Opts)]),
    "knn_adaptive_ds_multi": (C.c_int, [_P, C.c_int32, _P, C.c_int32, _P, C.c_int32, _P, C.c_double, C.c_uint64,
                                        C.POINTER(Opts), _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "knn_dataset_share": (C.c_int, [_P, C.c_uint64, C.c_int32, _P]),
    "knn_philox_blocks": (C.c_int, [C.c_int64, C.c_int32, _P, _P]),
    "knn_last_error": (C.c_char_p, []),
    "knn_version": (C.c_char_p, []),
}


def use_library(path: str) -> None:
    """Load ``path`` (a build of the same library, e.g. the phase-timing one)
    in place of the default; only before the first call into the library."""
    global LIB_PATH
    with _lock:
        if _lib is not None:
            raise KnnError("the library is already loaded")
        LIB_PATH = path


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise KnnError(f"{LIB_PATH} is missing: build it with paper_1902_09465_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        msg = lib().knn_last_error().decode()
        raise KnnError(f"knn status {rc}: {msg}")


def _dev(t: torch.Tensor, name: str, dtype=torch.float32):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise KnnError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise KnnError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise KnnError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


METRICS = {"l2": 0, "l1": 1}


def make_opts(k, h=None, bound="footnote", c_alpha=1.0, B0=16, B=16, grow=0, qid_base=0, share_points=False,
              share_queries=False, max_ctas=0, threads=0, block=1, metric="l2", replace=True,
              r0_tensor=False, query_order=True, row_pass=True) -> Opts:
    """knn_opts for a call; `block` = coordinates per sample (1: single
    coordinates; g > 1: blocks of g consecutive coordinates, B0 and B then
    count blocks); `metric` = "l2" (squared l2, the paper's) or "l1";
    `replace` = False draws each pair's coordinates without replacement;
    `r0_tensor` = True forms round 0 under shared coordinates as a
    tensor-core contraction (knn_opts.r0_tensor); `query_order` = False
    keeps the batch order of dataset calls (knn_opts.query_order);
    `row_pass` = False makes every round gather its own draws
    (knn_opts.row_pass; the results are the same)."""
    o = Opts()
    lib().knn_opts_default(C.byref(o))
    o.h = -1 if h is None else int(h)
    o.bound = BOUNDS[bound] if isinstance(bound, str) else int(bound)
    o.c_alpha = float(c_alpha)
    o.B0, o.B, o.grow = int(B0), int(B), int(grow)
    o.qid_base = int(qid_base)
    o.mask_p = 0 if share_points else FULL_MASK
    o.mask_q = 0 if share_queries else FULL_MASK
    o.max_ctas = int(max_ctas)
    o.threads = int(threads)
    o.block = int(block)
    o.metric = METRICS[metric] if isinstance(metric, str) else int(metric)
    o.sampling = 0 if replace else 1
    o.r0_tensor = 1 if r0_tensor else 0
    o.query_order = 1 if query_order else 0
    o.row_pass = 1 if row_pass else 0
    return o


def adaptive_workspace_size(n, m, nq, k, opts: Opts) -> int:
    return int(lib().knn_adaptive_workspace_size(int(n), int(m), int(nq), int(k), C.byref(opts)))


def adaptive(X: torch.Tensor, Q: torch.Tensor, k: int, delta: float = 0.01, seed: int = 0, *, trace: bool = False,
             workspace: torch.Tensor | None = None, stream=None, out=None, **opt_kw):
    """Batched adaptive rounds for every row of Q against X (knn_adaptive).

    Returns a dict: idx [nq, k+h] int64 (-1 padded), count [nq] int32,
    evals [nq] int64, rounds [nq] int32 and, with trace=True, code [nq, n]
    int32 (4*round + kind) and S [nq, n] float32.
    """
    n, m = X.shape
    nq = Q.shape[0]
    if Q.shape[1] != m:
        raise KnnError("X and Q must have the same number of columns")
    o = make_opts(k, **opt_kw)
    h = k if o.h < 0 else o.h
    dev = X.device
    if out is None:
        out = {"idx": torch.empty((nq, k + h), dtype=torch.int64, device=dev),
               "count": torch.empty(nq, dtype=torch.int32, device=dev),
               "evals": torch.empty(nq, dtype=torch.int64, device=dev),
               "rounds": torch.empty(nq, dtype=torch.int32, device=dev)}
    if trace:
        out["code"] = torch.empty((nq, n), dtype=torch.int32, device=dev)
        out["S"] = torch.empty((nq, n), dtype=torch.float32, device=dev)
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        ws_ptr, ws_bytes = _dev(workspace, "workspace", torch.uint8), workspace.numel()
    rc = lib().knn_adaptive(_dev(X, "X"), n, m, _dev(Q, "Q"), nq, int(k), float(delta), int(seed), C.byref(o),
                            _dev(out["idx"], "idx", torch.int64), _dev(out["count"], "count", torch.int32),
                            _dev(out["evals"], "evals", torch.int64), _dev(out["rounds"], "rounds", torch.int32),
                            _dev(out["code"], "code", torch.int32) if trace else None,
                            _dev(out["S"], "S") if trace else None, ws_ptr, ws_bytes, _stream(stream))
    _check(rc)
    return out


def _alloc_out(nq, n, kh, dev, trace):
    out = {"idx": torch.empty((nq, kh), dtype=torch.int64, device=dev),
           "count": torch.empty(nq, dtype=torch.int32, device=dev),
           "evals": torch.empty(nq, dtype=torch.int64, device=dev),
           "rounds": torch.empty(nq, dtype=torch.int32, device=dev)}
    if trace:
        out["code"] = torch.empty((nq, n), dtype=torch.int32, device=dev)
        out["S"] = torch.empty((nq, n), dtype=torch.float32, device=dev)
    return out


class Dataset:
    """A resident dataset (knn_dataset_create): the data range and, on
    request, BF16 / FP8 copies. X must stay alive and unchanged while the
    dataset is used; the object keeps a reference to it."""

    def __init__(self, X: torch.Tensor, copies=("bf16", "fp8"), stream=None):
        mask = 0
        for c in copies:
            mask |= COPY_SCREENS[c] if c in COPY_SCREENS else 1 << STORAGE[c]
        self.X = X
        self.n, self.m = X.shape
        self.copies = tuple(copies)
        h = C.c_void_p()
        _check(lib().knn_dataset_create(_dev(X, "X"), self.n, self.m, mask, _stream(stream), C.byref(h)))
        self._h = h

    def error(self, storage: str) -> float:
        """Largest |copy - X| of a copy (0 for f32)."""
        v = C.c_float()
        _check(lib().knn_dataset_error(self._h, STORAGE[storage], C.byref(v)))
        return float(v.value)

    def adaptive(self, Q: torch.Tensor, k: int, delta: float = 0.01, seed: int = 0, *, storage: str = "f32",
                 trace: bool = False, workspace: torch.Tensor | None = None, stream=None, out=None, **opt_kw):
        """knn_adaptive_ds: the adaptive rounds gathering from the chosen copy."""
        nq = Q.shape[0]
        o = make_opts(k, **opt_kw)
        h = k if o.h < 0 else o.h
        if out is None or (trace and "code" not in out):
            out = _alloc_out(nq, self.n, k + h, Q.device, trace)
        ws_ptr, ws_bytes = None, 0
        if workspace is not None:
            ws_ptr, ws_bytes = _dev(workspace, "workspace", torch.uint8), workspace.numel()
        rc = lib().knn_adaptive_ds(self._h, STORAGE[storage], _dev(Q, "Q"), nq, int(k), float(delta), int(seed),
                                   C.byref(o), _dev(out["idx"], "idx", torch.int64),
                                   _dev(out["count"], "count", torch.int32), _dev(out["evals"], "evals", torch.int64),
                                   _dev(out["rounds"], "rounds", torch.int32),
                                   _dev(out["code"], "code", torch.int32) if trace else None,
                                   _dev(out["S"], "S") if trace else None, ws_ptr, ws_bytes, _stream(stream))
        _check(rc)
        return out

    def share(self, seed: int, copies=("f32",), stream=None):
        """knn_dataset_share: shared-coordinate copies for `seed` (used by
        adaptive calls with share_points=True, share_queries=True and that seed)."""
        mask = 0
        for c in copies:
            mask |= 1 << STORAGE[c]
        _check(lib().knn_dataset_share(self._h, int(seed), mask, _stream(stream)))

    def multi_workspace_size(self, nq: int, k_max: int, **opt_kw) -> int:
        o = make_opts(k_max, **opt_kw)
        return int(lib().knn_adaptive_ds_multi_workspace_size(self._h, int(nq), int(k_max), C.byref(o)))

    def adaptive_multi(self, Q: torch.Tensor, ks: torch.Tensor, k_max: int, qids: torch.Tensor, delta: float = 0.01,
                       seed: int = 0, *, storage: str = "f32", workspace: torch.Tensor | None = None, stream=None,
                       out=None, **opt_kw):
        """knn_adaptive_ds_multi: a mixed batch, query q with its own k
        (ks[q], int32 on the device) and Philox query id (qids[q], int64 on
        the device). Rows of idx are k_max + h_max long."""
        nq = Q.shape[0]
        o = make_opts(k_max, **opt_kw)
        h_max = k_max if o.h < 0 else o.h
        if out is None:
            out = _alloc_out(nq, self.n, k_max + h_max, Q.device, False)
        ws_ptr, ws_bytes = None, 0
        if workspace is not None:
            ws_ptr, ws_bytes = _dev(workspace, "workspace", torch.uint8), workspace.numel()
        rc = lib().knn_adaptive_ds_multi(self._h, STORAGE[storage], _dev(Q, "Q"), nq, _dev(ks, "ks", torch.int32),
                                         int(k_max), _dev(qids, "qids", torch.int64), float(delta), int(seed),
                                         C.byref(o), _dev(out["idx"], "idx", torch.int64),
                                         _dev(out["count"], "count", torch.int32),
                                         _dev(out["evals"], "evals", torch.int64),
                                         _dev(out["rounds"], "rounds", torch.int32), ws_ptr, ws_bytes,
                                         _stream(stream))
        _check(rc)
        return out

    def best_screen(self) -> str:
        """The fastest screen whose operand the dataset holds: FP16, then
        BF16x3, then single BF16, else the FP32 SIMT screen."""
        for copy, screen in (("screen_f16", "f16"), ("screen", "bf16x3"), ("screen_bf16", "bf16")):
            if copy in self.copies:
                return screen
        return "f32"

    def exact_workspace_size(self, nq: int, screen: str | None = None) -> int:
        screen = screen or self.best_screen()
        return int(lib().knn_exact_ds_workspace_size(self._h, SCREENS[screen], int(nq)))

    def exact(self, Q: torch.Tensor, k: int, screen: str | None = None, workspace: torch.Tensor | None = None,
              stream=None):
        """knn_exact_ds: the naive exact method with the chosen screen (by
        default the fastest one the dataset holds, best_screen()).
        Returns (idx [nq,k] int64, dist [nq,k] f64)."""
        screen = screen or self.best_screen()
        nq = Q.shape[0]
        idx = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
        dist = torch.empty((nq, k), dtype=torch.float64, device=Q.device)
        ws_ptr, ws_bytes = None, 0
        if workspace is not None:
            ws_ptr, ws_bytes = _dev(workspace, "workspace", torch.uint8), workspace.numel()
        _check(lib().knn_exact_ds(self._h, SCREENS[screen], _dev(Q, "Q"), nq, int(k), _dev(idx, "idx", torch.int64),
                                  _dev(dist, "dist", torch.float64), ws_ptr, ws_bytes, _stream(stream)))
        return idx, dist

    def close(self):
        if getattr(self, "_h", None):
            lib().knn_dataset_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rerank(X: torch.Tensor, Q: torch.Tensor, cand: torch.Tensor, k: int, stream=None, metric="l2"):
    """Exact FP64 distances of the candidates of each query, top-k by
    (distance, index) (knn_rerank_metric; squared l2 or l1 distances).
    Returns (idx [nq,k] int64, dist [nq,k] f64)."""
    n, m = X.shape
    nq, ncand = cand.shape
    idx = torch.empty((nq, k), dtype=torch.int64, device=X.device)
    dist = torch.empty((nq, k), dtype=torch.float64, device=X.device)
    rc = lib().knn_rerank_metric(_dev(X, "X"), n, m, _dev(Q, "Q"), nq, _dev(cand, "cand", torch.int64), ncand,
                                 int(k), METRICS[metric], _dev(idx, "idx", torch.int64),
                                 _dev(dist, "dist", torch.float64), _stream(stream))
    _check(rc)
    return idx, dist


def exact_workspace_size(n, m, nq, k) -> int:
    return int(lib().knn_exact_workspace_size(int(n), int(m), int(nq), int(k)))


def exact(X: torch.Tensor, Q: torch.Tensor, k: int, workspace: torch.Tensor | None = None, stream=None,
          metric="l2"):
    """Naive exact k-NN (knn_exact; knn_exact_l1 with metric="l1").
    Returns (idx [nq,k] int64, dist [nq,k] f64)."""
    n, m = X.shape
    nq = Q.shape[0]
    idx = torch.empty((nq, k), dtype=torch.int64, device=X.device)
    dist = torch.empty((nq, k), dtype=torch.float64, device=X.device)
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        ws_ptr, ws_bytes = _dev(workspace, "workspace", torch.uint8), workspace.numel()
    fn = lib().knn_exact_l1 if metric == "l1" else lib().knn_exact
    rc = fn(_dev(X, "X"), n, m, _dev(Q, "Q"), nq, int(k), _dev(idx, "idx", torch.int64),
            _dev(dist, "dist", torch.float64), ws_ptr, ws_bytes, _stream(stream))
    _check(rc)
    return idx, dist


def debug_wait_limit(tries: int) -> None:
    """Test hook: the tensor-core kernels' pipeline waits give up after
    `tries` polls (negative: the default) -- knn_debug_wait_limit."""
    _check(lib().knn_debug_wait_limit(int(tries)))


def kernel_timing(enable: bool) -> None:
    """knn_kernel_timing: record CUDA events around the round-0 pass and the
    round-loop kernel of later adaptive dataset calls (not while capturing)."""
    _check(lib().knn_kernel_timing(1 if enable else 0))


def kernel_times(reset: bool = True):
    """knn_kernel_times: (round-0 pass ms, round-loop ms) summed over the
    calls since the last reset."""
    out = (C.c_double * 2)()
    _check(lib().knn_kernel_times(out, 1 if reset else 0))
    return float(out[0]), float(out[1])


def philox_blocks(iters: int, ctas: int, out: torch.Tensor, stream=None) -> None:
    """knn_philox_blocks: ctas x 1024 threads each evaluate `iters` blocks of
    the coordinate generator; out is an int32 CUDA tensor of ctas*1024."""
    if out.numel() < ctas * 1024:
        raise KnnError("out holds fewer than ctas * 1024 words")
    _check(lib().knn_philox_blocks(int(iters), int(ctas), _dev(out, "out", torch.int32), _stream(stream)))


def device_status() -> int:
    """Library status of the current device (waits for the device, clears it):
    nonzero if a kernel gave up a bounded wait."""
    v = C.c_int32()
    _check(lib().knn_device_status(C.byref(v)))
    return int(v.value)


PHASES = ("setup", "gather", "exact", "select", "thresholds", "decide_compact", "output")


def phase_clocks(reset: bool = False) -> dict:
    """Round-loop phase clock totals (a library built with phase timing only;
    the default one raises): {"rounds": {phase: clocks}, "round0": {...}}."""
    v = (C.c_uint64 * 16)()
    _check(lib().knn_phase_clocks(v, 1 if reset else 0))
    return {"rounds": {name: int(v[i]) for i, name in enumerate(PHASES)},
            "round0": {name: int(v[8 + i]) for i, name in enumerate(PHASES[:6])}}


def version() -> str:
    return lib().knn_version().decode()
