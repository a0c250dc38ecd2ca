"""CPU oracle for the adaptive k-NN method (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path never does; it shares
no code with the CUDA library. The arithmetic lives in ``knn_oracle.c``
(double precision); this module compiles it with gcc and wraps it with ctypes
and numpy.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knn_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libknn_oracle.so")
_lock = threading.Lock()
_lib = None

BOUND = {"footnote": 0, "lemma": 1, "exp": 2}
STORAGE = {"f32": 0, "bf16": 1, "fp8": 2}
ACTIVE, ELIMINATED, ACCEPTED = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "knn_oracle.h")))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class AdaptiveParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("h", C.c_int32), ("bound", C.c_int32), ("c_alpha", C.c_double),
                ("delta", C.c_double), ("B0", C.c_int32), ("B", C.c_int32), ("grow", C.c_int32),
                ("seed", C.c_uint64), ("qid", C.c_uint64), ("mask_p", C.c_uint64), ("mask_q", C.c_uint64),
                ("tol", C.c_double), ("storage", C.c_int32), ("block", C.c_int32), ("metric", C.c_int32),
                ("sampling", C.c_int32)]


class AdaptiveStats(C.Structure):
    _fields_ = [("evals", C.c_int64), ("rounds", C.c_int32), ("count", C.c_int32), ("term", C.c_int32),
                ("near", C.c_int64), ("near_disagree", C.c_int64), ("mismatch", C.c_int64),
                ("log_inconsistent", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_coordinate.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, C.c_int32,
                                         C.c_uint64, C.c_uint64]
            L.orc_coordinate.restype = C.c_int32
            L.orc_coordinate_wor.argtypes = L.orc_coordinate.argtypes
            L.orc_coordinate_wor.restype = C.c_int32
            L.orc_alpha.argtypes = [C.c_int32, C.c_double, C.c_int64, C.c_int64, C.c_double]
            L.orc_alpha.restype = C.c_double
            L.orc_exact_knn_batch.argtypes = [P, C.c_int64, C.c_int32, P, C.c_int32, C.c_int32, P, P, C.c_int32]
            L.orc_exact_knn_batch_metric.argtypes = [P, C.c_int64, C.c_int32, P, C.c_int32, C.c_int32, C.c_int32, P,
                                                     P, C.c_int32]
            L.orc_adaptive_batch.argtypes = [P, C.c_int64, C.c_int32, P, C.c_int32, C.POINTER(AdaptiveParams),
                                             P, P, P, P, P, P, C.c_int32]
            L.orc_adaptive_batch.restype = C.c_int32
            L.orc_sequential.argtypes = [P, C.c_int64, C.c_int32, P, C.POINTER(AdaptiveParams), C.c_int64,
                                         P, P, P]
            L.orc_sequential.restype = C.c_int32
            L.orc_sequential_heaps.argtypes = L.orc_sequential.argtypes
            L.orc_sequential_heaps.restype = C.c_int32
            L.orc_max_threads.restype = C.c_int32
            L.orc_quantize.argtypes = [C.c_int32, P, C.c_int64, C.c_int32, P, P]
            L.orc_quantize.restype = C.c_double
            L.orc_round_bf16.argtypes = [C.c_float]
            L.orc_round_bf16.restype = C.c_float
            L.orc_round_e4m3.argtypes = [C.c_float]
            L.orc_round_e4m3.restype = C.c_float
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def coordinate(seed, qid, point, s, m, mask_p=(1 << 64) - 1, mask_q=(1 << 64) - 1):
    return lib().orc_coordinate(seed, qid, point, s, m, mask_p, mask_q)


def coordinate_wor(seed, qid, point, s, m, mask_p=(1 << 64) - 1, mask_q=(1 << 64) - 1):
    """The s-th draw (s < m) of a pair sampled without replacement."""
    return lib().orc_coordinate_wor(seed, qid, point, s, m, mask_p, mask_q)


def alpha(form, u, n, delta, c_alpha=1.0):
    return lib().orc_alpha(BOUND[form] if isinstance(form, str) else int(form), float(c_alpha), int(u), int(n),
                           float(delta))


def quantize(X, storage):
    """Dequantised copy of X for a storage format ("f32", "bf16", "fp8"),
    the per-row FP8 scales, and the largest element error."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, m = X.shape
    out = np.empty_like(X)
    scale = np.ones(n, dtype=np.float32)
    emax = lib().orc_quantize(STORAGE[storage], _ptr(X), n, m, _ptr(out), _ptr(scale))
    return out, scale, float(emax)


def max_threads() -> int:
    return int(lib().orc_max_threads())


METRIC = {"l2": 0, "l1": 1}


def exact_knn(X, Q, k, threads=0, metric="l2"):
    """Brute force (Section 3). Returns (idx [nq,k] int64, dist [nq,k] f64):
    squared l2 distances, or l1 distances with metric="l1"."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    Q = np.ascontiguousarray(np.atleast_2d(Q), dtype=np.float32)
    n, m = X.shape
    nq = Q.shape[0]
    idx = np.empty((nq, k), dtype=np.int64)
    dist = np.empty((nq, k), dtype=np.float64)
    lib().orc_exact_knn_batch_metric(_ptr(X), n, m, _ptr(Q), nq, k, METRIC[metric], _ptr(idx), _ptr(dist),
                                     int(threads))
    return idx, dist


def make_params(k, h=None, delta=0.01, bound="footnote", c_alpha=1.0, B0=16, B=16, grow=0, seed=0,
                qid=0, share_points=False, share_queries=False, tol=1e-5, storage="f32", block=1, metric="l2",
                replace=True):
    """Parameters of the batched rounds; `block` = coordinates per sample
    (1: single coordinates as in the paper; g > 1: blocks of g consecutive
    coordinates, B0 and B then count blocks); `replace` = False draws a
    pair's coordinates without replacement (its keyed permutation of [0, m))."""
    full = (1 << 64) - 1
    return AdaptiveParams(int(k), int(k if h is None else h), BOUND[bound] if isinstance(bound, str) else int(bound),
                          float(c_alpha), float(delta), int(B0), int(B), int(grow), int(seed), int(qid),
                          0 if share_points else full, 0 if share_queries else full, float(tol),
                          STORAGE[storage] if isinstance(storage, str) else int(storage), int(block),
                          METRIC[metric] if isinstance(metric, str) else int(metric), 0 if replace else 1)


def adaptive(X, Q, params: AdaptiveParams, replay=None, want_state=True, threads=0):
    """Batched adaptive rounds for every query row of Q (query i has
    qid = params.qid + i). Returns a dict with idx [nq,k+h], code/S/T [nq,n]
    (if want_state) and per-query stats."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    Q = np.ascontiguousarray(np.atleast_2d(Q), dtype=np.float32)
    n, m = X.shape
    nq = Q.shape[0]
    kh = params.k + params.h
    idx = np.empty((nq, kh), dtype=np.int64)
    code = np.empty((nq, n), dtype=np.int32) if want_state else None
    S = np.empty((nq, n), dtype=np.float64) if want_state else None
    T = np.empty((nq, n), dtype=np.int32) if want_state else None
    st = (AdaptiveStats * nq)()
    rp = None
    if replay is not None:
        rp = np.ascontiguousarray(replay, dtype=np.int32)
        assert rp.shape == (nq, n)
    rc = lib().orc_adaptive_batch(_ptr(X), n, m, _ptr(Q), nq, C.byref(params), _ptr(rp), _ptr(idx),
                                  _ptr(code), _ptr(S), _ptr(T), C.cast(st, C.c_void_p), int(threads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return {"idx": idx, "code": code, "S": S, "T": T, "stats": [s.as_dict() for s in st]}


def sequential(X, q, params: AdaptiveParams, max_iter=None, heaps=False):
    """Algorithm 1 as printed, one query. Returns (idx [k+h], evals, iters).
    heaps=True runs the seven-heap implementation (Section 4.1), O(log n)
    per iteration; the default scans the sets, O(n) per iteration."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    q = np.ascontiguousarray(np.ravel(q), dtype=np.float32)
    n, m = X.shape
    kh = params.k + params.h
    idx = np.empty(kh, dtype=np.int64)
    ev = np.zeros(1, dtype=np.int64)
    it = np.zeros(1, dtype=np.int64)
    if max_iter is None:
        max_iter = 4 * n * m + 16
    fn = lib().orc_sequential_heaps if heaps else lib().orc_sequential
    rc = fn(_ptr(X), n, m, _ptr(q), C.byref(params), int(max_iter), _ptr(idx), _ptr(ev), _ptr(it))
    if rc == 1:
        raise ValueError("oracle rejected the arguments")
    return idx, int(ev[0]), int(it[0])
