"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/*.h declares (no compute calls: these run without a GPU)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1902_09465_gb300 import build
    return build.build()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(knn_\w+)\s*\(", text, flags=re.M):
            names.add(mt.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("knn_adaptive", "knn_exact", "knn_rerank", "knn_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_version_and_defaults_without_gpu(lib_path):
    from paper_1902_09465_gb300 import knn
    assert "sm_103a" in knn.version()
    o = knn.Opts()
    knn.lib().knn_opts_default(ctypes.byref(o))
    assert o.h == -1 and o.B0 >= 1 and o.B >= 1 and o.mask_p == (1 << 64) - 1


def test_invalid_arguments_are_rejected_on_the_host(lib_path):
    from paper_1902_09465_gb300 import knn
    L = knn.lib()
    o = knn.Opts()
    L.knn_opts_default(ctypes.byref(o))
    # k > n, delta outside (0,1), m = 0: all refused before any device work
    for (n, m, k, delta) in [(10, 4, 11, 0.1), (10, 4, 2, 1.5), (10, 0, 2, 0.1), (10, 4, 2, 0.0)]:
        rc = L.knn_adaptive(None, n, m, None, 1, k, delta, 0, ctypes.byref(o), None, None, None, None, None,
                            None, None, 0, None)
        assert rc == 1
        assert L.knn_last_error().decode()
    rc = L.knn_rerank(None, 10, 4, None, 1, None, 0, 1, None, None, None)
    assert rc == 1
    # option fields out of range: block above 64, an unknown metric, odd thread counts
    for field, value in (("block", 65), ("block", -1), ("metric", 2), ("threads", 300), ("grow", 2)):
        bad = knn.Opts()
        L.knn_opts_default(ctypes.byref(bad))
        setattr(bad, field, value)
        rc = L.knn_adaptive(None, 100, 8, None, 1, 2, 0.1, 0, ctypes.byref(bad), None, None, None, None, None,
                            None, None, 0, None)
        assert rc == 1, (field, value)
        assert field.split("_")[0] in L.knn_last_error().decode() or L.knn_last_error().decode()
    # sampling: an unknown mode, and without replacement over block samples
    for fields in ({"sampling": 2}, {"sampling": -1}, {"sampling": 1, "block": 8}):
        bad = knn.Opts()
        L.knn_opts_default(ctypes.byref(bad))
        for f, v in fields.items():
            setattr(bad, f, v)
        rc = L.knn_adaptive(None, 100, 8, None, 1, 2, 0.1, 0, ctypes.byref(bad), None, None, None, None, None,
                            None, None, 0, None)
        assert rc == 1 and "sampling" in L.knn_last_error().decode(), fields
    # the no-alloc entry draws with replacement only (refused before any device work)
    wor = knn.Opts()
    L.knn_opts_default(ctypes.byref(wor))
    wor.sampling = 1
    fn = L.knn_adaptive_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                   ctypes.c_double, ctypes.c_uint64, ctypes.POINTER(knn.Opts)] + [ctypes.c_void_p] * 7
    rc = fn(None, 100, 8, None, 1, 2, 0.1, 0, ctypes.byref(wor), None, None, None, None, None, None, None)
    assert rc == 1 and "replacement" in L.knn_last_error().decode()
    rc = L.knn_rerank_metric(None, 10, 4, None, 1, None, 4, 1, 3, None, None, None)
    assert rc == 1 and "metric" in L.knn_last_error().decode()
    o2 = knn.Opts()
    L.knn_opts_default(ctypes.byref(o2))
    assert o2.block == 1 and o2.metric == 0 and o2.sampling == 0


def test_phase_clocks_only_in_the_timing_build(lib_path):
    """The default library has no phase timing: the call is refused on the
    host (no device work); the binding refuses to swap a loaded library."""
    from paper_1902_09465_gb300 import knn
    L = knn.lib()
    v = (ctypes.c_uint64 * 16)()
    assert L.knn_phase_clocks(v, 0) == 4 and "phase timing" in L.knn_last_error().decode()
    assert L.knn_phase_clocks(None, 0) == 1
    with pytest.raises(knn.KnnError):
        knn.phase_clocks()
    with pytest.raises(knn.KnnError):
        knn.use_library(lib_path)


def test_oracle_and_library_share_no_code():
    lib_src = glob.glob(os.path.join(ROOT, "paper_1902_09465_gb300", "**", "*"), recursive=True)
    for f in lib_src:
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(f).read()
            assert "knn_oracle" not in text and "import oracle" not in text and "from oracle" not in text, f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if f.endswith((".py", ".c", ".h")):
            text = open(f).read()
            assert "knn_gb300" not in text and "paper_1902_09465_gb300" not in text, f
